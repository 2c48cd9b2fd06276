"""NUFFT synthesis (Sec. 2.5, 3.4, Algorithm 3) on the GPU against the oracle.

The level images of NUFFT synthesis are the type-3 sums of the level's
Gram-corrected visibilities over all baselines; the oracle evaluates that sum
directly (and the CPU tests pin it to the standard-synthesis images). The GPU
path approximates it with a type-3 NUFFT of tolerance eps. Per level, the L2
error must stay within 10 eps of max(||I_l||, ||V'_l||_F sqrt(n_pix)) plus
2e-6 ||I_l|| for the FP32 grids: the FP64 oracle NUFFT stays within 5 eps of
that scale (CPU pin); weak levels, whose images cancel, are measured against the
size of their strengths.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import nufft as onu
from paper_2310_09200_b300 import bipp_ss, inputs
from tests import helpers

pytestmark = pytest.mark.gpu


def _check(got, want, scale, eps):
    """Per-level L2 error within 10 eps max(||want_l||, scale_l) + 2e-6 ||want_l||."""
    nw = np.linalg.norm(want, axis=0)
    err = np.linalg.norm(got - want, axis=0)
    bound = 10 * eps * np.maximum(nw, scale) + 2e-6 * nw
    assert np.all(err <= bound), (err / nw, bound / nw)


def _direct(pix, wl, bounds, n_eig, st, vis, **kw):
    return onu.nufft_levels_with_scale(pix, wl, bounds, n_eig, st, vis, **kw)


@pytest.fixture(scope="module")
def small():
    inp = inputs.make_nufft_config(n_t=3, n_side=40, n_st=48)
    inp.n_eig = 16
    return inp


@pytest.mark.parametrize("eps", [1e-3, 1e-5])
def test_nufft_matches_direct_sum(small, eps):
    inp = small
    b, _ = helpers.oracle_prepass_bounds(inp)
    want, scale = _direct(inp.pix, inp.wl, b, 16, inp.st_xyz, inp.vis)
    with bipp_ss.StandardSynthesis(inp.pix, inp.wl, b, n_eig=16, synthesis="nufft", nufft_eps=eps) as ss:
        ss.collect_batch(inp.st_xyz, inp.vis)
        got = ss.get()
        assert ss.timings()["launches"] > 9
    _check(got, want, scale, eps)


@pytest.mark.parametrize("filt,gi,n_level", [("std", False, 1), ("lsq", True, 3), ("lsq", False, 5)])
def test_nufft_filters_gram_identity_and_level_counts(small, filt, gi, n_level):
    inp = small
    mus = []
    for p, V in zip(inp.st_xyz, inp.vis):
        G = None if gi else oracle.gram(p, inp.wl)
        mus.extend(oracle.geneig(V, G)[0][:16])
    b = bipp_ss.quantile_level_bounds(mus, n_level)
    want, scale = _direct(inp.pix, inp.wl, b, 16, inp.st_xyz, inp.vis, filter=filt, gram_identity=gi)
    with bipp_ss.StandardSynthesis(inp.pix, inp.wl, b, n_eig=16, synthesis="nufft", nufft_eps=1e-5, filter=filt,
                                   gram_identity=gi) as ss:
        ss.collect_batch(inp.st_xyz, inp.vis)
        got = ss.get()
    _check(got, want, scale, 1e-5)


def test_nufft_agrees_with_standard_synthesis_on_gpu(small):
    inp = small
    b, _ = helpers.oracle_prepass_bounds(inp)
    _, scale = _direct(inp.pix[:1], inp.wl, b, 16, inp.st_xyz, inp.vis)
    scale *= np.sqrt(inp.pix.shape[0])
    imgs = {}
    for syn in ("standard", "nufft"):
        with bipp_ss.StandardSynthesis(inp.pix, inp.wl, b, n_eig=16, synthesis=syn, precision="fp64") as ss:
            ss.collect_batch(inp.st_xyz, inp.vis)
            imgs[syn] = ss.get()
    _check(imgs["nufft"], imgs["standard"], scale, 1e-5)


def test_nufft_ragged_steps_and_channels():
    rng = np.random.default_rng(77)
    base = inputs.make_nufft_config(n_t=4, n_side=32, n_st=64)
    wls = [2.0, 3.0]
    st, vis, ne, chan = [], [], [], []
    for t, n in enumerate([40, 64, 23, 51]):
        keep = np.sort(rng.choice(64, n, replace=False))
        st.append(base.st_xyz[t][keep])
        vis.append(base.vis[t][np.ix_(keep, keep)])
        ne.append([12, 20, 7, 16][t])
        chan.append(0 if t < 2 else 1)
    b = np.array([[1e3, np.inf], [-np.inf, 1e3]])
    bounds = np.stack([b, b])
    want, scale = [], []
    for c in range(2):
        img, sc2 = None, 0.0
        for t in range(4):
            if chan[t] != c:
                continue
            f, sc = onu.nufft_levels_with_scale(base.pix, wls[c], b, ne[t], [st[t]], [vis[t]])
            img = f if img is None else img + f
            sc2 = sc2 + sc ** 2
        want.append(img)
        scale.append(np.sqrt(sc2))
    h = bipp_ss.bipp_ss_create_channels(base.pix, np.array(wls), bounds, n_eig=20, synthesis="nufft",
                                        nufft_eps=1e-5)
    try:
        bipp_ss.bipp_ss_collect_channels(h, chan, st, vis, n_eig=ne)
        got = bipp_ss.bipp_ss_get_f64(h, base.pix.shape[0], 2, 2)  # (chan, pix, level)
    finally:
        bipp_ss.bipp_ss_destroy(h)
    for c in range(2):
        _check(got[c], want[c], scale[c], 1e-5)


def test_nufft_single_station_is_the_zero_baseline_term():
    pix = inputs.pixel_grid(8, 1.0)
    p = np.array([[10.0, -3.0, 1.0]])
    V = np.array([[2.5 + 0j]])
    b = np.array([[-np.inf, np.inf]])
    want, *_ = onu.nufft_levels(pix, 2.0, b, 1, p, V)
    with bipp_ss.StandardSynthesis(pix, 2.0, b, n_eig=1, synthesis="nufft") as ss:
        ss.collect_batch([p], [V])
        got = ss.get()
    np.testing.assert_allclose(got, want, rtol=1e-12)


def test_nufft_failed_batch_leaves_images_unchanged(small):
    inp = small
    b, _ = helpers.oracle_prepass_bounds(inp)
    with bipp_ss.StandardSynthesis(inp.pix, inp.wl, b, n_eig=16, synthesis="nufft") as ss:
        ss.collect_batch(inp.st_xyz[:1], inp.vis[:1])
        before = ss.get()
        st_bad = inp.st_xyz[1].copy()
        st_bad[1] = st_bad[0]  # two stations at one position: the Gram matrix is singular
        with pytest.raises(bipp_ss.BippError) as e:
            ss.collect_batch([st_bad], [inp.vis[1]])
        assert e.value.code == bipp_ss.BIPP_ERR_GRAM_NOT_PD
        np.testing.assert_array_equal(ss.get(), before)


def test_nufft_benchmark_workload_sampled_pixels():
    """512 stations, 1024^2 pixels of 4 arcsec, N_eig 64, 4 levels, the
    benchmark's kernels and grid shapes (here over 4 of its 50 steps): sampled
    pixels against the oracle's standard synthesis (equal to the type-3 sum)."""
    inp = inputs.make_nufft_config(n_t=4)
    n_pix = inp.pix.shape[0]
    rng = np.random.default_rng(9)
    sample = np.unique(np.concatenate([rng.choice(n_pix, 200, replace=False), np.arange(0, 1024),
                                       np.arange(n_pix - 1024, n_pix, 7)]))
    bounds, _ = helpers.oracle_prepass_bounds(inp)
    want, sc2 = None, 0.0
    for p, V in zip(inp.st_xyz, inp.vis):
        want, mu, lev, W = oracle.ss_step(inp.pix[sample], inp.wl, bounds, inp.n_eig, p, V, img=want)
        sc2 = sc2 + onu.error_scale(W, mu, lev, 4, len(sample)) ** 2
    with bipp_ss.StandardSynthesis(inp.pix, inp.wl, bounds, n_eig=inp.n_eig, synthesis="nufft", nufft_eps=1e-5,
                                   eig_mode="mixed") as ss:
        ss.collect_batch(inp.st_xyz, inp.vis)
        got = ss.get()
    _check(got[sample], want, np.sqrt(sc2), 1e-5)


@pytest.mark.parametrize("part", [(3, 2, 1, 2, 2, 1), (1, 4, 2, 1, 1, 3), (2, 2, 2, 3, 1, 1)])
def test_nufft_domain_partitioning(small, part):
    """Sec. 3.4.1: input (baseline) cells x image cells, one transform per
    non-empty pair; the images match the unpartitioned sum."""
    inp = small
    b, _ = helpers.oracle_prepass_bounds(inp)
    want, scale = _direct(inp.pix, inp.wl, b, 16, inp.st_xyz, inp.vis)
    with bipp_ss.StandardSynthesis(inp.pix, inp.wl, b, n_eig=16, synthesis="nufft", nufft_eps=1e-5,
                                   nufft_partition=part) as ss:
        ss.collect_batch(inp.st_xyz, inp.vis)
        got = ss.get()
    _check(got, want, scale, 1e-5)


def test_nufft_partitioned_benchmark_workload_sampled_pixels():
    """The paper's setting, input and image partitions of (4, 4, 1), on the
    benchmark workload (4 of its 50 steps), sampled pixels against the oracle."""
    inp = inputs.make_nufft_config(n_t=4)
    n_pix = inp.pix.shape[0]
    rng = np.random.default_rng(11)
    sample = np.unique(np.concatenate([rng.choice(n_pix, 300, replace=False), np.arange(255 * 1024, 257 * 1024, 3)]))
    bounds, _ = helpers.oracle_prepass_bounds(inp)
    want, sc2 = None, 0.0
    for p, V in zip(inp.st_xyz, inp.vis):
        want, mu, lev, W = oracle.ss_step(inp.pix[sample], inp.wl, bounds, inp.n_eig, p, V, img=want)
        sc2 = sc2 + onu.error_scale(W, mu, lev, 4, len(sample)) ** 2
    with bipp_ss.StandardSynthesis(inp.pix, inp.wl, bounds, n_eig=inp.n_eig, synthesis="nufft", nufft_eps=1e-5,
                                   eig_mode="mixed", nufft_partition=(4, 4, 1, 4, 4, 1)) as ss:
        ss.collect_batch(inp.st_xyz, inp.vis)
        got = ss.get()
    _check(got[sample], want, np.sqrt(sc2), 1e-5)


@pytest.mark.parametrize("eps", [1e-7, 3e-2])
def test_nufft_kernel_width_extremes(small, eps):
    """The widest kernel (eps 1e-7: w = 8, 512-cell footprints) and a narrow one
    (eps 3e-2: w = 3); below ~1e-6 the FP32 grids set the floor."""
    inp = small
    b, _ = helpers.oracle_prepass_bounds(inp)
    want, scale = _direct(inp.pix, inp.wl, b, 16, inp.st_xyz, inp.vis)
    with bipp_ss.StandardSynthesis(inp.pix, inp.wl, b, n_eig=16, synthesis="nufft", nufft_eps=eps) as ss:
        ss.collect_batch(inp.st_xyz, inp.vis)
        got = ss.get()
    _check(got, want, scale, max(eps, 1e-6))


def test_nufft_sixteen_levels(small):
    """16 levels (four spreading passes of 4 interleaved levels), one eigenpair
    or none per level."""
    inp = small
    mus = []
    for p, V in zip(inp.st_xyz, inp.vis):
        mus.extend(oracle.geneig(V, oracle.gram(p, inp.wl))[0][:16])
    b = bipp_ss.quantile_level_bounds(mus, 16)
    want, scale = _direct(inp.pix, inp.wl, b, 16, inp.st_xyz, inp.vis)
    with bipp_ss.StandardSynthesis(inp.pix, inp.wl, b, n_eig=16, synthesis="nufft", nufft_eps=1e-5) as ss:
        ss.collect_batch(inp.st_xyz, inp.vis)
        got = ss.get()
    assert got.shape == want.shape == (inp.pix.shape[0], 16)
    _check(got, want, scale, 1e-5)
