"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle on
the same seeded inputs (element by element per level image), plus the
method's invariants and error paths.

Tolerances (relative L2 per level image, ||I_gpu - I_orc|| / ||I_orc||):
  FP64 path        1e-9   (FP64 end to end; Jacobi stop 1e-13 vs oracle 1e-14)
  FP32 path        1e-5   (exact phase reduction + SFU sincos + FP32 sums)
  split-BF16 path  1e-3
  split-FP16 path  1e-5
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2310_09200_b300 import bipp_ss, inputs
from tests import helpers

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-9, "fp32": 1e-5, "split_bf16": 1e-3, "split_fp16": 1e-5}


def rel_l2_per_level(a, b):
    return np.array([np.linalg.norm(a[:, l] - b[:, l]) / max(np.linalg.norm(b[:, l]), 1e-300)
                     for l in range(b.shape[1])])


def oracle_images(inp, bounds, n_eig=None, filter="lsq", gram_identity=False, pix=None, steps=None):
    pix = inp.pix if pix is None else pix
    img = None
    mus, levs = [], []
    steps = range(inp.n_t) if steps is None else steps
    for t in steps:
        ne = n_eig[t] if isinstance(n_eig, (list, np.ndarray)) else (n_eig or inp.n_eig)
        img, mu, lev, _ = oracle.ss_step(pix, inp.wl, bounds, ne, inp.st_xyz[t], inp.vis[t], img=img,
                                         filter=filter, gram_identity=gram_identity)
        mus.append(mu)
        levs.append(lev)
    return img, mus, levs


@pytest.fixture(scope="module")
def cfg0():
    inp = inputs.make_config(0)
    bounds, pooled = helpers.oracle_prepass_bounds(inp)
    assert helpers.min_edge_margin(pooled, bounds) > 1e-9
    img, mus, levs = oracle_images(inp, bounds)
    return inp, bounds, img, mus, levs


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_config0_end_to_end(cfg0, precision):
    inp, bounds, want, mus, levs = cfg0
    with bipp_ss.StandardSynthesis(inp.pix, inp.wl, bounds, n_eig=inp.n_eig, precision=precision) as ss:
        for p, V in zip(inp.st_xyz, inp.vis):
            ss.collect(p, V)
        got = ss.get()
        nt, nk, mu, lev = bipp_ss.bipp_ss_last_eigvals(ss.h, 1, inp.n_eig)
    err = rel_l2_per_level(got, want)
    assert np.all(err <= TOL[precision]), err
    np.testing.assert_allclose(mu[0], mus[-1], rtol=1e-11, atol=1e-11 * abs(mus[-1]).max())
    assert list(lev[0]) == list(levs[-1])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_config0_batched_equals_stepwise(cfg0, precision):
    inp, bounds, want, _, _ = cfg0
    with bipp_ss.StandardSynthesis(inp.pix, inp.wl, bounds, n_eig=inp.n_eig, precision=precision) as ss:
        ss.collect_batch(inp.st_xyz, inp.vis)
        got = ss.get()
        t = ss.timings()
    assert np.all(rel_l2_per_level(got, want) <= TOL[precision])
    assert t["sweeps_total"] >= inp.n_t and t["synth_ms"] > 0 and t["launches"] == 9


def test_ragged_batch_identity_gram_std_filter():
    """Ragged station counts (odd ones exercise the phantom Jacobi index),
    ragged n_eig, G = I, STD filter, pixel count not a multiple of the tile."""
    rng = np.random.default_rng(21)
    base = inputs.make_config(0, n_t=3, n_side=13)
    st, vis, ne = [], [], []
    for t, n in enumerate([17, 24, 13]):
        keep = np.sort(rng.choice(24, n, replace=False))
        st.append(base.st_xyz[t][keep])
        vis.append(base.vis[t][np.ix_(keep, keep)])
        ne.append([9, 24, 5][t])
    inp = inputs.SSInput("ragged", base.wl, base.pix, st, vis, 24, 3)
    bounds = np.array([[50.0, np.inf], [0.0, 50.0], [-np.inf, 0.0]])
    want, _, _ = oracle_images(inp, bounds, n_eig=ne, filter="std", gram_identity=True)
    for precision in ("fp64", "fp32"):
        with bipp_ss.StandardSynthesis(inp.pix, inp.wl, bounds, precision=precision, filter="std",
                                       gram_identity=1) as ss:
            ss.collect_batch(st, vis, n_eig=ne)
            got = ss.get()
        err = rel_l2_per_level(got, want)
        assert np.all(err <= TOL[precision]), (precision, err)


def test_ragged_batch_sinc_gram_odd_station_counts():
    rng = np.random.default_rng(22)
    base = inputs.make_config(0, n_t=3, n_side=9)
    st, vis = [], []
    for t, n in enumerate([23, 19, 21]):
        keep = np.sort(rng.choice(24, n, replace=False))
        st.append(base.st_xyz[t][keep])
        vis.append(base.vis[t][np.ix_(keep, keep)])
    inp = inputs.SSInput("ragged_sinc", base.wl, base.pix, st, vis, 7, 2)
    bounds = np.array([[30.0, np.inf], [-np.inf, 30.0]])
    want, _, _ = oracle_images(inp, bounds)
    with bipp_ss.StandardSynthesis(inp.pix, inp.wl, bounds, n_eig=7, precision="fp64") as ss:
        ss.collect_batch(st, vis)
        got = ss.get()
    assert np.all(rel_l2_per_level(got, want) <= TOL["fp64"])


def test_full_station_count_sampled_pixels():
    """512 stations (SKA-Low-like layout to 65 km), 2 steps, a strided 64 x 64
    subset of the 1024^2 grid plus its ragged last 37 pixels."""
    inp = inputs.make_config(1, n_t=2)
    side = inp.extra["n_side"]
    sel = (np.arange(0, side, 16)[:, None] * side + np.arange(0, side, 16)[None, :]).ravel()
    sel = np.concatenate([sel, np.arange(side * side - 37, side * side)])
    pix = inp.pix[sel]
    bounds, pooled = helpers.oracle_prepass_bounds(inp)
    want, mus, levs = oracle_images(inp, bounds, pix=pix)
    with bipp_ss.StandardSynthesis(pix, inp.wl, bounds, n_eig=inp.n_eig, precision="fp32") as ss:
        ss.collect_batch(inp.st_xyz, inp.vis)
        got = ss.get()
        nt, nk, mu, lev = bipp_ss.bipp_ss_last_eigvals(ss.h, 2, inp.n_eig)
    for t in range(2):
        np.testing.assert_allclose(mu[t], mus[t], rtol=1e-10)
        assert list(lev[t]) == list(levs[t])
    err = rel_l2_per_level(got, want)
    assert np.all(err <= TOL["fp32"]), err


def test_failed_batch_leaves_images_unchanged():
    """A batch commits only if every step succeeds: a non-finite station
    coordinate (device variant, not inspected on the host) makes a Cholesky
    pivot NaN -> GRAM_NOT_PD; a one-sweep cap -> EIG_NOT_CONVERGED."""
    import torch
    inp = inputs.make_config(0, n_t=2, n_side=8)
    b = np.array([[-np.inf, np.inf]])
    with bipp_ss.StandardSynthesis(inp.pix, inp.wl, b, n_eig=4, precision="fp32") as ss:
        ss.collect(inp.st_xyz[0], inp.vis[0])
        before = ss.get()
        p = inp.st_xyz[1].copy()
        p[5, 0] = np.nan
        nst, N, st, V = bipp_ss.pack_batch([inp.st_xyz[0], p], inp.vis)
        with pytest.raises(bipp_ss.BippError) as e:
            bipp_ss.bipp_ss_collect_device(ss.h, nst, torch.from_numpy(st).cuda(), torch.from_numpy(V).cuda())
        assert e.value.code == bipp_ss.BIPP_ERR_GRAM_NOT_PD
        assert "step 1" in str(e.value)
        np.testing.assert_array_equal(ss.get(), before)
        with pytest.raises(bipp_ss.BippError) as e:
            ss.collect(p, inp.vis[1])  # the host variant checks the positions itself
        assert e.value.code == bipp_ss.BIPP_ERR_INVALID_ARG
        np.testing.assert_array_equal(ss.get(), before)
    with bipp_ss.StandardSynthesis(inp.pix, inp.wl, b, n_eig=4, precision="fp32", max_jacobi_sweeps=1) as ss:
        with pytest.raises(bipp_ss.BippError) as e:
            ss.collect(inp.st_xyz[0], inp.vis[0])
        assert e.value.code == bipp_ss.BIPP_ERR_EIG_NOT_CONVERGED
        assert np.all(ss.get() == 0.0)


def test_split_precision_rejects_stations_beyond_the_phase_range():
    """The tensor-core synthesis forms its phase from 32-bit integer station
    words (8 p/wl): a step with a station 2^28 wavelengths or more from the
    origin fails with BIPP_ERR_UNSUPPORTED and the batch adds nothing. The
    layout is moved as a whole, so the Gram matrix and eigenpairs are those
    of a good step."""
    inp = inputs.make_config(0, n_t=2, n_side=8)
    b = np.array([[-np.inf, np.inf]])
    far = inp.st_xyz[1] + np.array([2.0 ** 29 * inp.wl, 0.0, 0.0])
    with bipp_ss.StandardSynthesis(inp.pix, inp.wl, b, n_eig=4, precision="split_fp16") as ss:
        ss.collect(inp.st_xyz[0], inp.vis[0])
        before = ss.get()
        with pytest.raises(bipp_ss.BippError) as e:
            ss.collect_batch([inp.st_xyz[0], far], inp.vis)
        assert e.value.code == bipp_ss.BIPP_ERR_UNSUPPORTED
        assert "step 1" in str(e.value)
        np.testing.assert_array_equal(ss.get(), before)
        ss.collect(inp.st_xyz[1], inp.vis[1])  # the handle images again after the failure
        assert np.all(np.isfinite(ss.get())) and not np.array_equal(ss.get(), before)


def test_collect_rejects_bad_sizes():
    inp = inputs.make_config(0, n_t=1, n_side=8)
    b = np.array([[-np.inf, np.inf]])
    with bipp_ss.StandardSynthesis(inp.pix, inp.wl, b, n_eig=30) as ss:
        with pytest.raises(bipp_ss.BippError) as e:
            ss.collect(inp.st_xyz[0], inp.vis[0])  # n_eig 30 > n_st 24
        assert e.value.code == bipp_ss.BIPP_ERR_UNSUPPORTED


def test_device_pointer_variant_matches_oracle():
    import torch
    inp = inputs.make_config(0, n_t=3, n_side=16)
    bounds, _ = helpers.oracle_prepass_bounds(inp)
    want, _, _ = oracle_images(inp, bounds)
    nst, N, st, V = bipp_ss.pack_batch(inp.st_xyz, inp.vis)
    d_st = torch.from_numpy(st).cuda()
    d_V = torch.from_numpy(V).cuda()
    stream = torch.cuda.Stream()
    with bipp_ss.StandardSynthesis(inp.pix, inp.wl, bounds, n_eig=inp.n_eig, precision="fp32") as ss:
        bipp_ss.bipp_ss_collect_device(ss.h, nst, d_st, d_V, stream=stream)
        got = ss.get()
        out = torch.zeros((inp.n_level, inp.n_pix), dtype=torch.float64, device="cuda")
        bipp_ss.bipp_ss_get_device_f64(ss.h, out, stream=stream)
        stream.synchronize()
    assert np.all(rel_l2_per_level(got, want) <= TOL["fp32"])
    np.testing.assert_array_equal(out.cpu().numpy().T, got)


def test_device_complex64_visibilities():
    """complex64 device visibilities (widened on the device) give the images of
    the same values passed as complex128, and those of the oracle on them."""
    import dataclasses
    import torch
    inp = inputs.make_config(0, n_t=3, n_side=16)
    inp = dataclasses.replace(inp, vis=[v.astype(np.complex64).astype(np.complex128) for v in inp.vis])
    bounds, _ = helpers.oracle_prepass_bounds(inp)
    want, _, _ = oracle_images(inp, bounds)
    nst, N, st, V = bipp_ss.pack_batch(inp.st_xyz, inp.vis)
    d_st = torch.from_numpy(st).cuda()
    stream = torch.cuda.Stream()
    got = {}
    for dt in (np.complex64, np.complex128):
        with bipp_ss.StandardSynthesis(inp.pix, inp.wl, bounds, n_eig=inp.n_eig, precision="fp32") as ss:
            bipp_ss.bipp_ss_collect_device(ss.h, nst, d_st, torch.from_numpy(V.astype(dt)).cuda(), stream=stream)
            got[dt] = ss.get()
    np.testing.assert_allclose(got[np.complex64], got[np.complex128], rtol=1e-12, atol=0)
    assert np.all(rel_l2_per_level(got[np.complex64], want) <= TOL["fp32"])


def test_device_variant_rejects_misaligned_pointers():
    """The device variants check pointer alignment on the host, before any
    launch: d_vis 8 bytes into an allocation is not a complex128 array."""
    import ctypes
    import torch
    inp = inputs.make_config(0, n_t=1, n_side=8)
    b = np.array([[-np.inf, np.inf]])
    nst, N, st, V = bipp_ss.pack_batch(inp.st_xyz, inp.vis)
    d_st = torch.from_numpy(st).cuda()
    buf = torch.zeros(2 * V.size + 2, dtype=torch.float64, device="cuda")
    L = bipp_ss.load()
    with bipp_ss.StandardSynthesis(inp.pix, inp.wl, b, n_eig=4, precision="fp32") as ss:
        rc = L.bipp_ss_collect_device(ss.h, 1, N, bipp_ss._ip(nst), None, ctypes.c_void_p(d_st.data_ptr()),
                                      ctypes.c_void_p(buf.data_ptr() + 8), None)
        assert rc == bipp_ss.BIPP_ERR_INVALID_ARG
        assert "aligned" in bipp_ss.bipp_ss_last_error(ss.h)
        assert np.all(ss.get() == 0.0)


def test_checkpoint_resume_is_additive():
    inp = inputs.make_config(0, n_t=4, n_side=16)
    b = np.array([[-np.inf, np.inf]])
    with bipp_ss.StandardSynthesis(inp.pix, inp.wl, b, n_eig=8, precision="fp64") as ss:
        ss.collect_batch(inp.st_xyz, inp.vis)
        full = ss.get()
    with bipp_ss.StandardSynthesis(inp.pix, inp.wl, b, n_eig=8, precision="fp64") as ss:
        ss.collect_batch(inp.st_xyz[:2], inp.vis[:2])
        ck = ss.get()
    with bipp_ss.StandardSynthesis(inp.pix, inp.wl, b, n_eig=8, precision="fp64") as ss:
        bipp_ss.bipp_ss_set_images(ss.h, ck)
        ss.collect_batch(inp.st_xyz[2:], inp.vis[2:])
        resumed = ss.get()
    np.testing.assert_allclose(resumed, full, rtol=1e-12, atol=1e-12 * np.abs(full).max())


def test_rank1_source_peak_on_gpu():
    """Single point source, G = I, no noise: the image peaks at N^2 at the source pixel."""
    rng = np.random.default_rng(6)
    n = 16
    p = inputs.layout_disk(n, 40.0, 2.0, 3.0, rng)
    pix = inputs.pixel_grid(11, 6.0)
    j0 = 3 + 11 * 7
    V = inputs.visibilities(p, 2.0, pix[j0][None, :], np.array([1.0]), None, rng)
    for precision in ("fp64", "fp32"):
        with bipp_ss.StandardSynthesis(pix, 2.0, np.array([[-np.inf, np.inf]]), n_eig=1, precision=precision,
                                       gram_identity=1) as ss:
            ss.collect(p, V)
            img = ss.get()[:, 0]
        assert int(np.argmax(img)) == j0
        assert abs(img[j0] - n * n) <= 1e-4 * n * n


# ---------------------------------------------------------------- tensor-core (split) precisions

@pytest.mark.parametrize("precision", ["split_bf16", "split_fp16"])
def test_split_config0_end_to_end(cfg0, precision):
    inp, bounds, want, _, _ = cfg0
    with bipp_ss.StandardSynthesis(inp.pix, inp.wl, bounds, n_eig=inp.n_eig, precision=precision) as ss:
        ss.collect_batch(inp.st_xyz, inp.vis)
        got = ss.get()
    err = rel_l2_per_level(got, want)
    assert np.all(err <= TOL[precision]), (precision, err)


@pytest.mark.parametrize("precision", ["split_bf16", "split_fp16"])
def test_split_ragged_batch(precision):
    """Odd and ragged station counts (partial 32-station chunks), ragged
    n_eig (N = 2 n_eig padded to 16), 13^2 pixels (a single ragged tile)."""
    rng = np.random.default_rng(23)
    base = inputs.make_config(0, n_t=3, n_side=13)
    st, vis, ne = [], [], []
    for t, n in enumerate([17, 24, 13]):
        keep = np.sort(rng.choice(24, n, replace=False))
        st.append(base.st_xyz[t][keep])
        vis.append(base.vis[t][np.ix_(keep, keep)])
        ne.append([9, 24, 5][t])
    inp = inputs.SSInput("ragged", base.wl, base.pix, st, vis, 24, 3)
    bounds = np.array([[50.0, np.inf], [0.0, 50.0], [-np.inf, 0.0]])
    want, _, _ = oracle_images(inp, bounds, n_eig=ne)
    with bipp_ss.StandardSynthesis(inp.pix, inp.wl, bounds, precision=precision) as ss:
        ss.collect_batch(st, vis, n_eig=ne)
        got = ss.get()
    err = rel_l2_per_level(got, want)
    assert np.all(err <= TOL[precision]), (precision, err)


@pytest.mark.parametrize("precision", ["split_bf16", "split_fp16"])
def test_split_full_station_count_sampled_pixels(precision):
    """512 stations, N_eig 64 (N = 128), 4133 pixels (33 tiles, ragged last), 2 steps."""
    inp = inputs.make_config(1, n_t=2)
    side = inp.extra["n_side"]
    sel = (np.arange(0, side, 16)[:, None] * side + np.arange(0, side, 16)[None, :]).ravel()
    sel = np.concatenate([sel, np.arange(side * side - 37, side * side)])
    pix = inp.pix[sel]
    bounds, _ = helpers.oracle_prepass_bounds(inp)
    want, _, _ = oracle_images(inp, bounds, pix=pix)
    with bipp_ss.StandardSynthesis(pix, inp.wl, bounds, n_eig=inp.n_eig, precision=precision) as ss:
        ss.collect_batch(inp.st_xyz, inp.vis)
        got = ss.get()
    err = rel_l2_per_level(got, want)
    assert np.all(err <= TOL[precision]), (precision, err)


def test_split_widest_accumulator_and_limit():
    """N_eig 128 (N = 256: two stages of 96 KB, all 512 TMEM columns) matches
    the FP64 path; N_eig 129 is rejected on the split path."""
    inp = inputs.make_config(1, n_t=1, n_side=12)
    p, V = inp.st_xyz[0][:160], inp.vis[0][:160, :160]
    b = np.array([[1000.0, np.inf], [-np.inf, 1000.0]])
    with bipp_ss.StandardSynthesis(inp.pix, inp.wl, b, n_eig=128, precision="fp64") as ss:
        ss.collect(p, V)
        want = ss.get()
    for precision in ("split_bf16", "split_fp16"):
        with bipp_ss.StandardSynthesis(inp.pix, inp.wl, b, n_eig=128, precision=precision) as ss:
            ss.collect(p, V)
            got = ss.get()
        assert np.all(rel_l2_per_level(got, want) <= TOL[precision]), precision
    with bipp_ss.StandardSynthesis(inp.pix, inp.wl, b, n_eig=129, precision="split_bf16") as ss:
        with pytest.raises(bipp_ss.BippError) as e:
            ss.collect(p, V)
        assert e.value.code == bipp_ss.BIPP_ERR_UNSUPPORTED
