"""Mixed-precision eigensolve (the leading pairs of the FP32 tridiagonal form by
multisection and inverse iteration, then FP64-class refinement of the kept
pairs) against the FP64 oracle: eigenvalues to 1e-10 relative, identical level
assignment, images within each synthesis precision's tolerance."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2310_09200_b300 import bipp_ss, inputs
from tests import helpers

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-9, "fp32": 1e-5, "split_bf16": 1e-3, "split_fp16": 1e-5}
BASE_LAUNCHES = 9
MIXED_LAUNCHES = 77  # kernels of the mixed eigensolver per batch
# a mixed batch: gram, cholesky, trinv, 2 FP32 reduction GEMMs, the eigensolver, select, synthesis
MIXED_BATCH = 7 + MIXED_LAUNCHES


def _rel(a, b):
    return np.array([np.linalg.norm(a[:, l] - b[:, l]) / max(np.linalg.norm(b[:, l]), 1e-300)
                     for l in range(b.shape[1])])


@pytest.fixture(scope="module")
def ska512():
    inp = inputs.make_config(1, n_t=2)
    side = inp.extra["n_side"]
    sel = (np.arange(0, side, 32)[:, None] * side + np.arange(0, side, 32)[None, :]).ravel()
    pix = inp.pix[np.concatenate([sel, np.arange(side * side - 11, side * side)])]
    bounds, pooled = helpers.oracle_prepass_bounds(inp)
    img, mus, levs = None, [], []
    for p, V in zip(inp.st_xyz, inp.vis):
        img, mu, lev, _ = oracle.ss_step(pix, inp.wl, bounds, inp.n_eig, p, V, img=img)
        mus.append(mu)
        levs.append(lev)
    return inp, pix, bounds, img, mus, levs


@pytest.mark.parametrize("precision", ["fp64", "fp32", "split_fp16"])
def test_mixed_eigensolve_512_stations(ska512, precision):
    inp, pix, bounds, want, mus, levs = ska512
    with bipp_ss.StandardSynthesis(pix, inp.wl, bounds, n_eig=inp.n_eig, precision=precision,
                                   eig_mode="mixed") as ss:
        ss.collect_batch(inp.st_xyz, inp.vis)
        got = ss.get()
        nt, nk, mu, lev = bipp_ss.bipp_ss_last_eigvals(ss.h, 2, inp.n_eig)
        t = ss.timings()
    assert t["launches"] >= MIXED_BATCH, t  # the mixed solver ran
    for s in range(2):
        np.testing.assert_allclose(mu[s], mus[s], rtol=1e-10)
        assert list(lev[s]) == list(levs[s])
    err = _rel(got, want)
    assert np.all(err <= TOL[precision]), (precision, err)


def test_mixed_eigensolve_ragged_batch():
    rng = np.random.default_rng(41)
    base = inputs.make_config(1, n_t=3, n_side=10)
    st, vis = [], []
    for t, n in enumerate([250, 301, 197]):
        keep = np.sort(rng.choice(512, n, replace=False))
        st.append(base.st_xyz[t][keep])
        vis.append(base.vis[t][np.ix_(keep, keep)])
    ne = [10, 20, 5]
    b = np.array([[500.0, np.inf], [-np.inf, 500.0]])
    want, mus = None, []
    for p, V, k in zip(st, vis, ne):
        want, mu, _, _ = oracle.ss_step(base.pix, base.wl, b, k, p, V, img=want)
        mus.append(mu)
    with bipp_ss.StandardSynthesis(base.pix, base.wl, b, precision="fp64", eig_mode="mixed") as ss:
        ss.collect_batch(st, vis, n_eig=ne)
        got = ss.get()
        nt, nk, mu, lev = bipp_ss.bipp_ss_last_eigvals(ss.h, 3, 20)
        assert ss.timings()["launches"] == MIXED_BATCH
    for s in range(3):
        np.testing.assert_allclose(mu[s, : ne[s]], mus[s], rtol=1e-10)
    assert np.all(_rel(got, want) <= TOL["fp64"])


def test_mixed_falls_back_to_fp64_jacobi_when_scratch_does_not_fit():
    inp = inputs.make_config(0, n_t=2, n_side=8)  # 24 stations, 12 pairs: kp = n
    b = np.array([[-np.inf, np.inf]])
    with bipp_ss.StandardSynthesis(inp.pix, inp.wl, b, n_eig=12, precision="fp64", eig_mode="mixed") as ss:
        ss.collect_batch(inp.st_xyz, inp.vis)
        assert ss.timings()["launches"] == BASE_LAUNCHES
        got = ss.get()
    want = None
    for p, V in zip(inp.st_xyz, inp.vis):
        want, *_ = oracle.ss_step(inp.pix, inp.wl, b, 12, p, V, img=want)
    assert np.all(_rel(got, want) <= TOL["fp64"])
