"""One image per kept eigenpair (options.eigenimages): every precision against
the oracle's eigensolve and synthesis with level id = rank, the sum over the
eigenimages against the single-level image, 64 eigenimages on the split
tensor-core path with the mixed eigensolver, and ragged per-step counts."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2310_09200_b300 import bipp_ss, inputs
from tests import helpers

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-9, "fp32": 1e-5, "split_bf16": 1e-3, "split_fp16": 1e-5}


def _rel(a, b):
    return np.array([np.linalg.norm(a[:, l] - b[:, l]) / max(np.linalg.norm(b[:, l]), 1e-300)
                     for l in range(b.shape[1])])


@pytest.fixture(scope="module")
def cfg0():
    inp = inputs.make_config(0)
    want = helpers.oracle_eigenimages(inp.pix, inp.wl, inp.st_xyz, inp.vis, inp.n_eig)
    return inp, want


@pytest.mark.parametrize("precision", ["fp64", "fp32", "split_bf16", "split_fp16"])
def test_eigenimages_config0(cfg0, precision):
    inp, want = cfg0
    with bipp_ss.StandardSynthesis(inp.pix, inp.wl, None, n_eig=inp.n_eig, precision=precision,
                                   eigenimages=True) as ss:
        ss.collect_batch(inp.st_xyz, inp.vis)
        got = ss.get()
    assert got.shape == want.shape == (inp.pix.shape[0], inp.n_eig)
    assert np.all(_rel(got, want) <= TOL[precision]), _rel(got, want)


def test_eigenimages_sum_to_the_single_level_image(cfg0):
    inp, _ = cfg0
    with bipp_ss.StandardSynthesis(inp.pix, inp.wl, None, n_eig=inp.n_eig, precision="fp64",
                                   eigenimages=True) as ss:
        ss.collect_batch(inp.st_xyz, inp.vis)
        eig = ss.get()
    with bipp_ss.StandardSynthesis(inp.pix, inp.wl, np.array([[-np.inf, np.inf]]), n_eig=inp.n_eig,
                                   precision="fp64") as ss:
        ss.collect_batch(inp.st_xyz, inp.vis)
        one = ss.get()
    np.testing.assert_allclose(eig.sum(axis=1), one[:, 0], rtol=1e-11, atol=1e-11 * np.max(np.abs(one)))


def test_sixty_four_eigenimages_split_mixed():
    inp = inputs.make_config(1, n_t=2)
    side = inp.extra["n_side"]
    sel = (np.arange(0, side, 16)[:, None] * side + np.arange(0, side, 16)[None, :]).ravel()
    pix = inp.pix[np.concatenate([sel, np.arange(side * side - 7, side * side)])]
    want = helpers.oracle_eigenimages(pix, inp.wl, inp.st_xyz, inp.vis, inp.n_eig)
    with bipp_ss.StandardSynthesis(pix, inp.wl, None, n_eig=inp.n_eig, precision="split_fp16", eig_mode="mixed",
                                   eigenimages=True) as ss:
        ss.collect_batch(inp.st_xyz, inp.vis)
        got = ss.get()
    assert got.shape[1] == 64
    assert np.all(_rel(got, want) <= TOL["split_fp16"]), _rel(got, want)


@pytest.mark.parametrize("precision", ["fp64", "split_fp16"])
def test_eigenimages_ragged_counts(precision):
    rng = np.random.default_rng(43)
    base = inputs.make_config(1, n_t=3, n_side=10)
    st, vis = [], []
    for t, n in enumerate([250, 301, 197]):
        keep = np.sort(rng.choice(512, n, replace=False))
        st.append(base.st_xyz[t][keep])
        vis.append(base.vis[t][np.ix_(keep, keep)])
    ne = [10, 20, 5]
    want = helpers.oracle_eigenimages(base.pix, base.wl, st, vis, ne)
    with bipp_ss.StandardSynthesis(base.pix, base.wl, None, n_eig=20, precision=precision,
                                   eigenimages=True) as ss:
        ss.collect_batch(st, vis, n_eig=ne)
        got = ss.get()
    assert np.all(_rel(got, want) <= TOL[precision]), _rel(got, want)
