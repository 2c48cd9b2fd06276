"""Parity at the benchmark's sizes and above the 512-station kernels.

1. The benchmark workload in its launch configuration: all 1024^2 pixels of
   configuration 1 (8192 tiles over the persistent grid), 512 stations, split
   FP16 synthesis and the mixed eigensolver, here over 3 steps; the oracle
   computes a few hundred sampled pixels (random ones, tile edges and the last
   pixels) one by one, and every step's kept eigenvalues.
2. A 700-station layout: the mixed eigensolver's paths for n_max > 512 (the
   full-storage Householder reduction, the two-rows-per-thread
   back-transformation and Z applier), against the oracle in FP64.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2310_09200_b300 import bipp_ss, inputs
from tests import helpers

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.array([np.linalg.norm(a[:, l] - b[:, l]) / max(np.linalg.norm(b[:, l]), 1e-300)
                     for l in range(b.shape[1])])


def test_benchmark_workload_sampled_pixels():
    inp = inputs.make_config(1, n_t=3)
    n_pix = inp.pix.shape[0]
    assert n_pix == 1024 * 1024
    rng = np.random.default_rng(7)
    sample = np.unique(np.concatenate([
        rng.choice(n_pix, 200, replace=False),
        np.arange(0, n_pix, 128 * 1031)[:60],          # first rows of scattered 128-pixel tiles
        np.arange(127, n_pix, 128 * 1031)[:30],        # last rows of tiles
        np.arange(n_pix - 10, n_pix),                  # the ragged end of the pixel range
    ]))
    bounds, _ = helpers.oracle_prepass_bounds(inp)
    want, mus = None, []
    for p, V in zip(inp.st_xyz, inp.vis):
        want, mu, _, _ = oracle.ss_step(inp.pix[sample], inp.wl, bounds, inp.n_eig, p, V, img=want)
        mus.append(mu)
    with bipp_ss.StandardSynthesis(inp.pix, inp.wl, bounds, n_eig=inp.n_eig, precision="split_fp16",
                                   eig_mode="mixed") as ss:
        ss.collect_batch(inp.st_xyz, inp.vis)
        got = ss.get()
        _, _, mu, _ = bipp_ss.bipp_ss_last_eigvals(ss.h, len(inp.vis), inp.n_eig)
    for s in range(len(inp.vis)):
        np.testing.assert_allclose(mu[s], mus[s], rtol=1e-10)
    err = _rel(got[sample], want)
    assert np.all(err <= 1e-5), err


def test_mixed_eigensolve_above_512_stations():
    rng = np.random.default_rng(1700)
    p0 = inputs.layout_lognormal(700, 1000.0, 1.0, 20.0, 65000.0, 5.0, 35.0, rng)
    src = inputs.sources_in_cap(200, 10.0, rng)
    flux = inputs.flux_powerlaw(200, rng)
    st, vis = inputs.make_steps(p0, 1, 60.0, 2.0, src, flux, 20.0, rng, np.complex128)
    pix = inputs.pixel_grid(24, 10.0)
    b = np.array([[-np.inf, np.inf]])
    n_eig = 48
    want, mu_want, _, _ = oracle.ss_step(pix, 2.0, b, n_eig, st[0], vis[0])
    with bipp_ss.StandardSynthesis(pix, 2.0, b, n_eig=n_eig, precision="fp64", eig_mode="mixed") as ss:
        ss.collect_batch(st, vis)
        got = ss.get()
        _, _, mu, _ = bipp_ss.bipp_ss_last_eigvals(ss.h, 1, n_eig)
        assert ss.timings()["launches"] > 9  # the mixed solver ran
    np.testing.assert_allclose(mu[0], mu_want, rtol=1e-10)
    assert np.all(_rel(got, want) <= 1e-9)
