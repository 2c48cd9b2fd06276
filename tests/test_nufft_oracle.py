"""Pins of the NUFFT-synthesis oracle (Sec. 2.5, Sec. 3.4, Algorithm 3) to what
the mathematics fixes: the kernel transform against adaptive quadrature, the
type-3 sum against brute-force loops and closed forms, the NUFFT against the
direct sum within its tolerance, and the baseline form of the level images
against the standard-synthesis oracle (the identity of Sec. 2.5)."""
from __future__ import annotations

import cmath
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from oracle import nufft as nu
from paper_2310_09200_b300 import inputs


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_kernel_params_follow_the_published_rule():
    assert nu.kernel_params(1e-5) == (6, 2.30 * 6)
    assert nu.kernel_params(1e-3)[0] == 4
    assert nu.kernel_params(0.99)[0] == 2


@pytest.mark.parametrize("xi", [0.0, 0.3, 1.7, 4.0, 9.5])
def test_kernel_transform_against_adaptive_quadrature(xi):
    w, beta = nu.kernel_params(1e-6)
    alpha = 0.37
    want, _ = integrate.quad(lambda y: math.exp(beta * (math.sqrt(max(0.0, 1 - (y / alpha) ** 2)) - 1))
                             * math.cos(xi * y), -alpha, alpha, limit=200, epsabs=1e-14, epsrel=1e-13)
    assert abs(nu.es_ft(xi, alpha, beta) - want) <= 1e-11 * alpha


def test_next_smooth():
    for n in [1, 2, 7, 13, 97, 1000, 1025]:
        m = nu.next_smooth(n)
        assert m >= n and m % 2 == 0
        r = m
        for p in (2, 3, 5):
            while r % p == 0:
                r //= p
        assert r == 1
        assert all(nu.next_smooth(k) == m for k in range(max(n, 2), m + 1) if k >= n)


def test_direct_sum_by_brute_force_loops():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(3, 3)) * 5
    s = rng.normal(size=(4, 3))
    c = rng.normal(size=3) + 1j * rng.normal(size=3)
    f = nu.type3_direct(x, c, s)
    for k in range(4):
        want = sum(c[n] * cmath.exp(1j * sum(s[k, d] * x[n, d] for d in range(3))) for n in range(3))
        assert abs(f[k] - want) < 1e-13


@pytest.mark.parametrize("eps", [1e-3, 1e-5, 1e-7])
def test_type3_within_its_tolerance(eps):
    rng = np.random.default_rng(int(-math.log10(eps)))
    x = rng.uniform(-1, 1, (400, 3)) * [25.0, 14.0, 3.0] + [4.0, -2.0, 0.5]
    s = rng.uniform(-1, 1, (200, 3)) * [1.2, 0.8, 0.2] + [0.3, -0.1, 0.9]
    c = rng.normal(size=(400, 2)) + 1j * rng.normal(size=(400, 2))
    assert _rel(nu.type3(x, c, s, eps), nu.type3_direct(x, c, s)) <= 4 * eps


def test_type3_closed_forms_and_degenerate_extents():
    rng = np.random.default_rng(2)
    s = rng.uniform(-1, 1, (50, 3)) * [2.0, 2.0, 0.0] + [0.0, 0.0, 1.0]  # targets flat in z (S_z = 0)
    # one point at the origin: f = c everywhere
    f = nu.type3(np.zeros((1, 3)), np.array([2.0 - 1.0j]), s, 1e-8)
    assert np.max(np.abs(f - (2.0 - 1.0j))) <= 10 * 1e-8 * abs(2.0 - 1.0j)  # max error within 10 eps
    # one point at x0: f(s) = c exp(i s.x0)
    x0 = np.array([[3.0, -7.0, 11.0]])
    f = nu.type3(x0, np.array([1.5j]), s, 1e-8)
    assert np.max(np.abs(f - 1.5j * np.exp(1j * (s @ x0[0])))) <= 10 * 1e-8 * 1.5
    # inputs all at one z (X_z = 0) and a plane wave of points
    x = rng.uniform(-1, 1, (80, 3)) * [9.0, 9.0, 0.0] + [0.0, 0.0, 4.0]
    c = rng.normal(size=80) + 0j
    assert _rel(nu.type3(x, c, s, 1e-6), nu.type3_direct(x, c, s)) <= 4e-6


@pytest.fixture(scope="module")
def small_obs():
    rng = np.random.default_rng(5)
    p0 = inputs.layout_disk(12, 60.0, 1.0, 6.0, rng)
    src = inputs.sources_in_cap(5, 8.0, rng)
    flux = inputs.flux_lognormal(5, rng)
    st, vis = inputs.make_steps(p0, 2, 60.0, 2.0, src, flux, 20.0, rng)
    pix = inputs.pixel_grid(16, 10.0)
    return st, vis, pix


@pytest.mark.parametrize("filt,gi", [("lsq", False), ("std", False), ("lsq", True)])
def test_baseline_form_equals_standard_synthesis(small_obs, filt, gi):
    st, vis, pix = small_obs
    b = np.array([[3.0, np.inf], [0.5, 3.0], [-np.inf, 0.5]])
    want = got = None
    for p, V in zip(st, vis):
        want, mu, lev, W = oracle.ss_step(pix, 2.0, b, 8, p, V, img=want, filter=filt, gram_identity=gi)
        f, mu2, lev2, _ = nu.nufft_levels(pix, 2.0, b, 8, p, V, filter=filt, gram_identity=gi)
        got = f if got is None else got + f
        np.testing.assert_array_equal(lev, lev2)
        np.testing.assert_allclose(mu, mu2, rtol=1e-14)
    assert np.all(np.linalg.norm(got - want, axis=0) <= 1e-12 * np.linalg.norm(want, axis=0))


def test_nufft_levels_within_tolerance_of_standard_synthesis(small_obs):
    st, vis, pix = small_obs
    b = np.array([[3.0, np.inf], [0.5, 3.0], [-np.inf, 0.5]])
    want = got = None
    for p, V in zip(st, vis):
        want, *_ = oracle.ss_step(pix, 2.0, b, 8, p, V, img=want)
        f, *_ = nu.nufft_levels(pix, 2.0, b, 8, p, V, eps=1e-6)
        got = f if got is None else got + f
    err = np.linalg.norm(got - want, axis=0) / np.linalg.norm(want, axis=0)
    assert np.all(err <= 4e-6), err


def test_level_visibilities_rank_one():
    a = np.array([1.0 + 1j, 2.0, -1j])
    Vl = nu.level_visibilities(a[:, None], np.array([3.0]), np.array([1]), 2)
    assert np.all(Vl[0] == 0)
    np.testing.assert_allclose(Vl[1], 3.0 * np.outer(a, a.conj()))
    np.testing.assert_allclose(Vl[1], Vl[1].conj().T)


@pytest.mark.parametrize("eps", [1e-3, 1e-5])
def test_nufft_level_error_within_its_scale(eps):
    """On the NUFFT workload's geometry (48 stations, 40^2 pixels of 4 arcsec),
    every level's error stays within 5 eps of max(||I_l||, ||V'_l||_F sqrt(n_pix)):
    weak levels, whose images cancel, are measured against the size of their
    strengths rather than of their image (the bound the GPU tests use, doubled)."""
    inp = inputs.make_nufft_config(n_t=3, n_side=40, n_st=48)
    b = np.array([[1217.0, np.inf], [514.0, 1217.0], [255.0, 514.0], [-np.inf, 255.0]])
    want, scale = nu.nufft_levels_with_scale(inp.pix, inp.wl, b, 16, inp.st_xyz, inp.vis)
    got, _ = nu.nufft_levels_with_scale(inp.pix, inp.wl, b, 16, inp.st_xyz, inp.vis, eps=eps)
    err = np.linalg.norm(got - want, axis=0)
    assert np.all(err <= 5 * eps * np.maximum(np.linalg.norm(want, axis=0), scale)), err


def test_gram_corrected_visibilities_appendix_a():
    """App. A: with all eigenpairs, the visibilities are the Gram-corrected ones
    V' = A diag(mu) A^H mixed by the Gram matrix, V = G V' G for G-orthonormal
    eigenvectors (V A = G A Lambda and A^-1 = A^H G; App. A prints V = G V', which
    drops one factor G, harmless when G ~ I); the back-projected image (G = I) is
    the type-3 sum of G V' G, the least-squares image that of V'."""
    rng = np.random.default_rng(21)
    p = inputs.layout_disk(20, 300.0, 1.0, 6.0, rng)
    wl = 5.656  # 53 MHz
    V = inputs.visibilities(p, wl, inputs.sources_in_cap(3, 2.0, rng), np.array([1000.0, 5.0, 2.0]), 20.0, rng)
    G = oracle.gram(p, wl)
    mu, A, _ = oracle.geneig(V, G)
    Vp = nu.level_visibilities(A, mu, np.zeros(len(mu), dtype=np.int32), 1)[0]
    np.testing.assert_allclose(G @ Vp @ G, V, atol=1e-10 * np.abs(V).max())
    assert np.abs(G @ Vp - V).max() > 1e-3 * np.abs(V).max()  # the printed form is not exact
    pix = inputs.pixel_grid(12, 0.6)
    b = np.array([[-np.inf, np.inf]])
    x, c = nu.baseline_points(p, wl, np.stack([Vp, G @ Vp @ G]))
    f = nu.type3_direct(x, c, pix).real
    lsq, *_ = oracle.ss_step(pix, wl, b, len(p), p, V)
    back, *_ = oracle.ss_step(pix, wl, b, len(p), p, V, gram_identity=True)
    np.testing.assert_allclose(f[:, 0], lsq[:, 0], rtol=1e-10, atol=1e-10 * np.abs(lsq).max())
    np.testing.assert_allclose(f[:, 1], back[:, 0], rtol=1e-10, atol=1e-10 * np.abs(back).max())
