"""Pins for the FP64 CPU oracle: closed forms, textbook special cases,
invariants and brute force fixed by the paper and the mathematics — never the
oracle checked against itself. CPU only."""
from __future__ import annotations

import math
import os

import numpy as np
import pytest
import scipy.linalg

import oracle
from paper_2310_09200_b300 import inputs
from tests import helpers

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_herm(n, rng):
    X = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    return 0.5 * (X + X.conj().T)


def _stations(n, rng, spread=200.0, min_sep=10.0):
    return inputs.layout_disk(n, spread, 3.0, min_sep, rng)


# ---------------------------------------------------------------- Gram (Eq. gram, App. A)

def test_gram_golden_sinc_points():
    rows = [l.split("#")[0].split() for l in open(os.path.join(GOLDEN, "sinc_points.txt"))]
    rows = [(float(a), float(b)) for a, b in (r for r in rows if r)]
    wl = 1.7
    for sep, want in rows:
        xyz = np.array([[0.0, 0.0, 0.0], [sep * wl * 0.6, sep * wl * 0.8, 0.0]])
        G = oracle.gram(xyz, wl)
        assert abs(G[0, 1] - want) < 1e-15 and abs(G[1, 0] - want) < 1e-15
        assert G[0, 0] == 1.0 and G[1, 1] == 1.0


def test_gram_matches_numpy_sinc():
    rng = np.random.default_rng(1)
    p = rng.normal(scale=30.0, size=(17, 3))
    wl = 2.3
    d = np.linalg.norm(p[:, None, :] - p[None, :, :], axis=2)
    want = np.sinc(2.0 * d / wl)  # numpy's sinc is the normalised one
    G = oracle.gram(p, wl)
    np.testing.assert_allclose(G, want, rtol=0, atol=1e-14)
    np.testing.assert_array_equal(G, G.T)


# ---------------------------------------------------------------- Jacobi / eigensolve (Eq. eigenvaleq)

def test_jacobi_known_spectrum_dft_basis():
    """C = F diag(lam) F^H with the unitary DFT matrix F has eigenvalues lam."""
    n = 16
    lam = np.linspace(-3.0, 5.0, n) ** 3
    j = np.arange(n)
    F = np.exp(-2j * math.pi * np.outer(j, j) / n) / math.sqrt(n)
    Cm = F @ np.diag(lam) @ F.conj().T
    mu, Q, Crot, sweeps = oracle.jacobi_herm(Cm)
    np.testing.assert_allclose(np.sort(mu), np.sort(lam), rtol=0, atol=1e-12 * np.max(np.abs(lam)))
    assert sweeps >= 1
    # columns of Q are eigenvectors: C Q = Q diag(mu)
    np.testing.assert_allclose(Cm @ Q, Q * mu[None, :], atol=1e-11 * np.max(np.abs(lam)))


def test_jacobi_random_hermitian_vs_library():
    rng = np.random.default_rng(2)
    Cm = _rand_herm(40, rng)
    mu, Q, _, _ = oracle.jacobi_herm(Cm)
    np.testing.assert_allclose(np.sort(mu), np.linalg.eigvalsh(Cm), atol=1e-12 * np.linalg.norm(Cm))
    np.testing.assert_allclose(Q.conj().T @ Q, np.eye(40), atol=1e-13)
    np.testing.assert_allclose(Q @ np.diag(mu) @ Q.conj().T, Cm, atol=1e-12 * np.linalg.norm(Cm))


def test_geneig_2x2_closed_form():
    """det(V - mu G) = 0 for G = [[1, g], [g, 1]], V = [[a, b], [b*, c]]:
    (1 - g^2) mu^2 - (a + c - 2 g Re b) mu + (a c - |b|^2) = 0."""
    for (a, b, c, g) in [(3.0, 1.0 + 2.0j, -1.0, 0.3), (2.0, -0.5j, 5.0, -0.6), (1.0, 0.5 + 0j, 2.0, 0.0)]:
        V = np.array([[a, b], [np.conj(b), c]])
        G = np.array([[1.0, g], [g, 1.0]])
        A2, B2, C2 = 1 - g * g, -(a + c - 2 * g * np.real(b)), a * c - abs(b) ** 2
        disc = math.sqrt(B2 * B2 - 4 * A2 * C2)
        roots = sorted([(-B2 + disc) / (2 * A2), (-B2 - disc) / (2 * A2)], reverse=True)
        mu, A, _ = oracle.geneig(V, G)
        np.testing.assert_allclose(mu, roots, rtol=0, atol=1e-13)
        np.testing.assert_allclose(A.conj().T @ G @ A, np.eye(2), atol=1e-13)


def test_geneig_residual_orthonormality_and_scipy():
    rng = np.random.default_rng(3)
    n = 30
    p = _stations(n, rng)
    wl = 2.0
    G = oracle.gram(p, wl)
    V = _rand_herm(n, rng)
    mu, A, _ = oracle.geneig(V, G)
    assert np.all(np.diff(mu) <= 0), "eigenvalues must be sorted descending"
    res = np.linalg.norm(V @ A - G @ A @ np.diag(mu)) / np.linalg.norm(V)
    assert res < 1e-12
    np.testing.assert_allclose(A.conj().T @ G @ A, np.eye(n), atol=1e-12)
    w = scipy.linalg.eigh(V, G, eigvals_only=True)[::-1]
    np.testing.assert_allclose(mu, w, atol=1e-12 * np.max(np.abs(w)))


def test_geneig_errors():
    rng = np.random.default_rng(4)
    G = np.eye(6)
    G[1, 3] = G[3, 1] = 1.5  # indefinite "Gram" matrix (eigenvalue -0.5)
    with pytest.raises(oracle.OracleError) as e:
        oracle.geneig(_rand_herm(6, rng), G)
    assert e.value.code == oracle.ENOTPD
    with pytest.raises(oracle.OracleError) as e:
        oracle.jacobi_herm(_rand_herm(20, rng), max_sweeps=1)
    assert e.value.code == oracle.ENOCONV


# ---------------------------------------------------------------- levels (Sec. 2.6)

def test_select_levels_half_open():
    b = np.array([[10.0, np.inf], [5.0, 10.0], [-np.inf, 5.0]])
    lev = oracle.select_levels(np.array([11.0, 10.0, 9.99, 5.0, 4.9, -3.0]), b)
    assert list(lev) == [0, 0, 1, 1, 2, 2]
    b2 = np.array([[1.0, 2.0]])
    assert list(oracle.select_levels(np.array([3.0, 2.0, 1.5, 1.0, 0.5]), b2)) == [-1, -1, 0, 0, -1]


# ---------------------------------------------------------------- whole pipeline identities

ALL = np.array([[-np.inf, np.inf]])


def _small_case(n_st=10, side=8, cap=8.0, seed=5, snr=20.0, n_src=4):
    rng = np.random.default_rng(seed)
    p = _stations(n_st, rng, spread=60.0, min_sep=4.0)
    wl = 2.0
    pix = inputs.pixel_grid(side, cap)
    src = inputs.sources_in_cap(n_src, cap, rng)
    flux = inputs.flux_lognormal(n_src, rng)
    V = inputs.visibilities(p, wl, src, flux, snr, rng)
    return p, wl, pix, V, src, flux


def test_rank1_point_source_closed_form_and_peak():
    """G = I, V = e0 e0^H: mu = N, image = |sum_i exp(j k <p_i, r0 - r>)|^2,
    peaking at N^2 exactly at r0 (placed on a pixel off the cap centre)."""
    rng = np.random.default_rng(6)
    n = 12
    p = _stations(n, rng, spread=40.0, min_sep=3.0)
    wl = 2.0
    pix = inputs.pixel_grid(9, 6.0)
    j0 = 2 + 9 * 6  # off-centre pixel (il=2, im=6)
    r0 = pix[j0]
    V = inputs.visibilities(p, wl, r0[None, :], np.array([1.0]), None, rng)
    img, mu, lev, W = oracle.ss_step(pix, wl, ALL, n, p, V, gram_identity=True)
    assert abs(mu[0] - n) < 1e-12 * n and np.all(np.abs(mu[1:]) < 1e-10)
    k = 2 * math.pi / wl
    want = np.abs(np.exp(1j * k * ((r0[None, :] - pix) @ p.T)).sum(axis=1)) ** 2
    np.testing.assert_allclose(img[:, 0], want, rtol=1e-11, atol=1e-10)
    assert int(np.argmax(img[:, 0])) == j0
    assert abs(img[j0, 0] - n * n) < 1e-9
    # sign of the phase: the mirror pixel (reflection through the cap centre) is not the peak
    jm = (8 - 2) + 9 * (8 - 6)
    assert img[jm, 0] < 0.9 * n * n


def test_identity_gram_all_pairs_is_dirty_image():
    """G = I and all eigenpairs: sum of levels = Phi^H V Phi (back-projection, Sec. 2.8)."""
    p, wl, pix, V, _, _ = _small_case()
    n = p.shape[0]
    b = np.array([[0.0, np.inf], [-np.inf, 0.0]])
    img, mu, lev, W = oracle.ss_step(pix, wl, b, n, p, V, gram_identity=True)
    want = helpers.quad_form_image(pix, p, wl, V)
    np.testing.assert_allclose(img.sum(axis=1), want, rtol=1e-11, atol=1e-11 * np.max(np.abs(want)))


def test_sinc_gram_all_pairs_is_lsq_image():
    """Sinc Gram and all eigenpairs: sum of levels = Phi^H G^-1 V G^-1 Phi (Eq. skyreco)."""
    p, wl, pix, V, _, _ = _small_case(seed=7)
    n = p.shape[0]
    img, mu, lev, W = oracle.ss_step(pix, wl, ALL, n, p, V)
    d = np.linalg.norm(p[:, None, :] - p[None, :, :], axis=2)
    G = np.sinc(2 * d / wl)
    M = np.linalg.solve(G, np.linalg.solve(G, V).conj().T).conj().T  # G^-1 V G^-1
    want = helpers.quad_form_image(pix, p, wl, M)
    np.testing.assert_allclose(img[:, 0], want, rtol=1e-10, atol=1e-10 * np.max(np.abs(want)))


def test_std_filter_all_pairs_is_inverse_gram_form():
    """STD filter (unit weights), all eigenpairs: A A^H = G^-1, so the sum of
    levels is Phi^H G^-1 Phi, independent of V."""
    p, wl, pix, V, _, _ = _small_case(seed=8)
    n = p.shape[0]
    img, *_ = oracle.ss_step(pix, wl, ALL, n, p, V, filter="std")
    d = np.linalg.norm(p[:, None, :] - p[None, :, :], axis=2)
    G = np.sinc(2 * d / wl)
    want = helpers.quad_form_image(pix, p, wl, np.linalg.inv(G))
    np.testing.assert_allclose(img[:, 0], want, rtol=1e-10)


def test_bruteforce_8x8_lsq_definition():
    """Explicit loops over B~_jj = sum_pq Psi_jp (G^-1 V G^-1)_pq Psi*_qj with
    Psi_jp = exp(-j k <x_p, r_j>) (Eq. skyreco, Eq. standard_synthesis)."""
    p, wl, pix, V, _, _ = _small_case(n_st=6, side=8, seed=9)
    n = p.shape[0]
    img, *_ = oracle.ss_step(pix, wl, ALL, n, p, V)
    d = np.linalg.norm(p[:, None, :] - p[None, :, :], axis=2)
    Ginv = np.linalg.inv(np.sinc(2 * d / wl))
    M = Ginv @ V @ Ginv
    k = 2 * math.pi / wl
    for j in range(pix.shape[0]):
        acc = 0.0 + 0.0j
        for a in range(n):
            psi_a = complex(math.cos(k * pix[j] @ p[a]), -math.sin(k * pix[j] @ p[a]))
            for b in range(n):
                psi_b_conj = complex(math.cos(k * pix[j] @ p[b]), math.sin(k * pix[j] @ p[b]))
                acc += psi_a * M[a, b] * psi_b_conj
        assert abs(acc.imag) < 1e-9 * max(1.0, abs(acc.real))
        assert abs(img[j, 0] - acc.real) <= 1e-10 * max(1.0, abs(acc.real))


def test_partition_invariance_and_nonnegativity():
    """Sum over 1, 2 or 4 levels is the same image (Sec. 4.2); levels holding
    only non-negative eigenvalues are non-negative images."""
    p, wl, pix, V, _, _ = _small_case(seed=10)
    n = p.shape[0]
    n_eig = 7
    _, mu, _, _ = oracle.ss_step(pix, wl, ALL, n_eig, p, V)
    sums = []
    for n_level in (1, 2, 4):
        b = helpers.quantile_bounds(mu, n_level)
        img, _, lev, _ = oracle.ss_step(pix, wl, b, n_eig, p, V)
        sums.append(img.sum(axis=1))
        for l in range(n_level):
            if np.any(lev == l) and np.all(mu[lev == l] >= 0):
                assert np.all(img[:, l] >= -1e-12 * np.max(np.abs(img)))
    np.testing.assert_allclose(sums[1], sums[0], rtol=1e-12, atol=1e-12 * np.max(np.abs(sums[0])))
    np.testing.assert_allclose(sums[2], sums[0], rtol=1e-12, atol=1e-12 * np.max(np.abs(sums[0])))


def test_psd_visibilities_give_nonnegative_levels():
    p, wl, pix, V, _, _ = _small_case(seed=11, snr=None)
    n = p.shape[0]
    b = np.array([[0.0, np.inf]])
    img, mu, lev, _ = oracle.ss_step(pix, wl, b, 4, p, V)
    assert np.all(mu[:4] > 0)
    assert np.all(img >= 0.0)


def test_time_accumulation_is_a_plain_sum():
    inp = inputs.make_config(0, n_t=2, n_side=8)
    b = np.array([[-np.inf, np.inf]])
    acc = None
    parts = []
    for p, V in zip(inp.st_xyz, inp.vis):
        acc, *_ = oracle.ss_step(inp.pix, inp.wl, b, inp.n_eig, p, V, img=acc)
        one, *_ = oracle.ss_step(inp.pix, inp.wl, b, inp.n_eig, p, V)
        parts.append(one)
    np.testing.assert_allclose(acc, parts[0] + parts[1], rtol=1e-13)


def test_eigenvector_phase_invariance_of_synthesis():
    """|Phi^H w|^2 does not depend on a unit-modulus factor on w."""
    p, wl, pix, V, _, _ = _small_case(seed=12)
    n = p.shape[0]
    mu, A, _ = oracle.geneig(V, oracle.gram(p, wl))
    lev = np.zeros(5, dtype=np.int32)
    i1 = oracle.synth_levels(pix, p, wl, A[:, :5], mu[:5], lev, 1)
    ph = np.exp(1j * np.linspace(0, 5, 5))
    i2 = oracle.synth_levels(pix, p, wl, A[:, :5] * ph[None, :], mu[:5], lev, 1)
    np.testing.assert_allclose(i1, i2, rtol=1e-12)


# ---------------------------------------------------------------- gradient

def test_oracle_gradient_matches_central_differences():
    rng = np.random.default_rng(13)
    n_st, n_eig, T, n_level = 5, 3, 2, 2
    p = np.stack([_stations(n_st, rng, spread=30.0, min_sep=3.0) for _ in range(T)])
    pix = inputs.pixel_grid(5, 8.0)
    W = rng.normal(size=(T, n_st, n_eig)) + 1j * rng.normal(size=(T, n_st, n_eig))
    d = np.abs(rng.normal(size=(T, n_eig))) + 0.5
    lev = rng.integers(0, n_level, size=(T, n_eig)).astype(np.int32)
    g = inputs.gains(n_st, 0.05, rng)
    target = np.abs(rng.normal(size=(pix.shape[0], n_level))) * 10
    wl = 2.0
    L0, img, gg, gW = oracle.grad(pix, wl, n_level, p, W, d, lev, g, target)

    def loss(gv, Wv):
        return oracle.grad(pix, wl, n_level, p, Wv, d, lev, gv, target)[0]

    h = 1e-6
    for i in range(n_st):
        num = 0j
        for unit in (1.0, 1j):
            gp, gm = g.copy(), g.copy()
            gp[i] += h * unit
            gm[i] -= h * unit
            num += unit * (loss(gp, W) - loss(gm, W)) / (2 * h)
        assert abs(num - gg[i]) <= 1e-6 * max(1.0, abs(gg[i])), (i, num, gg[i])
    for (t, i, e) in [(0, 0, 0), (1, 3, 2), (0, 4, 1)]:
        num = 0j
        for unit in (1.0, 1j):
            Wp, Wm = W.copy(), W.copy()
            Wp[t, i, e] += h * unit
            Wm[t, i, e] -= h * unit
            num += unit * (loss(g, Wp) - loss(g, Wm)) / (2 * h)
        assert abs(num - gW[t, i, e]) <= 1e-6 * max(1.0, abs(gW[t, i, e])), (t, i, e, num, gW[t, i, e])


def test_eigenimages_partition_and_closed_form():
    """One image per kept eigenpair: they sum to the single-level image, and
    image e is d_e |Phi^H a_e|^2 written out from the eigenvectors."""
    p, wl, pix, V, _, _ = _small_case(seed=12)
    n_eig = 6
    eig = helpers.oracle_eigenimages(pix, wl, [p], [V], n_eig)
    one, mu, _, _ = oracle.ss_step(pix, wl, ALL, n_eig, p, V)
    np.testing.assert_allclose(eig.sum(axis=1), one[:, 0], rtol=1e-12, atol=1e-12 * np.max(np.abs(one)))
    mu_all, A, _ = oracle.geneig(V, oracle.gram(p, wl))
    P = helpers.phi_matrix(pix, p, wl)
    for e in range(n_eig):
        want = mu_all[e] * np.abs(P.conj() @ A[:, e]) ** 2
        np.testing.assert_allclose(eig[:, e], want, rtol=1e-10, atol=1e-12 * np.max(np.abs(want)))
    std = helpers.oracle_eigenimages(pix, wl, [p], [V], n_eig, filter="std")
    assert np.all(std >= 0.0)


def test_single_station_degenerate_case():
    """One station: G = [1], V = [v] with v > 0, so mu = v and a = [1] (A^H G A = 1),
    and |Phi(r) a|^2 = 1 at every pixel: the LSQ image is v everywhere, the STD
    image 1, each in the level holding v; the other levels stay zero."""
    pix = inputs.pixel_grid(5, 10.0)
    p = np.array([[1234.5, -321.0, 2.5]])
    v = 37.25
    bounds = np.array([[100.0, np.inf], [10.0, 100.0], [-np.inf, 10.0]])
    for filt, want_val in (("lsq", v), ("std", 1.0)):
        img, mu, lev, W = oracle.ss_step(pix, 2.0, bounds, 1, p, np.array([[v + 0j]]), filter=filt)
        assert mu[0] == pytest.approx(v, rel=1e-15) and lev[0] == 1
        assert abs(abs(W[0, 0]) - 1.0) < 1e-15
        np.testing.assert_allclose(img[:, 1], want_val, rtol=1e-13)
        assert np.all(img[:, [0, 2]] == 0.0)


def test_station_permutation_invariance():
    """Relabelling the stations (rows of the positions, rows and columns of V
    together) changes neither the eigenvalues nor the images: a position and
    its visibilities must travel together through every index of the path."""
    inp = inputs.make_config(0, n_t=1, n_side=10)
    p, V = inp.st_xyz[0], inp.vis[0]
    perm = np.random.default_rng(9).permutation(p.shape[0])
    bounds = np.array([[200.0, np.inf], [50.0, 200.0], [-np.inf, 50.0]])
    a, mu_a, lev_a, _ = oracle.ss_step(inp.pix, inp.wl, bounds, inp.n_eig, p, V)
    b, mu_b, lev_b, _ = oracle.ss_step(inp.pix, inp.wl, bounds, inp.n_eig, p[perm], V[np.ix_(perm, perm)])
    np.testing.assert_allclose(mu_b, mu_a, rtol=1e-11)
    assert list(lev_a) == list(lev_b)
    np.testing.assert_allclose(b, a, rtol=1e-10, atol=1e-12 * np.abs(a).max())


def test_visibility_scaling():
    """V -> c V (c > 0) with the level edges scaled by c: the eigenvalues scale
    by c and the G-orthonormal eigenvectors do not change, so the LSQ images
    (weights mu) scale by c and the STD images (weights 1) stay the same."""
    inp = inputs.make_config(0, n_t=1, n_side=10)
    p, V = inp.st_xyz[0], inp.vis[0]
    c = 7.5
    bounds = np.array([[200.0, np.inf], [50.0, 200.0], [-np.inf, 50.0]])
    for filt, factor in (("lsq", c), ("std", 1.0)):
        a, mu_a, lev_a, _ = oracle.ss_step(inp.pix, inp.wl, bounds, inp.n_eig, p, V, filter=filt)
        b, mu_b, lev_b, _ = oracle.ss_step(inp.pix, inp.wl, c * bounds, inp.n_eig, p, c * V, filter=filt)
        np.testing.assert_allclose(mu_b, c * mu_a, rtol=1e-11)
        assert list(lev_a) == list(lev_b)
        np.testing.assert_allclose(b, factor * a, rtol=1e-10, atol=1e-12 * factor * np.abs(a).max())
