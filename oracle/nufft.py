"""NUFFT synthesis (Sec. 2.5 "NUFFT Image Synthesis", Sec. 3.4 "NUFFT
Synthesis", Algorithm 3), written plainly in numpy FP64.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline may use it; the library never does.

What the method computes. Per step and level l, the Gram-corrected
visibilities restricted to the level (eigenvalues outside the level's interval
set to zero, Sec. 2.6) are V'_l = sum_{e in l} d_e a_e a_e^H, and the level image
is the type-3 sum over all station pairs (p, q) (the baseline form of the
synthesis equation, Sec. 2.5):

    I_l(r) = sum_{p,q} V'_l,pq exp(-j 2 pi / wl <p_p - p_q, r>),

which is real because V'_l is Hermitian and the baselines are antisymmetric,
and which equals the standard-synthesis level image sum_e d_e |Phi^H a_e|^2
exactly. The phase sign follows the standard-synthesis reading
z_e(r) = sum_i exp(-j k <r, p_i>) a_ie.

- ``type3_direct``: the defining sum f_k = sum_n c_n exp(i <s_k, x_n>), term by
  term.
- ``type3``: the approximation of Sec. 3.4, step by step: (1) centre the input
  points x and the targets s and pre-phase the strengths, (2) spread them onto a
  regular grid of spacing h with the exponential-of-semicircle kernel,
  (3) evaluate that grid as a Fourier series at the rescaled targets s' h with a
  type-2 NUFFT (divide the modes by the second kernel's Fourier transform,
  FFT on a twice finer grid, interpolate with the kernel), (4) divide by the
  spreading kernel's Fourier transform at the targets (the diagonal correction)
  and apply the post-phase. Kernel and grid rules are those of the
  exponential-of-semicircle NUFFT (Barnett, Magland and af Klinteberg, SIAM J.
  Sci. Comput. 41, 2019): width w = ceil(log10(1/eps)) + 1 grid points,
  beta = 2.30 w, upsampling sigma = 2; the type-3 grid spacing follows from
  requiring the spread function's spectrum, sampled at spacing h, to alias
  only beyond the kernel's pass band: h = pi / (sigma S), with
  M = 2 sigma X S / pi + w + 2 points per dimension for inputs in [C - X, C + X]
  and targets in [D - S, D + S].
- ``nufft_levels``: the level images of one step by either evaluation.
"""
from __future__ import annotations

import math

import numpy as np

from . import geneig, gram, select_levels

SIGMA = 2.0


def kernel_params(eps):
    """Kernel width w (grid points) and shape beta for tolerance eps."""
    if not (1e-15 < eps < 1.0):
        raise ValueError("eps must be in (1e-15, 1)")
    w = int(math.ceil(math.log10(1.0 / eps))) + 1
    w = max(2, min(w, 16))
    return w, 2.30 * w


def es_kernel(z, beta):
    """phi(z) = exp(beta (sqrt(1 - z^2) - 1)) on |z| <= 1, zero outside."""
    z = np.asarray(z, dtype=np.float64)
    out = np.zeros_like(z)
    m = np.abs(z) <= 1.0
    out[m] = np.exp(beta * (np.sqrt(1.0 - z[m] ** 2) - 1.0))
    return out


_GL = np.polynomial.legendre.leggauss(200)


def es_ft(xi, alpha, beta):
    """Fourier transform of psi(y) = phi(y / alpha):
    psi_hat(xi) = alpha * int_{-1}^{1} phi(z) cos(alpha xi z) dz, by 200-point
    Gauss-Legendre quadrature."""
    z, wq = _GL
    xi = np.asarray(xi, dtype=np.float64)
    phi = es_kernel(z, beta)
    return alpha * np.cos(alpha * np.multiply.outer(xi, z)) @ (wq * phi)


def next_smooth(n):
    """Least even integer >= n whose prime factors are 2, 3 and 5."""
    m = max(2, int(n))
    while True:
        if m % 2 == 0:
            r = m
            for p in (2, 3, 5):
                while r % p == 0:
                    r //= p
            if r == 1:
                return m
        m += 1


def type3_direct(x, c, s):
    """f[k, :] = sum_n c[n, :] exp(i <s_k, x_n>); x (n, 3), s (m, 3), c (n,) or (n, L)."""
    x = np.asarray(x, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    c = np.asarray(c, dtype=np.complex128)
    vec = c.ndim == 1
    c2 = c[:, None] if vec else c
    out = np.zeros((s.shape[0], c2.shape[1]), dtype=np.complex128)
    for k0 in range(0, s.shape[0], 256):
        ph = s[k0:k0 + 256] @ x.T
        out[k0:k0 + 256] = np.exp(1j * ph) @ c2
    return out[:, 0] if vec else out


def type3_grid(x, s, eps):
    """Per-dimension centres, half-widths, grid sizes and spacings of type3."""
    w, beta = kernel_params(eps)
    x = np.asarray(x, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    C = 0.5 * (x.min(0) + x.max(0))
    X = 0.5 * (x.max(0) - x.min(0))
    D = 0.5 * (s.min(0) + s.max(0))
    S = 0.5 * (s.max(0) - s.min(0))
    M = np.zeros(3, dtype=np.int64)
    h = np.zeros(3)
    for d in range(3):
        M[d] = next_smooth(max(2 * w, math.ceil(2.0 * SIGMA * X[d] * S[d] / math.pi) + w + 2))
        if S[d] > 0:
            h[d] = math.pi / (SIGMA * S[d])
        elif X[d] > 0:
            h[d] = 2.0 * X[d] / (M[d] - w - 2)
        else:
            h[d] = 1.0
    return dict(w=w, beta=beta, C=C, X=X, D=D, S=S, M=M, h=h)


def _spread_weights(g, w, beta):
    """Start index and the w kernel weights of each coordinate g (grid units)."""
    m0 = np.ceil(g - 0.5 * w).astype(np.int64)
    j = np.arange(w)
    wt = es_kernel(2.0 * (m0[:, None] + j[None, :] - g[:, None]) / w, beta)
    return m0, wt


def type3(x, c, s, eps):
    """Approximates type3_direct(x, c, s) to relative accuracy ~eps (steps of Sec. 3.4)."""
    x = np.asarray(x, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    c = np.asarray(c, dtype=np.complex128)
    vec = c.ndim == 1
    c2 = c[:, None] if vec else c
    L = c2.shape[1]
    P = type3_grid(x, s, eps)
    w, beta, C, D, M, h = P["w"], P["beta"], P["C"], P["D"], P["M"], P["h"]

    # (1) centred inputs and targets, pre-phased strengths: s.x = s'.x' + s'.C + D.x
    xc = x - C
    sc = s - D
    cp = c2 * np.exp(1j * (x @ D))[:, None]

    # (2) spread onto the grid y_m = (m - M/2) h: F[m] = sum_n c'_n prod_d psi(y_m,d - x'_n,d)
    F = np.zeros((M[0], M[1], M[2], L), dtype=np.complex128)
    g = [xc[:, d] / h[d] + M[d] / 2 for d in range(3)]
    sw = [_spread_weights(g[d], w, beta) for d in range(3)]
    for a in range(w):
        for b in range(w):
            for e in range(w):
                wt = sw[0][1][:, a] * sw[1][1][:, b] * sw[2][1][:, e]
                idx = (sw[0][0] + a, sw[1][0] + b, sw[2][0] + e)
                np.add.at(F, idx, wt[:, None] * cp)

    # (3) type-2 at t = s' h: f(t) = sum_k F[k] exp(i k.t), k = m - M/2
    N2 = 2 * M
    alpha2 = w * math.pi / N2
    Fp = F
    for d in range(3):  # divide each mode by the interpolation kernel's transform
        k = np.arange(M[d]) - M[d] // 2
        shape = [1, 1, 1, 1]
        shape[d] = M[d]
        Fp = Fp / es_ft(k, alpha2[d], beta).reshape(shape)
    G = np.zeros((N2[0], N2[1], N2[2], L), dtype=np.complex128)
    ix = [np.mod(np.arange(M[d]) - M[d] // 2, N2[d]) for d in range(3)]
    G[np.ix_(ix[0], ix[1], ix[2])] = Fp
    G = np.fft.ifftn(G, axes=(0, 1, 2)) * float(np.prod(N2))  # sum_k G_k exp(+i k u_j)
    t = sc * h[None, :]
    tg = [t[:, d] * N2[d] / (2 * math.pi) for d in range(3)]
    iw = [_spread_weights(tg[d], w, beta) for d in range(3)]
    f = np.zeros((s.shape[0], L), dtype=np.complex128)
    for a in range(w):
        for b in range(w):
            for e in range(w):
                wt = iw[0][1][:, a] * iw[1][1][:, b] * iw[2][1][:, e]
                f += wt[:, None] * G[np.mod(iw[0][0] + a, N2[0]), np.mod(iw[1][0] + b, N2[1]),
                                     np.mod(iw[2][0] + e, N2[2])]
    f *= float(np.prod(2 * math.pi / N2))

    # (4) trapezoid factor, diagonal correction by the spreading kernel's transform, post-phase
    corr = np.ones(s.shape[0])
    for d in range(3):
        corr *= h[d] / es_ft(sc[:, d], 0.5 * w * h[d], beta)
    out = f * (corr * np.exp(1j * (sc @ C)))[:, None]
    return out[:, 0] if vec else out


def level_visibilities(W, d, level_id, n_level):
    """V'_l = sum_{e: level_id[e] = l} d_e a_e a_e^H for l < n_level (Sec. 2.6)."""
    n = W.shape[0]
    Vl = np.zeros((n_level, n, n), dtype=np.complex128)
    for e in range(W.shape[1]):
        if 0 <= level_id[e] < n_level:
            Vl[level_id[e]] += d[e] * np.outer(W[:, e], W[:, e].conj())
    return Vl


def error_scale(W, d, level_id, n_level, n_pix):
    """Per level, ||V'_l||_F sqrt(n_pix): the l2 size of a type-3 sum over the
    level's strengths with unrelated phases, the scale of the NUFFT's error
    (squares add over steps: combine as sqrt(sum of squares))."""
    Vl = level_visibilities(W, d, level_id, n_level)
    return np.sqrt(np.sum(np.abs(Vl) ** 2, axis=(1, 2)) * n_pix)


def baseline_points(st_xyz, wl, Vl):
    """Input points x_n = -2 pi / wl (p_p - p_q) of all ordered pairs and their
    per-level strengths c_n = V'_l,pq, so that I_l = Re sum_n c_n exp(i <r, x_n>)."""
    p = np.asarray(st_xyz, dtype=np.float64)
    n = p.shape[0]
    b = (p[:, None, :] - p[None, :, :]).reshape(n * n, 3)
    x = -2.0 * math.pi / wl * b
    c = Vl.reshape(Vl.shape[0], n * n).T
    return x, c


def nufft_levels(pix, wl, bounds, n_eig, st_xyz, V, eps=None, filter="lsq", gram_identity=False,
                 tol=1e-14, max_sweeps=60):
    """One step of Algorithm 3: level images (n_pix, n_level) by the direct type-3
    sum (eps None) or by the type-3 NUFFT; also returns mu, level_id, W."""
    st_xyz = np.asarray(st_xyz, dtype=np.float64)
    G = None if gram_identity else gram(st_xyz, wl)
    mu, A, _ = geneig(V, G, tol, max_sweeps)
    mu, W = mu[:n_eig], A[:, :n_eig]
    bounds = np.asarray(bounds, dtype=np.float64)
    lev = select_levels(mu, bounds)
    d = mu if filter == "lsq" else np.ones_like(mu)
    Vl = level_visibilities(W, d, lev, bounds.shape[0])
    x, c = baseline_points(st_xyz, wl, Vl)
    f = type3_direct(x, c, pix) if eps is None else type3(x, c, pix, eps)
    return np.asfortranarray(f.real), mu, lev, W


def nufft_levels_with_scale(pix, wl, bounds, n_eig, st_list, vis_list, eps=None, **kw):
    """Level images summed over the steps, and the per-level error scale
    sqrt(sum_t error_scale_t^2)."""
    img, sc2 = None, 0.0
    bounds = np.asarray(bounds, dtype=np.float64)
    for p, V in zip(st_list, vis_list):
        f, mu, lev, W = nufft_levels(pix, wl, bounds, n_eig, p, V, eps=eps, **kw)
        d = mu if kw.get("filter", "lsq") == "lsq" else np.ones_like(mu)
        sc2 = sc2 + error_scale(W, d, lev, bounds.shape[0], pix.shape[0]) ** 2
        img = f if img is None else img + f
    return img, np.sqrt(sc2)
