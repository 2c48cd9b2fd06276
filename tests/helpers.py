"""Test-side helpers: level bounds from an oracle pre-pass, and numpy brute-force
forms of the closed-form identities used to pin the oracle.

Nothing here is used by the GPU product path.
"""
from __future__ import annotations

import math

import numpy as np

import oracle
from oracle import estimate as oest


def quantile_bounds(pooled_mu, n_level: int) -> np.ndarray:
    """Level intervals from pooled eigenvalues (the "parameter estimation"
    pre-pass of Table tts), by the oracle's equal-count rule: inner edges at
    the 1/n_level quantiles, each halfway between the two nearest pooled
    values; outer edges +-inf; level 0 holds the largest eigenvalues.
    Returns (n_level, 2) rows [lo, hi)."""
    return np.array(oest.quantile_bounds(pooled_mu, n_level), dtype=np.float64)


def min_edge_margin(pooled_mu, bounds) -> float:
    """Smallest |mu - edge| over finite edges, relative to max |mu|."""
    mu = np.asarray(pooled_mu)
    edges = [x for x in np.asarray(bounds).ravel() if np.isfinite(x)]
    if not edges:
        return np.inf
    scale = max(np.max(np.abs(mu)), 1e-300)
    return min(np.min(np.abs(mu - e)) for e in edges) / scale


def oracle_prepass_bounds(inp, n_level=None, filter="lsq"):
    """Eigenvalues of every step by the oracle, pooled, then quantile bounds."""
    n_level = n_level or inp.n_level
    pooled = []
    for p, V in zip(inp.st_xyz, inp.vis):
        G = oracle.gram(p, inp.wl)
        mu, _, _ = oracle.geneig(V, G)
        pooled.extend(mu[: inp.n_eig])
    b = quantile_bounds(pooled, n_level)
    return b, np.asarray(pooled)


def phi_matrix(pix, st_xyz, wl):
    """Phi(r, i) = exp(+j 2 pi <r, p_i> / wl), shape (n_pix, n_st)."""
    return np.exp(1j * 2.0 * math.pi * (pix @ st_xyz.T) / wl)


def quad_form_image(pix, st_xyz, wl, M):
    """Phi(r)^H M Phi(r) for every pixel (real part), M (n_st, n_st)."""
    P = phi_matrix(pix, st_xyz, wl)
    return np.real(np.einsum("ri,ij,rj->r", P.conj(), M, P))


def oracle_eigenimages(pix, wl, st_list, vis_list, n_eig, filter="lsq", gram_identity=False):
    """One image per kept eigenpair (rank order), summed over steps, from the
    oracle's eigensolve and synthesis with level id = rank. n_eig: one count
    for all steps or one per step; the image count is the largest."""
    counts = [n_eig] * len(st_list) if np.isscalar(n_eig) else list(n_eig)
    n_img = max(counts)
    img = None
    for p, V, k in zip(st_list, vis_list, counts):
        G = np.eye(p.shape[0]) if gram_identity else oracle.gram(p, wl)
        mu, A, _ = oracle.geneig(V, G)
        d = mu[:k] if filter == "lsq" else np.ones(k)
        img = oracle.synth_levels(pix, p, wl, A[:, :k], d, np.arange(k, dtype=np.int32), n_img, img=img)
    return img
