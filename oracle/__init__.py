"""FP64 CPU oracle for Bluebild standard synthesis (BIPP, arXiv:2310.09200).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the CPU-baseline
leg of the benchmark may import this package; the GPU product path never does.
It wraps ``libbipp_oracle.so`` (plain C, FP64) with numpy marshalling only:
every number is computed in ``bipp_oracle.c``.

Array conventions: positions are ``(n, 3)`` float64, complex matrices are
``(n, m)`` complex128; they are passed column-major as the paper's interface
prescribes (Sec. 3.2).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None

OK, EINVAL, ENOTPD, ENOCONV = 0, -1, -2, -3


class OracleError(RuntimeError):
    def __init__(self, where: str, code: int):
        super().__init__(f"{where} failed with code {code}")
        self.code = code


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp, ip, i64 = C.POINTER(C.c_double), C.POINTER(C.c_int), C.c_int64
        vp = C.c_void_p
        L.orc_gram.argtypes = [C.c_int, dp, C.c_double, dp]
        L.orc_cholesky.argtypes = [C.c_int, dp, dp]
        L.orc_jacobi_herm.argtypes = [C.c_int, vp, dp, vp, C.c_double, C.c_int, ip]
        L.orc_geneig.argtypes = [C.c_int, vp, dp, dp, vp, C.c_double, C.c_int, ip]
        L.orc_select_levels.argtypes = [C.c_int, dp, C.c_int, dp, ip]
        L.orc_synth_levels.argtypes = [i64, dp, C.c_int, dp, C.c_double, C.c_int, vp, dp, ip, C.c_int, dp]
        L.orc_synth_levels.restype = None
        L.orc_ss_step.argtypes = [i64, dp, C.c_double, C.c_int, dp, C.c_int, C.c_int, C.c_int,
                                  C.c_int, dp, vp, dp, dp, ip, vp, C.c_double, C.c_int]
        L.orc_grad.argtypes = [i64, dp, C.c_double, C.c_int, C.c_int, C.c_int, C.c_int, dp,
                               vp, dp, ip, vp, dp, dp, dp, vp, vp]
        _lib = L
    return _lib


def _f64(a, shape=None):
    a = np.asfortranarray(np.asarray(a, dtype=np.float64))
    if shape is not None and a.shape != shape:
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


def _c128(a, shape=None):
    a = np.asfortranarray(np.asarray(a, dtype=np.complex128))
    if shape is not None and a.shape != shape:
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _vp(a):
    return C.c_void_p(a.ctypes.data)


def _check(where, rc):
    if rc != 0:
        raise OracleError(where, rc)


def gram(xyz, wl):
    """G_ij = sinc(2 ||p_i - p_j|| / wl) (Eq. gram)."""
    xyz = _f64(xyz)
    n = xyz.shape[0]
    G = np.zeros((n, n), order="F")
    _check("orc_gram", lib().orc_gram(n, _dp(xyz), float(wl), _dp(G)))
    return G


def cholesky(G):
    G = _f64(G)
    n = G.shape[0]
    L = np.zeros((n, n), order="F")
    _check("orc_cholesky", lib().orc_cholesky(n, _dp(G), _dp(L)))
    return L


def jacobi_herm(Cm, tol=1e-14, max_sweeps=60):
    """Cyclic complex Jacobi; returns (mu unsorted, Q, rotated C, sweeps)."""
    Cm = _c128(Cm).copy(order="F")
    n = Cm.shape[0]
    mu = np.zeros(n)
    Q = np.zeros((n, n), dtype=np.complex128, order="F")
    sw = C.c_int(0)
    _check("orc_jacobi_herm", lib().orc_jacobi_herm(n, _vp(Cm), _dp(mu), _vp(Q), tol, max_sweeps, C.byref(sw)))
    return mu, Q, Cm, sw.value


def geneig(V, G=None, tol=1e-14, max_sweeps=60):
    """V a = mu G a; returns (mu descending, A with A^H G A = I, sweeps)."""
    V = _c128(V)
    n = V.shape[0]
    Gp = None
    if G is not None:
        G = _f64(G, (n, n))
        Gp = _dp(G)
    mu = np.zeros(n)
    A = np.zeros((n, n), dtype=np.complex128, order="F")
    sw = C.c_int(0)
    _check("orc_geneig", lib().orc_geneig(n, _vp(V), Gp, _dp(mu), _vp(A), tol, max_sweeps, C.byref(sw)))
    return mu, A, sw.value


def select_levels(mu, bounds):
    mu = _f64(mu)
    bounds = _f64(bounds)
    n_level = bounds.shape[0]
    lev = np.zeros(mu.shape[0], dtype=np.int32)
    _check("orc_select_levels", lib().orc_select_levels(mu.shape[0], _dp(mu), n_level, _dp(bounds), _ip(lev)))
    return lev


def synth_levels(pix, st_xyz, wl, W, d, level_id, n_level, img=None):
    """Accumulate sum_{e in l} d_e |sum_i exp(-j k<r,p_i>) W_ie|^2 into img."""
    pix = _f64(pix)
    st_xyz = _f64(st_xyz)
    W = _c128(W)
    d = _f64(d)
    lev = np.ascontiguousarray(level_id, dtype=np.int32)
    n_pix, n_st, n_eig = pix.shape[0], st_xyz.shape[0], W.shape[1]
    if img is None:
        img = np.zeros((n_pix, n_level), order="F")
    assert img.flags.f_contiguous and img.dtype == np.float64
    lib().orc_synth_levels(n_pix, _dp(pix), n_st, _dp(st_xyz), float(wl), n_eig, _vp(W), _dp(d),
                           _ip(lev), n_level, _dp(img))
    return img


def ss_step(pix, wl, bounds, n_eig, st_xyz, V, img=None, filter="lsq", gram_identity=False,
            tol=1e-14, max_sweeps=60):
    """One collect() step of Algorithm 1. Returns (img, mu, level_id, W)."""
    pix = _f64(pix)
    bounds = _f64(bounds)
    st_xyz = _f64(st_xyz)
    V = _c128(V)
    n_pix, n_level, n_st = pix.shape[0], bounds.shape[0], st_xyz.shape[0]
    if img is None:
        img = np.zeros((n_pix, n_level), order="F")
    mu = np.zeros(n_eig)
    lev = np.zeros(n_eig, dtype=np.int32)
    W = np.zeros((n_st, n_eig), dtype=np.complex128, order="F")
    f = {"lsq": 0, "std": 1}[filter]
    _check("orc_ss_step", lib().orc_ss_step(n_pix, _dp(pix), float(wl), n_level, _dp(bounds), n_eig, f,
                                            int(bool(gram_identity)), n_st, _dp(st_xyz), _vp(V), _dp(img),
                                            _dp(mu), _ip(lev), _vp(W), tol, max_sweeps))
    return img, mu, lev, W


def grad(pix, wl, n_level, st_xyz, W, d, level_id, g, target):
    """Loss and complex gradients (dL/dRe + j dL/dIm) w.r.t. gains and W.

    st_xyz: (T, n_st, 3); W: (T, n_st, n_eig); d, level_id: (T, n_eig);
    g: (n_st,); target: (n_pix, n_level). Returns (loss, img, grad_g, grad_W).
    """
    pix = _f64(pix)
    st_xyz = np.asarray(st_xyz, dtype=np.float64)
    T, n_st, _ = st_xyz.shape
    n_eig = W.shape[2]
    # per-step column-major blocks, concatenated over t
    st_blk = np.concatenate([np.asfortranarray(st_xyz[t]).ravel(order="F") for t in range(T)])
    W_blk = np.concatenate([np.asfortranarray(W[t]).ravel(order="F") for t in range(T)]).astype(np.complex128)
    d_blk = np.ascontiguousarray(np.asarray(d, dtype=np.float64).reshape(T * n_eig))
    lev_blk = np.ascontiguousarray(np.asarray(level_id, dtype=np.int32).reshape(T * n_eig))
    g = np.ascontiguousarray(g, dtype=np.complex128)
    target = _f64(target, (pix.shape[0], n_level))
    loss = C.c_double(0.0)
    img = np.zeros((pix.shape[0], n_level), order="F")
    gg = np.zeros(n_st, dtype=np.complex128)
    gW = np.zeros(T * n_st * n_eig, dtype=np.complex128)
    _check("orc_grad", lib().orc_grad(pix.shape[0], _dp(pix), float(wl), n_level, T, n_st, n_eig,
                                      _dp(st_blk), _vp(W_blk), _dp(d_blk), _ip(lev_blk), _vp(g), _dp(target),
                                      C.byref(loss), _dp(img), _vp(gg), _vp(gW)))
    gW = np.stack([gW[t * n_st * n_eig:(t + 1) * n_st * n_eig].reshape((n_st, n_eig), order="F") for t in range(T)])
    return loss.value, img, gg, gW
