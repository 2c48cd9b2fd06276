"""ctypes binding of libbipp_ss.so (C ABI in include/bipp_ss.h).

Argument marshalling only: every stage of standard synthesis runs in the CUDA
library. The library is required: importing works without a GPU, but any
compute call raises if ``libbipp_ss.so`` is missing or no CUDA device is
present — there is no CPU fallback.

Array conventions follow the ABI (column-major, Sec. 3.2 of BIPP): positions
are given here as ``(n, 3)`` float64 arrays, visibilities as ``(n, n)``
complex128, images come back as ``(n_pix, n_level)``.
"""
from __future__ import annotations

import ctypes as C
import math
import os
from typing import Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libbipp_ss.so")

BIPP_OK = 0
BIPP_ERR_INVALID_ARG = -1
BIPP_ERR_CUDA = -2
BIPP_ERR_OUT_OF_MEMORY = -3
BIPP_ERR_GRAM_NOT_PD = -4
BIPP_ERR_EIG_NOT_CONVERGED = -5
BIPP_ERR_DEVICE_TIMEOUT = -6
BIPP_ERR_UNSUPPORTED = -7

BIPP_PREC_FP64, BIPP_PREC_FP32, BIPP_PREC_SPLIT_BF16, BIPP_PREC_SPLIT_FP16 = 0, 1, 2, 3
PRECISIONS = {"fp64": 0, "fp32": 1, "split_bf16": 2, "split_fp16": 3}
BIPP_FILTER_LSQ, BIPP_FILTER_STD = 0, 1
FILTERS = {"lsq": 0, "std": 1}
BIPP_EIG_JACOBI64, BIPP_EIG_MIXED = 0, 1
EIG_MODES = {"jacobi64": 0, "mixed": 1}
BIPP_SYNTH_STANDARD, BIPP_SYNTH_NUFFT = 0, 1
SYNTHESES = {"standard": 0, "nufft": 1}

ERROR_NAMES = {
    -1: "BIPP_ERR_INVALID_ARG", -2: "BIPP_ERR_CUDA", -3: "BIPP_ERR_OUT_OF_MEMORY",
    -4: "BIPP_ERR_GRAM_NOT_PD", -5: "BIPP_ERR_EIG_NOT_CONVERGED", -6: "BIPP_ERR_DEVICE_TIMEOUT",
    -7: "BIPP_ERR_UNSUPPORTED",
}

EXPORTED = [
    "bipp_ss_default_options", "bipp_ss_create", "bipp_ss_collect", "bipp_ss_collect_batch",
    "bipp_ss_collect_device", "bipp_ss_get", "bipp_ss_get_f64", "bipp_ss_get_device_f64", "bipp_ss_reset",
    "bipp_ss_set_images", "bipp_ss_last_eigvals", "bipp_ss_get_timings", "bipp_ss_destroy",
    "bipp_ss_last_error", "bipp_ss_collect_noalloc", "bipp_ss_synth_levels_device",
    "bipp_ss_synth_adjoint_device", "bipp_ss_create_channels", "bipp_ss_collect_channels",
    "bipp_ss_energy_neig", "bipp_ss_kmeans_bounds", "bipp_ss_get_nufft_timings", "bipp_ss_collect_device_c64",
    "bipp_ss_debug_fail_wait", "bipp_ss_quantile_bounds", "bipp_ss_measure_sincos_rate",
    "bipp_ss_measure_fma_rates", "bipp_ss_get_synth_shape",
]

BIPP_NOALLOC_MAX_STATIONS = 128
BIPP_NOALLOC_MAX_EIG = 128
BIPP_MAX_EIGENIMAGES = 64


class BippError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


class bipp_ss_options(C.Structure):
    _fields_ = [
        ("n_eig", C.c_int32), ("precision", C.c_int32), ("filter", C.c_int32), ("gram_identity", C.c_int32),
        ("max_jacobi_sweeps", C.c_int32), ("jacobi_tol", C.c_double), ("device", C.c_int32),
        ("eig_mode", C.c_int32), ("use_graph", C.c_int32), ("autotune", C.c_int32), ("eigenimages", C.c_int32),
        ("synthesis", C.c_int32), ("nufft_eps", C.c_double), ("nufft_partition", C.c_int32 * 6),
        ("reserved", C.c_int32 * 2),
    ]


_lib = None


def load(path: str | None = None):
    """Load libbipp_ss.so (raises if it is missing: no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing; build it with `python -m paper_2310_09200_b300.build`")
    L = C.CDLL(path)
    dp, ip, vp, i32, i64 = C.POINTER(C.c_double), C.POINTER(C.c_int32), C.c_void_p, C.c_int32, C.c_int64
    H = C.c_void_p
    L.bipp_ss_default_options.argtypes = [C.POINTER(bipp_ss_options)]
    L.bipp_ss_default_options.restype = None
    L.bipp_ss_create.argtypes = [C.POINTER(H), i64, dp, C.c_double, i32, dp, C.POINTER(bipp_ss_options)]
    L.bipp_ss_collect.argtypes = [H, i32, dp, dp]
    L.bipp_ss_collect_batch.argtypes = [H, i32, i32, ip, ip, dp, dp]
    L.bipp_ss_collect_device.argtypes = [H, i32, i32, ip, ip, vp, vp, vp]
    L.bipp_ss_collect_device_c64.argtypes = [H, i32, i32, ip, ip, vp, vp, vp]
    L.bipp_ss_get.argtypes = [H, C.POINTER(C.c_float)]
    L.bipp_ss_get_f64.argtypes = [H, dp]
    L.bipp_ss_get_device_f64.argtypes = [H, vp, vp]
    L.bipp_ss_reset.argtypes = [H]
    L.bipp_ss_set_images.argtypes = [H, dp]
    L.bipp_ss_last_eigvals.argtypes = [H, i32, i32, ip, ip, dp, ip]
    L.bipp_ss_get_timings.argtypes = [H, dp]
    L.bipp_ss_get_synth_shape.argtypes = [H, ip]
    L.bipp_ss_get_nufft_timings.argtypes = [H, dp]
    L.bipp_ss_debug_fail_wait.argtypes = [H, i32]
    L.bipp_ss_destroy.argtypes = [H]
    L.bipp_ss_energy_neig.argtypes = [i32, dp, C.c_double, ip]
    L.bipp_ss_kmeans_bounds.argtypes = [i32, dp, i32, dp]
    L.bipp_ss_quantile_bounds.argtypes = [i32, dp, i32, dp]
    L.bipp_ss_measure_sincos_rate.argtypes = [i32, i32, dp]
    L.bipp_ss_measure_fma_rates.argtypes = [i32, i32, dp, dp]
    L.bipp_ss_last_error.argtypes = [H]
    L.bipp_ss_last_error.restype = C.c_char_p
    L.bipp_ss_collect_noalloc.argtypes = [i64, vp, C.c_double, i32, dp, i32, i32, i32, i32, vp, vp, vp, vp,
                                          C.c_char_p, i32]
    L.bipp_ss_synth_levels_device.argtypes = [i64, vp, C.c_double, i32, i32, i32, i32, vp, vp, vp, vp, vp, vp, i32,
                                              vp]
    L.bipp_ss_create_channels.argtypes = [C.POINTER(H), i64, dp, i32, dp, i32, dp, C.POINTER(bipp_ss_options)]
    L.bipp_ss_collect_channels.argtypes = [H, i32, i32, ip, ip, ip, vp, vp, i32, vp]
    L.bipp_ss_synth_adjoint_device.argtypes = [i64, vp, C.c_double, i32, i32, i32, i32, vp, vp, vp, vp, vp, vp,
                                               vp, vp, i32, vp]
    for name in EXPORTED:
        if name not in ("bipp_ss_default_options", "bipp_ss_last_error"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def bipp_ss_last_error(h) -> str:
    return load().bipp_ss_last_error(h).decode()


def _check(h, rc):
    if rc != BIPP_OK:
        raise BippError(rc, bipp_ss_last_error(h))


def bipp_ss_default_options(**kw) -> bipp_ss_options:
    o = bipp_ss_options()
    load().bipp_ss_default_options(C.byref(o))
    names = {"precision": PRECISIONS, "filter": FILTERS, "eig_mode": EIG_MODES, "synthesis": SYNTHESES}
    fields = {f[0] for f in bipp_ss_options._fields_}
    for k, v in kw.items():
        if k not in fields:  # a ctypes Structure would silently take an unknown attribute
            raise TypeError(f"unknown option {k!r}; options are {sorted(fields)}")
        if k in names and isinstance(v, str):
            if v not in names[k]:
                raise ValueError(f"{k}={v!r}; choose from {sorted(names[k])}")
            v = names[k][v]
        if k == "nufft_partition":  # (uvw cells, image cells), each a triple
            flat = [int(x) for x in np.ravel(v)]
            if len(flat) != 6:
                raise ValueError("nufft_partition needs 6 values: 3 input cells, then 3 image cells")
            v = (C.c_int32 * 6)(*flat)
        setattr(o, k, int(v) if isinstance(v, bool) else v)
    return o


def _colmajor_xyz(xyz) -> np.ndarray:
    a = np.asarray(xyz, dtype=np.float64)
    if a.ndim != 2 or a.shape[1] != 3:
        raise ValueError("positions must be (n, 3)")
    return np.ascontiguousarray(a.T)  # memory layout == column-major (n, 3)


def bipp_ss_create(pix_xyz, wl: float, level_bounds, **opts) -> C.c_void_p:
    """Create a handle. level_bounds: (n_level, 2) rows [lo, hi); None with
    eigenimages=1 (one image per kept eigenpair, n_level = n_eig)."""
    L = load()
    pix = _colmajor_xyz(pix_xyz)
    o = bipp_ss_default_options(**opts)
    if level_bounds is None:
        n_level, bptr = int(o.n_eig), None
    else:
        b = np.asarray(level_bounds, dtype=np.float64)
        if b.ndim != 2 or b.shape[1] != 2:
            raise ValueError("level_bounds must be (n_level, 2)")
        bc = np.ascontiguousarray(b.T)
        n_level, bptr = b.shape[0], _dp(bc)
    h = C.c_void_p()
    rc = L.bipp_ss_create(C.byref(h), pix.shape[1], _dp(pix), float(wl), n_level, bptr, C.byref(o))
    if rc != BIPP_OK:
        raise BippError(rc, bipp_ss_last_error(None))
    return h


def bipp_ss_create_channels(pix_xyz, wl, level_bounds, **opts) -> C.c_void_p:
    """Multi-channel handle. wl: (n_chan,) metres; level_bounds: (n_chan,
    n_level, 2) rows [lo, hi) per channel."""
    L = load()
    pix = _colmajor_xyz(pix_xyz)
    wl = np.ascontiguousarray(wl, dtype=np.float64)
    b = np.asarray(level_bounds, dtype=np.float64)
    if b.ndim != 3 or b.shape[0] != wl.shape[0] or b.shape[2] != 2:
        raise ValueError("level_bounds must be (n_chan, n_level, 2)")
    bc = np.ascontiguousarray(np.transpose(b, (0, 2, 1)))  # per channel: column-major n_level x 2
    o = bipp_ss_default_options(**opts)
    h = C.c_void_p()
    rc = L.bipp_ss_create_channels(C.byref(h), pix.shape[1], _dp(pix), wl.shape[0], _dp(wl), b.shape[1], _dp(bc),
                                   C.byref(o))
    if rc != BIPP_OK:
        raise BippError(rc, bipp_ss_last_error(None))
    return h


def bipp_ss_collect_channels(h, chan, st_xyz, vis, n_eig=None) -> None:
    """Host variant: steps from several channels (chan non-decreasing)."""
    nst, N, st, V = pack_batch(st_xyz, vis)
    ch = np.ascontiguousarray(chan, dtype=np.int32)
    ne = None if n_eig is None else np.ascontiguousarray(n_eig, dtype=np.int32)
    rc = load().bipp_ss_collect_channels(h, len(nst), N, _ip(ch), _ip(nst), None if ne is None else _ip(ne),
                                         C.c_void_p(st.ctypes.data), C.c_void_p(V.ctypes.data), 0, None)
    _check(h, rc)


def bipp_ss_collect_channels_device(h, chan, n_st, d_st, d_vis, n_eig=None, stream=None) -> None:
    """Device variant of bipp_ss_collect_channels (layout as collect_device)."""
    ch = np.ascontiguousarray(chan, dtype=np.int32)
    nst = np.ascontiguousarray(n_st, dtype=np.int32)
    ne = None if n_eig is None else np.ascontiguousarray(n_eig, dtype=np.int32)
    N = int(d_st.shape[-1])
    sp = None if stream is None else C.c_void_p(stream.cuda_stream)
    rc = load().bipp_ss_collect_channels(h, len(nst), N, _ip(ch), _ip(nst), None if ne is None else _ip(ne),
                                         C.c_void_p(d_st.data_ptr()), C.c_void_p(d_vis.data_ptr()), 1, sp)
    _check(h, rc)


def pack_batch(st_xyz: Sequence[np.ndarray], vis: Sequence[np.ndarray], n_st_max: int | None = None):
    """Ragged steps -> the ABI's block layout (n_t blocks of n_st_max x 3 and
    n_st_max x n_st_max complex128, each column-major)."""
    n_t = len(st_xyz)
    nst = np.array([p.shape[0] for p in st_xyz], dtype=np.int32)
    N = int(n_st_max or nst.max())
    st = np.zeros((n_t, 3, N), dtype=np.float64)
    V = np.zeros((n_t, N, N), dtype=np.complex128)  # V[t] holds vis[t].T: column-major block
    for t in range(n_t):
        n = nst[t]
        st[t, :, :n] = np.asarray(st_xyz[t], dtype=np.float64).T
        V[t, :n, :n] = np.asarray(vis[t], dtype=np.complex128).T
    return nst, N, st, V


def bipp_ss_collect(h, st_xyz, vis) -> None:
    p = _colmajor_xyz(st_xyz)
    V = np.ascontiguousarray(np.asarray(vis, dtype=np.complex128).T)
    _check(h, load().bipp_ss_collect(h, p.shape[1], _dp(p), _dp(V.view(np.float64))))


def bipp_ss_collect_batch(h, st_xyz: Sequence[np.ndarray], vis: Sequence[np.ndarray], n_eig=None) -> None:
    nst, N, st, V = pack_batch(st_xyz, vis)
    ne = None if n_eig is None else np.ascontiguousarray(n_eig, dtype=np.int32)
    rc = load().bipp_ss_collect_batch(h, len(nst), N, _ip(nst), None if ne is None else _ip(ne), _dp(st),
                                      _dp(V.view(np.float64)))
    _check(h, rc)


def bipp_ss_collect_batch_packed(h, nst, n_st_max: int, st_addr: int, vis_addr: int, n_eig=None) -> None:
    """bipp_ss_collect_batch on buffers already in the ABI block layout (e.g.
    pinned host tensors); st_addr / vis_addr are host addresses."""
    nst = np.ascontiguousarray(nst, dtype=np.int32)
    ne = None if n_eig is None else np.ascontiguousarray(n_eig, dtype=np.int32)
    rc = load().bipp_ss_collect_batch(h, len(nst), int(n_st_max), _ip(nst), None if ne is None else _ip(ne),
                                      C.cast(C.c_void_p(st_addr), C.POINTER(C.c_double)),
                                      C.cast(C.c_void_p(vis_addr), C.POINTER(C.c_double)))
    _check(h, rc)


def bipp_ss_collect_device(h, n_st, d_st, d_vis, n_eig=None, stream=None) -> None:
    """Device variant. d_st: torch float64 (T, 3, N) contiguous; d_vis: torch
    complex128 or complex64 (T, N, N) contiguous, holding each block
    column-major (i.e. V[t].T, as ``pack_batch`` returns; complex64 goes
    through bipp_ss_collect_device_c64); n_st / n_eig host int sequences;
    stream: a torch.cuda.Stream or None (the handle's stream)."""
    nst = np.ascontiguousarray(n_st, dtype=np.int32)
    ne = None if n_eig is None else np.ascontiguousarray(n_eig, dtype=np.int32)
    N = int(d_st.shape[-1])
    sp = None if stream is None else C.c_void_p(stream.cuda_stream)
    dt = str(d_vis.dtype)
    if (dt not in ("torch.complex128", "torch.complex64") or str(d_st.dtype) != "torch.float64"
            or not d_vis.is_contiguous() or not d_st.is_contiguous()):
        raise ValueError("d_st must be contiguous float64 and d_vis contiguous complex128 or complex64")
    fn = load().bipp_ss_collect_device_c64 if dt == "torch.complex64" else load().bipp_ss_collect_device
    rc = fn(h, len(nst), N, _ip(nst), None if ne is None else _ip(ne), C.c_void_p(d_st.data_ptr()),
            C.c_void_p(d_vis.data_ptr()), sp)
    _check(h, rc)


def bipp_ss_collect_device_c64(h, n_st, d_st, d_vis, n_eig=None, stream=None) -> None:
    """bipp_ss_collect_device with complex64 visibilities (d_vis a torch
    complex64 (T, N, N) tensor, blocks column-major)."""
    if str(d_vis.dtype) != "torch.complex64":
        raise ValueError("d_vis must be complex64")
    bipp_ss_collect_device(h, n_st, d_st, d_vis, n_eig, stream)


def bipp_ss_get(h, n_pix: int, n_level: int, n_chan: int = 1) -> np.ndarray:
    """Images as (n_pix, n_level) (one channel) or (n_chan, n_pix, n_level)."""
    out = np.zeros((n_chan, n_level, n_pix), dtype=np.float32)
    _check(h, load().bipp_ss_get(h, out.ctypes.data_as(C.POINTER(C.c_float))))
    out = np.transpose(out, (0, 2, 1))
    return out[0] if n_chan == 1 else out


def bipp_ss_get_f64(h, n_pix: int, n_level: int, n_chan: int = 1) -> np.ndarray:
    out = np.zeros((n_chan, n_level, n_pix), dtype=np.float64)
    _check(h, load().bipp_ss_get_f64(h, _dp(out)))
    out = np.transpose(out, (0, 2, 1))
    return out[0] if n_chan == 1 else out


def bipp_ss_get_device_f64(h, d_out, stream=None) -> None:
    """d_out: torch float64 (n_level, n_pix) contiguous on the handle's device."""
    sp = None if stream is None else C.c_void_p(stream.cuda_stream)
    _check(h, load().bipp_ss_get_device_f64(h, C.c_void_p(d_out.data_ptr()), sp))


def bipp_ss_reset(h) -> None:
    _check(h, load().bipp_ss_reset(h))


def bipp_ss_set_images(h, img) -> None:
    a = np.ascontiguousarray(np.asarray(img, dtype=np.float64).T)
    _check(h, load().bipp_ss_set_images(h, _dp(a)))


def bipp_ss_last_eigvals(h, n_t_cap: int, n_eig_cap: int):
    nt = C.c_int32(0)
    nk = np.zeros(n_t_cap, dtype=np.int32)
    mu = np.zeros((n_t_cap, n_eig_cap), dtype=np.float64)
    lv = np.zeros((n_t_cap, n_eig_cap), dtype=np.int32)
    _check(h, load().bipp_ss_last_eigvals(h, n_t_cap, n_eig_cap, C.byref(nt), _ip(nk), _dp(mu), _ip(lv)))
    return nt.value, nk, mu, lv


def bipp_ss_get_timings(h) -> dict:
    a = np.zeros(6, dtype=np.float64)
    _check(h, load().bipp_ss_get_timings(h, _dp(a)))
    return {"gram_reduce_ms": a[0], "eig_ms": a[1], "select_ms": a[2], "synth_ms": a[3], "sweeps_total": int(a[4]),
            "launches": int(a[5])}


def bipp_ss_get_synth_shape(h) -> dict:
    a = np.zeros(4, dtype=np.int32)
    _check(h, load().bipp_ss_get_synth_shape(h, a.ctypes.data_as(C.POINTER(C.c_int32))))
    return {"stages": int(a[0]), "fused_mma": bool(a[1]), "epilogue_warps": bool(a[2]), "autotuned": bool(a[3])}


def bipp_ss_get_nufft_timings(h) -> dict:
    a = np.zeros(11, dtype=np.float64)
    _check(h, load().bipp_ss_get_nufft_timings(h, _dp(a)))
    return {"sort_ms": a[0], "spread_ms": a[1], "pad_ms": a[2], "fft_ms": a[3], "interp_ms": a[4],
            "levels_ms": a[5], "grid": (int(a[6]), int(a[7]), int(a[8])), "w": int(a[9]), "points": int(a[10])}


def bipp_ss_debug_fail_wait(h, on: bool) -> None:
    """Fault injection for failure-detection tests: while on, the tensor-core
    synthesis kernel's bounded wait runs out and collects raise
    BIPP_ERR_DEVICE_TIMEOUT (no GPU fault)."""
    _check(h, load().bipp_ss_debug_fail_wait(h, 1 if on else 0))


def bipp_ss_measure_sincos_rate(device: int = -1, repeats: int = 5) -> float:
    """Measured sine + cosine pairs per second of __sincosf on the device (the
    SFU bound of the synthesis' phase generation)."""
    r = C.c_double(0.0)
    rc = load().bipp_ss_measure_sincos_rate(int(device), int(repeats), C.byref(r))
    if rc != BIPP_OK:
        raise BippError(rc, bipp_ss_last_error(None))
    return float(r.value)


def bipp_ss_measure_fma_rates(device: int = -1, repeats: int = 5) -> tuple:
    """Measured (FP32, FP64) FMA rates of the device in flop/s."""
    a, b = C.c_double(0.0), C.c_double(0.0)
    rc = load().bipp_ss_measure_fma_rates(int(device), int(repeats), C.byref(a), C.byref(b))
    if rc != BIPP_OK:
        raise BippError(rc, bipp_ss_last_error(None))
    return float(a.value), float(b.value)


def bipp_ss_destroy(h) -> None:
    if h:
        load().bipp_ss_destroy(h)


def _noalloc_tensor(name, t, dtype, shape):
    """Host-side check of one tensor handed to bipp_ss_collect_noalloc: the
    kernels read or write exactly `shape` elements of `dtype` at its address,
    on the device."""
    if not hasattr(t, "data_ptr") or str(t.dtype) != f"torch.{dtype}":
        raise ValueError(f"{name} must be a torch {dtype} tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def bipp_ss_collect_noalloc(d_pix, wl, level_bounds, n_eig, d_st, d_vis, d_img, filter="lsq",
                            gram_identity=False, stream=None) -> None:
    """One collect() step that allocates no device memory, for callers that
    may not allocate (e.g. a pipeline whose device memory is fixed at
    start-up). All intermediates live in a fixed array inside the library
    (at most BIPP_NOALLOC_MAX_STATIONS stations); calls share it, so do not
    let two calls overlap on one GPU.

    d_pix: torch float64 (3, n_pix) contiguous (column-major n_pix x 3);
    d_st: torch float64 (3, n_st); d_vis: torch complex128 (n_st, n_st)
    holding vis.T (column-major); d_img: torch float64 (n_level, n_pix),
    to which the step's level images are added; level_bounds (n_level, 2).
    Every tensor must be contiguous on the current CUDA device; anything else
    raises ValueError before the library is called."""
    b = np.asarray(level_bounds, dtype=np.float64)
    if b.ndim != 2 or b.shape[1] != 2 or b.shape[0] < 1:
        raise ValueError("level_bounds must be (n_level, 2)")
    if getattr(d_pix, "ndim", 0) != 2 or getattr(d_st, "ndim", 0) != 2:
        raise ValueError("d_pix must be (3, n_pix) and d_st (3, n_st)")
    n_pix, n_st, n_level = int(d_pix.shape[1]), int(d_st.shape[1]), int(b.shape[0])
    _noalloc_tensor("d_pix", d_pix, "float64", (3, n_pix))
    _noalloc_tensor("d_st", d_st, "float64", (3, n_st))
    _noalloc_tensor("d_vis", d_vis, "complex128", (n_st, n_st))
    _noalloc_tensor("d_img", d_img, "float64", (n_level, n_pix))
    named = (("d_pix", d_pix), ("d_st", d_st), ("d_vis", d_vis), ("d_img", d_img))
    for name, t in named:
        if not t.is_cuda:
            raise ValueError(f"{name} must be on a CUDA device, got {t.device}")
    import torch
    cur = torch.cuda.current_device()
    for name, t in named:
        if t.device.index != cur:
            raise ValueError(f"{name} is on {t.device}; the step runs on the current device cuda:{cur}")
    bc = np.ascontiguousarray(b.T)
    msg = C.create_string_buffer(512)
    sp = None if stream is None else C.c_void_p(stream.cuda_stream)
    rc = load().bipp_ss_collect_noalloc(n_pix, C.c_void_p(d_pix.data_ptr()), float(wl), n_level,
                                        _dp(bc), int(n_eig), FILTERS[filter] if isinstance(filter, str) else int(filter),
                                        int(bool(gram_identity)), n_st, C.c_void_p(d_st.data_ptr()),
                                        C.c_void_p(d_vis.data_ptr()), C.c_void_p(d_img.data_ptr()), sp, msg, 512)
    if rc != BIPP_OK:
        raise BippError(rc, msg.value.decode())


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    return None if stream is None else C.c_void_p(stream.cuda_stream)


def _precision_code(precision) -> int:
    if isinstance(precision, str):
        if precision not in ("fp32", "split_bf16", "split_fp16"):
            raise ValueError(f"precision={precision!r}; choose from fp32, split_bf16, split_fp16")
        return PRECISIONS[precision]
    return int(precision)


def bipp_ss_synth_levels_device(pix_cm, wl, st_cm, W_cm, d, level, gains, img, precision="fp32",
                                stream=None) -> None:
    """Forward of the differentiable synthesis on torch CUDA tensors in the ABI
    layout: pix_cm (3, n_pix) f64, st_cm (T, 3, n_st) f64, W_cm (T, n_eig, n_st)
    c128 (column-major blocks), d (T, n_eig) f64, level (T, n_eig) int32,
    gains (n_st,) c128, img (n_level, n_pix) f64 output; precision "fp32"
    (CUDA cores) or "split_fp16" / "split_bf16" (tensor cores)."""
    T, K, N = W_cm.shape
    rc = load().bipp_ss_synth_levels_device(int(pix_cm.shape[1]), _ptr(pix_cm), float(wl), T, N, K,
                                            int(img.shape[0]), _ptr(st_cm), _ptr(W_cm), _ptr(d), _ptr(level),
                                            _ptr(gains), _ptr(img), _precision_code(precision),
                                            _stream_ptr(stream))
    if rc != BIPP_OK:
        raise BippError(rc, "synth_levels_device failed")


def bipp_ss_synth_adjoint_device(pix_cm, wl, st_cm, W_cm, d, level, gains, grad_img, grad_W_cm, grad_g,
                                 precision="fp32", stream=None) -> None:
    """Adjoint of bipp_ss_synth_levels_device; grad_img (n_level, n_pix) f64,
    outputs grad_W_cm (T, n_eig, n_st) c128 and grad_g (n_st,) c128."""
    T, K, N = W_cm.shape
    rc = load().bipp_ss_synth_adjoint_device(int(pix_cm.shape[1]), _ptr(pix_cm), float(wl), T, N, K,
                                             int(grad_img.shape[0]), _ptr(st_cm), _ptr(W_cm), _ptr(d),
                                             _ptr(level), _ptr(gains), _ptr(grad_img), _ptr(grad_W_cm),
                                             _ptr(grad_g), _precision_code(precision), _stream_ptr(stream))
    if rc != BIPP_OK:
        raise BippError(rc, "synth_adjoint_device failed")


class StandardSynthesis:
    """Handle wrapper: create once, collect per step (or per batch), get images."""

    def __init__(self, pix_xyz, wl, level_bounds, **opts):
        self.n_pix = int(np.asarray(pix_xyz).shape[0])
        self.n_level = int(opts["n_eig"]) if level_bounds is None else int(np.asarray(level_bounds).shape[0])
        self.h = None
        self.h = bipp_ss_create(pix_xyz, wl, level_bounds, **opts)

    def collect(self, st_xyz, vis):
        bipp_ss_collect(self.h, st_xyz, vis)

    def collect_batch(self, st_xyz, vis, n_eig=None):
        bipp_ss_collect_batch(self.h, st_xyz, vis, n_eig)

    def get(self, f64=True):
        if f64:
            return bipp_ss_get_f64(self.h, self.n_pix, self.n_level)
        return bipp_ss_get(self.h, self.n_pix, self.n_level)

    def reset(self):
        bipp_ss_reset(self.h)

    def timings(self):
        return bipp_ss_get_timings(self.h)

    def nufft_timings(self):
        return bipp_ss_get_nufft_timings(self.h)

    def synth_shape(self):
        return bipp_ss_get_synth_shape(self.h)

    def close(self):
        if self.h:
            bipp_ss_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def bipp_ss_quantile_bounds(pooled_mu, n_level: int) -> np.ndarray:
    """Level intervals (n_level, 2) rows [lo, hi) at the quantiles of the
    pooled eigenvalues (bipp_ss_quantile_bounds): inner edges halfway between
    neighbouring values at the 1/n_level quantiles, outer edges +-inf, level 0
    holding the largest eigenvalues."""
    v = np.ascontiguousarray(pooled_mu, dtype=np.float64).ravel()
    out = np.zeros(2 * n_level, dtype=np.float64)
    rc = load().bipp_ss_quantile_bounds(v.shape[0], _dp(v), int(n_level), _dp(out))
    if rc != BIPP_OK:
        raise BippError(rc, bipp_ss_last_error(None))
    return np.ascontiguousarray(out.reshape(2, n_level).T)


quantile_level_bounds = bipp_ss_quantile_bounds


def bipp_ss_energy_neig(mu_desc, fraction: float) -> int:
    """Least number of leading eigenpairs holding `fraction` of the positive energy."""
    mu = np.ascontiguousarray(mu_desc, dtype=np.float64)
    k = C.c_int32(0)
    rc = load().bipp_ss_energy_neig(mu.shape[0], _dp(mu), float(fraction), C.byref(k))
    if rc != BIPP_OK:
        raise BippError(rc, bipp_ss_last_error(None))
    return int(k.value)


def bipp_ss_kmeans_bounds(values, n_level: int) -> np.ndarray:
    """Level intervals (n_level, 2) rows [lo, hi) from 1-D k-means of the values."""
    v = np.ascontiguousarray(values, dtype=np.float64).ravel()
    out = np.zeros(2 * n_level, dtype=np.float64)
    rc = load().bipp_ss_kmeans_bounds(v.shape[0], _dp(v), int(n_level), _dp(out))
    if rc != BIPP_OK:
        raise BippError(rc, bipp_ss_last_error(None))
    return np.ascontiguousarray(out.reshape(2, n_level).T)


def _prepass_eigvals(st_xyz, vis, wl, n_eig, **opts):
    """GPU Gram + eigensolve of the given steps (synthesis on one pixel only);
    returns each step's kept eigenvalues, descending. n_eig: one count or one
    per step."""
    one_px = np.array([[0.0, 0.0, 1.0]])
    opts = {k: v for k, v in opts.items() if k != "n_eig"}
    per_step = None if np.isscalar(n_eig) else [int(k) for k in n_eig]
    k_max = int(n_eig) if per_step is None else max(per_step)
    with StandardSynthesis(one_px, wl, np.array([[-math.inf, math.inf]]), n_eig=k_max, **opts) as ss:
        ss.collect_batch(st_xyz, vis, per_step)
        nt, nk, mu, _ = bipp_ss_last_eigvals(ss.h, len(vis), k_max)
    return [mu[t, : nk[t]] for t in range(nt)]


def estimate_level_bounds(st_xyz, vis, wl, n_eig, n_level, method: str = "quantile", **opts):
    """Parameter-estimation pre-pass (Table tts): run the GPU Gram + eigensolve
    on the given steps, pool the kept eigenvalues and derive level bounds by
    quantiles or by k-means clustering (Sec. 2.6). Returns (bounds, pooled)."""
    pooled = np.concatenate(_prepass_eigvals(st_xyz, vis, wl, n_eig, **opts))
    if method == "kmeans":
        return bipp_ss_kmeans_bounds(pooled, n_level), pooled
    if method != "quantile":
        raise ValueError(f"unknown method {method!r}")
    return quantile_level_bounds(pooled, n_level), pooled


def estimate_n_eig(st_xyz, vis, wl, fraction: float, **opts) -> int:
    """Truncation of Sec. 2.6 estimated from an observation: the least number
    of leading eigenpairs holding `fraction` of each step's energy, maximised
    over the given steps (all eigenpairs are solved for in the pre-pass)."""
    steps = _prepass_eigvals(st_xyz, vis, wl, [int(np.asarray(p).shape[0]) for p in st_xyz], **opts)
    return max(bipp_ss_energy_neig(mu, fraction) for mu in steps)
