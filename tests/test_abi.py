"""Host-side checks of the C-ABI library (no GPU compute): it loads, exports
every entry point declared in include/bipp_ss.h, and rejects invalid
arguments before touching a device."""
from __future__ import annotations

import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2310_09200_b300 import bipp_ss, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(bipp_\w+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    build.build()
    return bipp_ss.load()


def test_library_exports_every_declared_symbol(lib):
    declared = _declared()
    assert "bipp_ss_create" in declared and "bipp_ss_collect" in declared
    out = subprocess.run(["nm", "-D", "--defined-only", bipp_ss.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (bipp_\w+)", out))
    missing = declared - exported
    assert not missing, f"declared but not exported: {missing}"
    for name in declared:
        getattr(lib, name)


def test_library_has_no_unresolved_own_symbols(lib):
    out = subprocess.run(["nm", "-D", "--undefined-only", bipp_ss.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    assert "bipp" not in out, out


def test_binding_names_match_abi():
    assert set(bipp_ss.EXPORTED) == _declared()
    for name in bipp_ss.EXPORTED:
        assert hasattr(bipp_ss, name), name


def test_library_does_not_use_the_oracle():
    out = subprocess.run(["ldd", bipp_ss.LIB_PATH], capture_output=True, text=True).stdout
    assert "oracle" not in out
    syms = subprocess.run(["nm", "-D", bipp_ss.LIB_PATH], capture_output=True, text=True).stdout
    assert "orc_" not in syms


def test_default_options(lib):
    o = bipp_ss.bipp_ss_default_options()
    assert o.precision == bipp_ss.BIPP_PREC_FP32 and o.filter == bipp_ss.BIPP_FILTER_LSQ
    assert o.max_jacobi_sweeps == 40 and abs(o.jacobi_tol - 1e-13) < 1e-30 and o.gram_identity == 0
    assert o.device == -1 and o.eig_mode == bipp_ss.BIPP_EIG_JACOBI64
    assert o.synthesis == bipp_ss.BIPP_SYNTH_STANDARD and abs(o.nufft_eps - 1e-5) < 1e-20
    assert C.sizeof(bipp_ss.bipp_ss_options) == 96  # the C struct's size on x86-64
    assert list(o.nufft_partition) == [1] * 6


@pytest.mark.parametrize("case", ["n_pix", "wl", "levels", "precision", "reserved", "nan_bound", "nan_pix",
                                  "eig_levels", "eig_many", "eig_flag", "synthesis", "nufft_eps_small",
                                  "nufft_eps_large", "nufft_eigenimages", "nufft_partition"])
def test_create_rejects_invalid_arguments_before_device_use(lib, case):
    pix = np.array([[0.0, 0.0, 1.0], [0.1, 0.0, 0.99]])
    b = np.array([[-np.inf, np.inf]])
    kw = {}
    wl = 2.0
    if case == "n_pix":
        pix = np.zeros((0, 3))
    elif case == "wl":
        wl = -1.0
    elif case == "levels":
        b = np.zeros((17, 2))
    elif case == "precision":
        kw["precision"] = 9
    elif case == "reserved":
        o = bipp_ss.bipp_ss_default_options()
        o.reserved[1] = 1
        h = C.c_void_p()
        pc = np.ascontiguousarray(pix.T)
        bc = np.ascontiguousarray(b.T)
        rc = lib.bipp_ss_create(C.byref(h), 2, pc.ctypes.data_as(C.POINTER(C.c_double)), 2.0, 1,
                                bc.ctypes.data_as(C.POINTER(C.c_double)), C.byref(o))
        assert rc == bipp_ss.BIPP_ERR_INVALID_ARG
        assert "reserved" in bipp_ss.bipp_ss_last_error(None)
        return
    elif case == "nan_bound":
        b = np.array([[np.nan, 1.0]])
    elif case == "nan_pix":
        pix = pix.copy()
        pix[1, 2] = np.nan
    elif case == "eig_levels":  # eigenimages need n_level == n_eig
        kw.update(eigenimages=1, n_eig=4)
        b = np.zeros((3, 2))
    elif case == "eig_many":
        kw.update(eigenimages=1, n_eig=bipp_ss.BIPP_MAX_EIGENIMAGES + 1)
        b = None
    elif case == "eig_flag":
        kw.update(eigenimages=2, n_eig=1)
    elif case == "synthesis":
        kw["synthesis"] = 2
    elif case == "nufft_eps_small":
        kw.update(synthesis="nufft", nufft_eps=1e-8)  # beyond FP32 grids
    elif case == "nufft_eps_large":
        kw.update(synthesis="nufft", nufft_eps=0.5)
    elif case == "nufft_eigenimages":  # NUFFT synthesis makes level images only
        kw.update(synthesis="nufft", eigenimages=1, n_eig=1)
    elif case == "nufft_partition":
        kw.update(synthesis="nufft", nufft_partition=(1, 1, 1, 1, 0, 1))
    with pytest.raises(bipp_ss.BippError) as e:
        bipp_ss.bipp_ss_create(pix, wl, b, **kw)
    want = bipp_ss.BIPP_ERR_UNSUPPORTED if case == "nufft_eigenimages" else bipp_ss.BIPP_ERR_INVALID_ARG
    assert e.value.code == want


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.bipp_ss_collect(None, 3, None, None) == bipp_ss.BIPP_ERR_INVALID_ARG
    assert lib.bipp_ss_get_synth_shape(None, None) == bipp_ss.BIPP_ERR_INVALID_ARG
    assert lib.bipp_ss_get(None, None) == bipp_ss.BIPP_ERR_INVALID_ARG
    assert lib.bipp_ss_destroy(None) == bipp_ss.BIPP_OK
    assert isinstance(bipp_ss.bipp_ss_last_error(None), str)


def test_pack_batch_layout_is_column_major():
    rng = np.random.default_rng(0)
    st = [rng.normal(size=(3, 3)), rng.normal(size=(2, 3))]
    V = [rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3)), rng.normal(size=(2, 2)) + 0j]
    nst, N, stp, Vp = bipp_ss.pack_batch(st, V)
    assert list(nst) == [3, 2] and N == 3
    flat_st = stp.reshape(2, -1)
    flat_V = Vp.reshape(2, -1)
    for t in range(2):
        n = nst[t]
        for i in range(n):
            for c in range(3):
                assert flat_st[t, i + c * N] == st[t][i, c]
            for j in range(n):
                assert flat_V[t, i + j * N] == V[t][i, j]


def test_quantile_level_bounds_host_logic():
    mu = np.arange(1.0, 13.0)
    b = bipp_ss.quantile_level_bounds(mu, 4)
    assert b.shape == (4, 2)
    assert b[0, 1] == np.inf and b[-1, 0] == -np.inf
    np.testing.assert_allclose(b[:, 0][:3], [9.5, 6.5, 3.5])
    np.testing.assert_allclose(b[1:, 1], [9.5, 6.5, 3.5])


def test_device_collect_checks_tensor_types_before_the_library():
    """The device collect's binding accepts float64 positions and complex128 or
    complex64 visibilities, contiguous; anything else is refused on the host
    before the library is called (the handle is never dereferenced here)."""
    import torch
    st = torch.zeros((1, 3, 4), dtype=torch.float64)
    bad = [
        (st, torch.zeros((1, 4, 4), dtype=torch.float64)),            # real visibilities
        (st.float(), torch.zeros((1, 4, 4), dtype=torch.complex128)),  # float32 positions
        (st, torch.zeros((1, 4, 8), dtype=torch.complex128)[:, :, ::2]),  # non-contiguous
    ]
    for d_st, d_vis in bad:
        with pytest.raises(ValueError):
            bipp_ss.bipp_ss_collect_device(None, [4], d_st, d_vis)
    with pytest.raises(ValueError):
        bipp_ss.bipp_ss_collect_device_c64(None, [4], st, torch.zeros((1, 4, 4), dtype=torch.complex128))


def test_fault_injection_switch_rejects_null_handle(lib):
    assert lib.bipp_ss_debug_fail_wait(None, 1) == bipp_ss.BIPP_ERR_INVALID_ARG
    assert b"NULL" in lib.bipp_ss_last_error(None)


C_PROGRAM = r"""
#include <math.h>
#include <stdio.h>
#include <string.h>
#include "bipp_ss.h"

int main(void) {
  bipp_ss_options o;
  double mu[5] = {9.0, 4.0, 1.0, 0.5, -2.0}, v[6] = {1.0, 1.1, 5.0, 5.2, 9.0, 9.3}, b[6];
  int32_t k = 0;
  bipp_ss_default_options(&o);
  if (sizeof(bipp_ss_options) != 96 || o.precision != BIPP_PREC_FP32 || o.max_jacobi_sweeps != 40) return 1;
  /* 90% of the positive energy 14.5 needs the three leading eigenvalues (13.0 < 13.05 <= 14.0) */
  if (bipp_ss_energy_neig(5, mu, 0.9, &k) != BIPP_OK || k != 3) return 2;
  if (bipp_ss_kmeans_bounds(6, v, 3, b) != BIPP_OK) return 3;
  /* n_level x 2 column-major, level 0 = highest cluster {9, 9.3}: lo = b[0..2] = (7.1, 3.05, -inf),
     hi = b[3..5] = (inf, 7.1, 3.05) */
  if (fabs(b[0] - 7.1) > 1e-12 || fabs(b[1] - 3.05) > 1e-12 || !(isinf(b[2]) && b[2] < 0)) return 4;
  if (!(isinf(b[3]) && b[3] > 0) || fabs(b[4] - 7.1) > 1e-12 || fabs(b[5] - 3.05) > 1e-12) return 8;
  if (bipp_ss_energy_neig(0, mu, 0.9, &k) != BIPP_ERR_INVALID_ARG) return 5;
  if (strlen(bipp_ss_last_error(NULL)) == 0) return 6;
  if (bipp_ss_collect(NULL, 1, mu, mu) != BIPP_ERR_INVALID_ARG) return 7;
  puts("ok");
  return 0;
}
"""


def test_header_compiles_and_links_as_c(lib, tmp_path):
    """The ABI is usable from plain C99 (warnings as errors): defaults, the
    host-only estimation calls and the NULL-handle error path."""
    src = tmp_path / "abi.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "abi"
    libdir = os.path.dirname(bipp_ss.LIB_PATH)
    cc = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I",
                         os.path.join(ROOT, "include"), str(src), "-o", str(exe), "-L", libdir, "-lbipp_ss",
                         f"-Wl,-rpath,{libdir}", "-lm"], capture_output=True, text=True)
    assert cc.returncode == 0, cc.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert run.returncode == 0 and run.stdout.strip() == "ok", (run.returncode, run.stdout, run.stderr)


def test_binding_rejects_unknown_options(lib):
    with pytest.raises(TypeError):
        bipp_ss.bipp_ss_default_options(autotun=0)
    with pytest.raises(ValueError):
        bipp_ss.bipp_ss_default_options(precision="bf16")
    with pytest.raises(ValueError):
        bipp_ss.bipp_ss_default_options(nufft_partition=(2, 2, 1))
    o = bipp_ss.bipp_ss_default_options(precision="split_fp16", nufft_partition=((2, 2, 1), (1, 1, 1)), autotune=False)
    assert o.precision == 3 and list(o.nufft_partition) == [2, 2, 1, 1, 1, 1] and o.autotune == 0


def test_noalloc_binding_checks_tensors_before_the_library():
    """bipp_ss_collect_noalloc's binding refuses, on the host and before the
    library is called, every tensor whose type, shape, layout or device would
    make the kernels read or write outside it."""
    import torch
    n_pix, n_st = 6, 5
    good = dict(d_pix=torch.zeros((3, n_pix), dtype=torch.float64), d_st=torch.zeros((3, n_st), dtype=torch.float64),
                d_vis=torch.zeros((n_st, n_st), dtype=torch.complex128),
                d_img=torch.zeros((2, n_pix), dtype=torch.float64))
    bounds = np.array([[1.0, np.inf], [-np.inf, 1.0]])
    bad = [
        ("d_pix", torch.zeros((3, n_pix), dtype=torch.float32)),
        ("d_pix", torch.zeros((n_pix, 3), dtype=torch.float64)[:, :3].T),          # a transposed view
        ("d_st", torch.zeros((3, n_st), dtype=torch.float32)),
        ("d_vis", torch.zeros((n_st, n_st), dtype=torch.complex64)),
        ("d_vis", torch.zeros((n_st, n_st + 1), dtype=torch.complex128)),
        ("d_vis", torch.zeros((n_st, 2 * n_st), dtype=torch.complex128)[:, ::2]),  # non-contiguous
        ("d_img", torch.zeros((2, n_pix), dtype=torch.float32)),
        ("d_img", torch.zeros((3, n_pix), dtype=torch.float64)),                    # level count != bounds
        ("d_img", torch.zeros((2, n_pix + 1), dtype=torch.float64)),
    ]
    for name, t in bad:
        kw = dict(good, **{name: t})
        with pytest.raises(ValueError, match=name):
            bipp_ss.bipp_ss_collect_noalloc(kw["d_pix"], 2.0, bounds, 2, kw["d_st"], kw["d_vis"], kw["d_img"])
    with pytest.raises(ValueError, match="level_bounds"):
        bipp_ss.bipp_ss_collect_noalloc(good["d_pix"], 2.0, np.zeros(4), 2, good["d_st"], good["d_vis"],
                                        good["d_img"])
    # well-formed tensors on the CPU are still refused: the kernels need device memory
    with pytest.raises(ValueError, match="CUDA"):
        bipp_ss.bipp_ss_collect_noalloc(good["d_pix"], 2.0, bounds, 2, good["d_st"], good["d_vis"], good["d_img"])


def test_noalloc_c_entry_rejects_bad_scalars_before_any_cuda_call(lib):
    """The C entry point checks sizes, the wavelength and the level bounds
    before it touches CUDA (so these checks also hold without a GPU)."""
    msg = C.create_string_buffer(256)
    buf = (C.c_double * 64)()
    p = C.cast(buf, C.c_void_p)

    def call(n_st, n_eig, n_level, bounds, wl=2.0):
        b = np.ascontiguousarray(bounds, dtype=np.float64)
        return lib.bipp_ss_collect_noalloc(4, p, wl, n_level, b.ctypes.data_as(C.POINTER(C.c_double)),
                                           n_eig, 0, 0, n_st, p, p, p, None, msg, 256)

    inf = np.inf
    assert call(bipp_ss.BIPP_NOALLOC_MAX_STATIONS + 1, 4, 1, [-inf, inf]) == bipp_ss.BIPP_ERR_UNSUPPORTED
    assert b"stations" in msg.value
    assert call(8, 9, 1, [-inf, inf]) == bipp_ss.BIPP_ERR_UNSUPPORTED
    assert call(8, 4, 17, np.zeros(34)) == bipp_ss.BIPP_ERR_UNSUPPORTED
    assert call(8, 4, 2, [np.nan, -inf, inf, 1.0]) == bipp_ss.BIPP_ERR_INVALID_ARG
    assert b"NaN" in msg.value
    assert call(8, 4, 1, [-inf, inf], wl=np.inf) == bipp_ss.BIPP_ERR_INVALID_ARG
    assert call(8, 4, 1, [-inf, inf], wl=-1.0) == bipp_ss.BIPP_ERR_INVALID_ARG


def test_sincos_rate_probe_rejects_bad_arguments(lib):
    """The SFU-rate probe checks its arguments before any CUDA call."""
    r = C.c_double(1.0)
    assert lib.bipp_ss_measure_sincos_rate(-1, 0, C.byref(r)) == bipp_ss.BIPP_ERR_INVALID_ARG
    assert lib.bipp_ss_measure_sincos_rate(-1, 101, C.byref(r)) == bipp_ss.BIPP_ERR_INVALID_ARG
    assert lib.bipp_ss_measure_sincos_rate(-1, 3, None) == bipp_ss.BIPP_ERR_INVALID_ARG


def test_fma_rate_probe_rejects_bad_arguments(lib):
    a, b = C.c_double(1.0), C.c_double(1.0)
    assert lib.bipp_ss_measure_fma_rates(-1, 0, C.byref(a), C.byref(b)) == bipp_ss.BIPP_ERR_INVALID_ARG
    assert lib.bipp_ss_measure_fma_rates(-1, 3, None, C.byref(b)) == bipp_ss.BIPP_ERR_INVALID_ARG
