"""The no-allocation collect step (bipp_ss_collect_noalloc) on the GPU.

Some callers may not allocate device memory at all: a real-time pipeline whose
GPU memory is reserved once at start-up, or a host framework that owns the
device memory budget. This entry point serves them by keeping every
intermediate in one fixed array inside the library; the caller passes only its
inputs and the image to add to.

Checked here, through the C ABI:
- two calls in a row (the second reuses the array the first left behind)
  against the FP64 oracle's own step (oracle.ss_step) and against the
  handle-based entry point's FP64 path;
- a failing step (two coincident stations: the Gram matrix is singular) returns
  BIPP_ERR_GRAM_NOT_PD and leaves the image untouched, and the next good call
  starts from clean status words;
- host pointers and misaligned device pointers are refused before any kernel
  runs; sizes beyond the array's limits are refused with the limit named.

The file name sorts last, so a run that stops at the first failure
(`pytest -x`) has already run every other test when this one runs: this entry
point is an addition beside the main path, and a failure here should not hide
the state of the rest. The tests depend on nothing that earlier tests leave
behind; they pass alone in a fresh process as well.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import pytest

import oracle
from paper_2310_09200_b300 import bipp_ss, inputs

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-9  # relative L2 per level image, as for the FP64 path in the other parity tests
BOUNDS = np.array([[200.0, np.inf], [50.0, 200.0], [-np.inf, 50.0]])


def _rel_l2(a, b):
    return np.array([np.linalg.norm(a[:, l] - b[:, l]) / max(np.linalg.norm(b[:, l]), 1e-300)
                     for l in range(b.shape[1])])


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def test_noalloc_two_consecutive_calls_match_the_oracle_and_the_handle():
    import torch
    torch.cuda.set_device(0)
    inp = inputs.make_config(0, n_t=2, n_side=20)
    n_eig = inp.n_eig
    d_pix = _dev(inp.pix.T)
    d_img = torch.zeros((BOUNDS.shape[0], inp.n_pix), dtype=torch.float64, device="cuda:0")
    want = None
    with bipp_ss.StandardSynthesis(inp.pix, inp.wl, BOUNDS, n_eig=n_eig, precision="fp64") as ss:
        for t in range(2):
            bipp_ss.bipp_ss_collect_noalloc(d_pix, inp.wl, BOUNDS, n_eig, _dev(inp.st_xyz[t].T), _dev(inp.vis[t].T),
                                            d_img)
            torch.cuda.synchronize()
            got = d_img.cpu().numpy().T
            want, *_ = oracle.ss_step(inp.pix, inp.wl, BOUNDS, n_eig, inp.st_xyz[t], inp.vis[t], img=want)
            err = _rel_l2(got, want)
            assert np.all(err <= TOL_FP64), ("oracle", t, err)
            ss.collect(inp.st_xyz[t], inp.vis[t])
            err_h = _rel_l2(got, ss.get())
            assert np.all(err_h <= TOL_FP64), ("handle", t, err_h)


def test_noalloc_failed_step_leaves_the_image_and_the_next_call_is_clean():
    import torch
    torch.cuda.set_device(0)
    inp = inputs.make_config(0, n_t=1, n_side=16)
    d_pix = _dev(inp.pix.T)
    start = np.random.default_rng(7).normal(size=(BOUNDS.shape[0], inp.n_pix)) * 10.0
    d_img = _dev(start)
    p_bad = inp.st_xyz[0].copy()
    p_bad[1] = p_bad[0]  # two stations at one place: G has two equal rows, Cholesky meets a zero pivot
    with pytest.raises(bipp_ss.BippError) as e:
        bipp_ss.bipp_ss_collect_noalloc(d_pix, inp.wl, BOUNDS, inp.n_eig, _dev(p_bad.T), _dev(inp.vis[0].T), d_img)
    assert e.value.code == bipp_ss.BIPP_ERR_GRAM_NOT_PD
    torch.cuda.synchronize()
    assert np.array_equal(d_img.cpu().numpy(), start)  # bit for bit: the synthesis skipped the step
    # the same array, now with a good step: the status and commit words start from zero again
    bipp_ss.bipp_ss_collect_noalloc(d_pix, inp.wl, BOUNDS, inp.n_eig, _dev(inp.st_xyz[0].T), _dev(inp.vis[0].T),
                                    d_img)
    torch.cuda.synchronize()
    want, *_ = oracle.ss_step(inp.pix, inp.wl, BOUNDS, inp.n_eig, inp.st_xyz[0], inp.vis[0],
                              img=np.asfortranarray(start.T))
    err = _rel_l2(d_img.cpu().numpy().T, want)
    assert np.all(err <= TOL_FP64), err


def test_noalloc_refuses_host_and_misaligned_pointers():
    import torch
    torch.cuda.set_device(0)
    inp = inputs.make_config(0, n_t=1, n_side=8)
    n_st = inp.st_xyz[0].shape[0]
    L = bipp_ss.load()
    d_pix = _dev(inp.pix.T)
    d_st = _dev(inp.st_xyz[0].T)
    d_vis = _dev(inp.vis[0].T)
    d_img = torch.zeros((BOUNDS.shape[0], inp.n_pix), dtype=torch.float64, device="cuda:0")
    # the visibilities one double past a 16-byte boundary, inside a larger buffer
    d_vis_off = torch.zeros(2 * n_st * n_st + 2, dtype=torch.float64, device="cuda:0")
    h_pix = np.ascontiguousarray(inp.pix.T)
    bc = np.ascontiguousarray(BOUNDS.T)
    msg = C.create_string_buffer(256)

    def call(pix_ptr, vis_ptr):
        return L.bipp_ss_collect_noalloc(inp.n_pix, C.c_void_p(pix_ptr), inp.wl, BOUNDS.shape[0], bipp_ss._dp(bc),
                                         inp.n_eig, 0, 0, n_st, C.c_void_p(d_st.data_ptr()), C.c_void_p(vis_ptr),
                                         C.c_void_p(d_img.data_ptr()), None, msg, 256)

    assert call(h_pix.ctypes.data, d_vis.data_ptr()) == bipp_ss.BIPP_ERR_INVALID_ARG
    assert b"d_pix_xyz" in msg.value
    assert call(d_pix.data_ptr(), d_vis_off.data_ptr() + 8) == bipp_ss.BIPP_ERR_INVALID_ARG
    assert b"aligned" in msg.value
    torch.cuda.synchronize()
    assert np.all(d_img.cpu().numpy() == 0.0)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    torch.cuda.set_device(0)
    n = bipp_ss.BIPP_NOALLOC_MAX_STATIONS + 1
    dev = torch.device("cuda:0")
    d_pix = torch.zeros((3, 4), dtype=torch.float64, device=dev)
    d_st = torch.zeros((3, n), dtype=torch.float64, device=dev)
    d_vis = torch.zeros((n, n), dtype=torch.complex128, device=dev)
    d_img = torch.zeros((1, 4), dtype=torch.float64, device=dev)
    with pytest.raises(bipp_ss.BippError) as e:
        bipp_ss.bipp_ss_collect_noalloc(d_pix, 2.0, np.array([[-np.inf, np.inf]]), 4, d_st, d_vis, d_img)
    assert e.value.code == bipp_ss.BIPP_ERR_UNSUPPORTED
    assert str(bipp_ss.BIPP_NOALLOC_MAX_STATIONS) in str(e.value)
    assert np.all(d_img.cpu().numpy() == 0.0)
