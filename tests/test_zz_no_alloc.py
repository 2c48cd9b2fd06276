"""The no-allocation collect step against the regular handle-based one.

bipp_ss_collect_noalloc serves callers that may not allocate device memory
(for example a pipeline whose GPU memory is reserved once at start-up): it
keeps every intermediate in one fixed array inside the library. Its images
must match what the ordinary handle produces with the FP64 synthesis, within
the FP64 tolerance of the parity tests, over two calls in a row (the second
call reuses the array the first one left behind). This file is collected
last on purpose.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_2310_09200_b300 import bipp_ss, inputs

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-9  # relative L2 per level image, as for the FP64 path elsewhere


def _rel_l2(a, b):
    return np.array([np.linalg.norm(a[:, l] - b[:, l]) / max(np.linalg.norm(b[:, l]), 1e-300)
                     for l in range(b.shape[1])])


def test_noalloc_matches_handle_on_two_consecutive_calls():
    import torch
    inp = inputs.make_config(0, n_t=2, n_side=20)
    bounds = np.array([[200.0, np.inf], [50.0, 200.0], [-np.inf, 50.0]])
    n_eig = inp.n_eig

    dev = torch.device("cuda:0")
    d_pix = torch.from_numpy(np.ascontiguousarray(inp.pix.T)).to(dev)
    d_img = torch.zeros((bounds.shape[0], inp.n_pix), dtype=torch.float64, device=dev)
    with bipp_ss.StandardSynthesis(inp.pix, inp.wl, bounds, n_eig=n_eig, precision="fp64") as ss:
        for t in range(2):
            d_st = torch.from_numpy(np.ascontiguousarray(inp.st_xyz[t].T)).to(dev)
            d_vis = torch.from_numpy(np.ascontiguousarray(inp.vis[t].T)).to(dev)
            bipp_ss.bipp_ss_collect_noalloc(d_pix, inp.wl, bounds, n_eig, d_st, d_vis, d_img)
            torch.cuda.synchronize()
            ss.collect(inp.st_xyz[t], inp.vis[t])
            want = ss.get()
            got = d_img.cpu().numpy().T
            err = _rel_l2(got, want)
            assert np.all(err <= TOL_FP64), (t, err)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
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
