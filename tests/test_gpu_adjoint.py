"""Differentiation: the CUDA forward and adjoint (through the C ABI and the
torch.autograd glue) against the FP64 oracle's forward and gradient, which
is itself pinned to central finite differences in test_oracle_pins.

Both arithmetic paths are checked: "fp32" (CUDA cores) and the tensor-core
path ("split_fp16", "split_bf16": the forward is the tcgen05 synthesis kernel
on W' = diag(conj g) W; the adjoint recomputes z with it and contracts Phi^T Y
over pixels on the tensor cores).

Tolerances: forward level images 1e-5 relative L2 (FP32 and split FP16;
1e-4 for split BF16, whose bound is 1e-3); gradients 1e-4 relative (norm of
the difference over the norm of the oracle gradient).
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2310_09200_b300 import inputs

pytestmark = pytest.mark.gpu


def _problem(n_st, side, T, K, n_level, seed, cap=10.0):
    rng = np.random.default_rng(seed)
    full = inputs.make_config(4, n_t=T, n_side=side) if n_st > 24 else inputs.make_config(0, n_t=T, n_side=side)
    st = np.stack([p[:n_st] for p in full.st_xyz])
    pix = inputs.pixel_grid(side, cap)
    W = (rng.normal(size=(T, n_st, K)) + 1j * rng.normal(size=(T, n_st, K))) / np.sqrt(n_st)
    d = np.abs(rng.normal(size=(T, K))) * 50.0 + 1.0
    lev = rng.integers(-1, n_level, size=(T, K)).astype(np.int32)
    g = inputs.gains(n_st, 0.05, rng)
    return full.wl, pix, st, W, d, lev, g, rng


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


FWD_TOL = {"fp32": 1e-5, "split_fp16": 1e-5, "split_bf16": 1e-4}


@pytest.mark.parametrize("precision", ["fp32", "split_fp16", "split_bf16"])
@pytest.mark.parametrize("case", [(16, 32, 2, 6, 2), (256, 64, 4, 32, 4), (77, 21, 3, 70, 3), (130, 45, 2, 64, 3)])
def test_forward_and_gradients_match_oracle(case, precision):
    import torch
    from paper_2310_09200_b300.autograd import synth_levels
    n_st, side, T, K, n_level = case
    if precision != "fp32" and K > 64:
        pytest.skip("the tensor-core adjoint takes n_eig <= 64")
    wl, pix, st, W, d, lev, g, rng = _problem(n_st, side, T, K, n_level, seed=31 + n_st)
    n_pix = pix.shape[0]
    target = np.abs(rng.normal(size=(n_pix, n_level))) * 1e3
    loss_o, img_o, gg_o, gW_o = oracle.grad(pix, wl, n_level, st, W, d, lev, g, target)

    dev = torch.device("cuda:0")
    tW = torch.tensor(W, device=dev, requires_grad=True)
    tg = torch.tensor(g, device=dev, requires_grad=True)
    img = synth_levels(torch.tensor(pix, device=dev), torch.tensor(st, device=dev), tW,
                       torch.tensor(d, device=dev), torch.tensor(lev, device=dev), tg, wl, n_level, precision)
    assert img.shape == (n_pix, n_level)
    img_np = img.detach().cpu().numpy()
    for l in range(n_level):
        if np.linalg.norm(img_o[:, l]) > 0:
            assert _rel(img_np[:, l], img_o[:, l]) <= FWD_TOL[precision], (l, _rel(img_np[:, l], img_o[:, l]))
    loss = ((img - torch.tensor(target, device=dev)) ** 2).sum()
    loss.backward()
    assert abs(loss.item() - loss_o) <= 1e-4 * loss_o
    assert _rel(tg.grad.cpu().numpy(), gg_o) <= 1e-4, _rel(tg.grad.cpu().numpy(), gg_o)
    assert _rel(tW.grad.cpu().numpy(), gW_o) <= 1e-4, _rel(tW.grad.cpu().numpy(), gW_o)


@pytest.mark.parametrize("precision", ["fp32", "split_fp16"])
def test_adjoint_is_deterministic(precision):
    import torch
    from paper_2310_09200_b300.autograd import synth_levels
    wl, pix, st, W, d, lev, g, rng = _problem(48, 40, 2, 16, 2, seed=5)
    dev = torch.device("cuda:0")
    grads = []
    for _ in range(2):
        tW = torch.tensor(W, device=dev, requires_grad=True)
        tg = torch.tensor(g, device=dev, requires_grad=True)
        img = synth_levels(torch.tensor(pix, device=dev), torch.tensor(st, device=dev), tW,
                           torch.tensor(d, device=dev), torch.tensor(lev, device=dev), tg, wl, 2, precision)
        (img ** 2).sum().backward()
        grads.append((tW.grad.cpu().numpy(), tg.grad.cpu().numpy()))
    np.testing.assert_array_equal(grads[0][0], grads[1][0])
    np.testing.assert_array_equal(grads[0][1], grads[1][1])
