"""Differentiable level images: torch.autograd glue over the C ABI.

``synth_levels(pix, st_xyz, W, d, level, gains, wl, n_level, precision)``
returns the level images I (n_pix, n_level) of the gain-corrected standard
synthesis

    z_te(r) = sum_i conj(g_i exp(j 2 pi <r, p_ti>/wl)) W[t, i, e],
    I_l(r)  = sum_t sum_{e: level[t, e] = l} d[t, e] |z_te(r)|^2,

and is differentiable with respect to the complex eigenvectors W and the
complex station gains g. Forward and backward both run in libbipp_ss.so
(the backward is the hand-written adjoint, which recomputes the phase matrix
instead of storing it): with precision "split_fp16" / "split_bf16" on the
tcgen05 tensor cores, with "fp32" on the CUDA cores. This module only
arranges tensors into the ABI's column-major layout and calls it on the
current CUDA stream.

Shapes: pix (n_pix, 3) f64; st_xyz (T, n_st, 3) f64; W (T, n_st, n_eig)
c128; d (T, n_eig) f64; level (T, n_eig) int; gains (n_st,) c128.
"""
from __future__ import annotations

import torch

from . import bipp_ss


def _abi_layout(pix, st_xyz, W, d, level, gains):
    pix_cm = pix.to(torch.float64).t().contiguous()                 # (3, n_pix)
    st_cm = st_xyz.to(torch.float64).transpose(1, 2).contiguous()   # (T, 3, n_st)
    W_cm = W.to(torch.complex128).transpose(1, 2).contiguous()      # (T, n_eig, n_st)
    d_c = d.to(torch.float64).contiguous()
    lev_c = level.to(torch.int32).contiguous()
    g_c = gains.to(torch.complex128).contiguous()
    return pix_cm, st_cm, W_cm, d_c, lev_c, g_c


class SynthLevels(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pix, st_xyz, W, d, level, gains, wl, n_level, precision):
        for t in (pix, st_xyz, W, d, level, gains):
            if not t.is_cuda:
                raise ValueError("synth_levels runs on CUDA tensors only")
        pix_cm, st_cm, W_cm, d_c, lev_c, g_c = _abi_layout(pix, st_xyz, W, d, level, gains)
        img = torch.empty((n_level, pix.shape[0]), dtype=torch.float64, device=pix.device)
        bipp_ss.bipp_ss_synth_levels_device(pix_cm, wl, st_cm, W_cm, d_c, lev_c, g_c, img, precision=precision,
                                            stream=torch.cuda.current_stream(pix.device))
        ctx.save_for_backward(pix_cm, st_cm, W_cm, d_c, lev_c, g_c)
        ctx.wl = wl
        ctx.precision = precision
        ctx.w_dtype = W.dtype
        ctx.g_dtype = gains.dtype
        return img.t()

    @staticmethod
    def backward(ctx, grad_img):
        pix_cm, st_cm, W_cm, d_c, lev_c, g_c = ctx.saved_tensors
        gI = grad_img.to(torch.float64).t().contiguous()  # (n_level, n_pix)
        gW_cm = torch.empty_like(W_cm)
        gg = torch.empty_like(g_c)
        bipp_ss.bipp_ss_synth_adjoint_device(pix_cm, ctx.wl, st_cm, W_cm, d_c, lev_c, g_c, gI, gW_cm, gg,
                                             precision=ctx.precision, stream=torch.cuda.current_stream(gI.device))
        gW = gW_cm.transpose(1, 2).to(ctx.w_dtype) if ctx.needs_input_grad[2] else None
        gG = gg.to(ctx.g_dtype) if ctx.needs_input_grad[5] else None
        return None, None, gW, None, None, gG, None, None, None


def synth_levels(pix, st_xyz, W, d, level, gains, wl: float, n_level: int, precision: str = "fp32"):
    """Level images (n_pix, n_level), differentiable in W and gains.
    precision: "fp32" (CUDA cores), "split_fp16" or "split_bf16" (tensor
    cores; the adjoint needs n_eig <= 64 and n_level <= 4)."""
    return SynthLevels.apply(pix, st_xyz, W, d, level, gains, float(wl), int(n_level), precision)
