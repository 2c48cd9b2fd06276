"""The batched form at the batched workload's own shapes: channels spread over
wl 1.5-3 m, steps whose station counts (48..512, after random flagging of the
512-station layout) and kept eigenpair counts (8..64) differ from step to step,
and 512^2 pixels, collected in one call from device memory (the synthesis one
persistent launch) and then again through the captured CUDA graph's replay.

The problems are fixed so that the extremes are present: 512 stations (the
largest K = 2 n_st of the tensor-core GEMM, 16 chunks of 32 stations), 48
stations, counts that are not multiples of 32 (a ragged last chunk), 64 kept
pairs (the widest accumulator) and 8. Each channel's level images are checked
against the FP64 oracle (Gram, Jacobi eigensolve, direct per-pixel sum; Sec.
2.3, Eq. standard_synthesis, Algorithm 1) on a few hundred sampled pixels that
include the first, the edges of 128-pixel tiles and the whole last tile.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2310_09200_b300 import bipp_ss, inputs
from tests import helpers

pytestmark = pytest.mark.gpu

# per channel, per step: (n_st, n_eig)
SIZES = [
    [(512, 64), (77, 8), (200, 30)],
    [(48, 8), (333, 64), (129, 17)],
    [(480, 50), (96, 12), (255, 64)],
    [(512, 33), (61, 61), (160, 24)],
]
TOL = {"split_fp16": 1e-5, "split_bf16": 1e-3}  # relative L2 per level image (FP32 and split-BF16 bounds)


def _rel(a, b):
    return np.array([np.linalg.norm(a[:, l] - b[:, l]) / max(np.linalg.norm(b[:, l]), 1e-300)
                     for l in range(b.shape[1])])


@pytest.fixture(scope="module")
def batch():
    cfg = inputs.make_batch_config(n_chan=len(SIZES), n_t=len(SIZES[0]), n_side=512, sizes=SIZES)
    pix = cfg["pix"]
    n_pix, L = pix.shape[0], cfg["n_level"]
    rng = np.random.default_rng(33)
    tile_edges = [0, 1, 127, 128, 129, 255, 256, 4095, 4096, n_pix // 2 - 1, n_pix // 2]
    last_tile = list(range(n_pix - 128, n_pix))
    sample = np.unique(np.concatenate([rng.choice(n_pix, 300, replace=False), tile_edges, last_tile]))
    bounds, want = [], []
    for ch in cfg["channels"]:
        eig = []
        for p, V in zip(ch["st_xyz"], ch["vis"]):
            mu, A, _ = oracle.geneig(V, oracle.gram(p, ch["wl"]))
            eig.append((mu, A))
        pooled = np.concatenate([mu[:k] for (mu, _), k in zip(eig, ch["n_eig"])])
        b = helpers.quantile_bounds(pooled, L)
        assert helpers.min_edge_margin(pooled, b) > 1e-9
        img = None
        for (mu, A), p, k in zip(eig, ch["st_xyz"], ch["n_eig"]):  # LSQ filter: d = mu
            lev = oracle.select_levels(mu[:k], b)
            img = oracle.synth_levels(pix[sample], p, ch["wl"], A[:, :k], mu[:k], lev, L, img=img)
        bounds.append(b)
        want.append(img)
    st = [p for ch in cfg["channels"] for p in ch["st_xyz"]]
    vis = [V for ch in cfg["channels"] for V in ch["vis"]]
    ne = [k for ch in cfg["channels"] for k in ch["n_eig"]]
    chan = [c for c, ch in enumerate(cfg["channels"]) for _ in ch["st_xyz"]]
    wl = [ch["wl"] for ch in cfg["channels"]]
    assert min(k for k in ne) == 8 and max(ne) == 64 and max(p.shape[0] for p in st) == 512
    assert any(p.shape[0] % 32 for p in st)
    return pix, sample, wl, np.stack(bounds), st, vis, ne, chan, want


@pytest.mark.parametrize("precision", ["split_fp16", "split_bf16"])
def test_batched_shapes_match_oracle_direct_and_replayed(batch, precision):
    import torch
    pix, sample, wl, bounds, st, vis, ne, chan, want = batch
    nst, N, stp, Vp = bipp_ss.pack_batch(st, vis)
    d_st, d_V = torch.from_numpy(stp).cuda(), torch.from_numpy(Vp).cuda()
    h = bipp_ss.bipp_ss_create_channels(pix, wl, bounds, precision=precision, eig_mode="mixed")
    try:
        L = bounds.shape[1]
        # 1: direct (the autotuner times the tensor-core kernel on this geometry)
        bipp_ss.bipp_ss_collect_channels_device(h, chan, nst, d_st, d_V, n_eig=ne)
        first = bipp_ss.bipp_ss_get_f64(h, pix.shape[0], L, len(wl))
        nt, nk, mu, lev = bipp_ss.bipp_ss_last_eigvals(h, len(ne), 64)
        assert nt == len(ne) and list(nk) == list(ne)
        # 2: captured into a CUDA graph, 3: the graph replayed
        for _ in range(2):
            bipp_ss.bipp_ss_collect_channels_device(h, chan, nst, d_st, d_V, n_eig=ne)
        third = bipp_ss.bipp_ss_get_f64(h, pix.shape[0], L, len(wl))
    finally:
        bipp_ss.bipp_ss_destroy(h)
    for c in range(len(wl)):
        err1 = _rel(first[c][sample], want[c])
        assert np.all(err1 <= TOL[precision]), (precision, "direct", c, err1)
        err23 = _rel((third[c] - first[c])[sample] / 2.0, want[c])
        assert np.all(err23 <= TOL[precision]), (precision, "captured + replayed", c, err23)
        assert np.all(np.isfinite(first[c]))
