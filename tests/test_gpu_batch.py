"""Batched multi-channel collection: many channels (own wavelength, level
bounds and images) x steps with ragged station counts and ragged n_eig in
one launch sequence, compared per channel with the FP64 oracle; repeated
geometry is captured into a CUDA graph and replayed."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2310_09200_b300 import bipp_ss, inputs
from tests import helpers

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-9, "fp32": 1e-5, "split_bf16": 1e-3, "split_fp16": 1e-5}


def _rel(a, b):
    return np.array([np.linalg.norm(a[:, l] - b[:, l]) / max(np.linalg.norm(b[:, l]), 1e-300)
                     for l in range(b.shape[1])])


@pytest.fixture(scope="module")
def small_batch():
    cfg = inputs.make_batch_config(n_chan=3, n_t=3, n_side=24, n_st_lo=20, n_st_hi=70, n_eig_lo=4, n_eig_hi=20)
    pix = cfg["pix"]
    n_level = cfg["n_level"]
    chans, bounds, want = [], [], []
    for c, ch in enumerate(cfg["channels"]):
        pooled = []
        for p, V, k in zip(ch["st_xyz"], ch["vis"], ch["n_eig"]):
            mu, _, _ = oracle.geneig(V, oracle.gram(p, ch["wl"]))
            pooled.extend(mu[:k])
        b = helpers.quantile_bounds(pooled, n_level)
        assert helpers.min_edge_margin(pooled, b) > 1e-9
        img = None
        for p, V, k in zip(ch["st_xyz"], ch["vis"], ch["n_eig"]):
            img, *_ = oracle.ss_step(pix, ch["wl"], b, k, p, V, img=img)
        bounds.append(b)
        want.append(img)
    st = [p for ch in cfg["channels"] for p in ch["st_xyz"]]
    vis = [V for ch in cfg["channels"] for V in ch["vis"]]
    ne = [k for ch in cfg["channels"] for k in ch["n_eig"]]
    chan = [c for c, ch in enumerate(cfg["channels"]) for _ in ch["st_xyz"]]
    wl = [ch["wl"] for ch in cfg["channels"]]
    return pix, wl, np.stack(bounds), st, vis, ne, chan, want


@pytest.mark.parametrize("precision", ["fp64", "fp32", "split_bf16", "split_fp16"])
def test_multichannel_batch_matches_oracle(small_batch, precision):
    pix, wl, bounds, st, vis, ne, chan, want = small_batch
    h = bipp_ss.bipp_ss_create_channels(pix, wl, bounds, precision=precision)
    try:
        bipp_ss.bipp_ss_collect_channels(h, chan, st, vis, n_eig=ne)
        got = bipp_ss.bipp_ss_get_f64(h, pix.shape[0], bounds.shape[1], len(wl))
    finally:
        bipp_ss.bipp_ss_destroy(h)
    for c in range(len(wl)):
        err = _rel(got[c], want[c])
        assert np.all(err <= TOL[precision]), (precision, c, err)


@pytest.mark.parametrize("precision", ["fp32", "split_fp16"])
def test_graph_replay_accumulates_like_separate_batches(small_batch, precision):
    """Batch 1 runs directly (and autotunes the split kernel), batch 2 of the
    same geometry is captured into a graph, batch 3 replays it: the images are
    three times those of one batch."""
    import torch
    pix, wl, bounds, st, vis, ne, chan, want = small_batch
    nst, N, stp, Vp = bipp_ss.pack_batch(st, vis)
    d_st, d_V = torch.from_numpy(stp).cuda(), torch.from_numpy(Vp).cuda()
    h = bipp_ss.bipp_ss_create_channels(pix, wl, bounds, precision=precision)
    try:
        for _ in range(3):
            bipp_ss.bipp_ss_collect_channels_device(h, chan, nst, d_st, d_V, n_eig=ne)
            t = bipp_ss.bipp_ss_get_timings(h)
            assert np.isfinite(t["synth_ms"]) and t["synth_ms"] > 0 and np.isfinite(t["eig_ms"])
        got = bipp_ss.bipp_ss_get_f64(h, pix.shape[0], bounds.shape[1], len(wl))
    finally:
        bipp_ss.bipp_ss_destroy(h)
    for c in range(len(wl)):
        err = _rel(got[c] / 3.0, want[c])
        assert np.all(err <= TOL[precision]), (precision, c, err)


def test_channel_order_is_validated(small_batch):
    pix, wl, bounds, st, vis, ne, chan, want = small_batch
    h = bipp_ss.bipp_ss_create_channels(pix, wl, bounds, precision="fp32")
    try:
        bad = list(reversed(chan))
        with pytest.raises(bipp_ss.BippError) as e:
            bipp_ss.bipp_ss_collect_channels(h, bad, st, vis, n_eig=ne)
        assert e.value.code == bipp_ss.BIPP_ERR_INVALID_ARG
        with pytest.raises(bipp_ss.BippError) as e:
            bipp_ss.bipp_ss_collect_channels(h, [0] * (len(chan) - 1) + [7], st, vis, n_eig=ne)
        assert e.value.code == bipp_ss.BIPP_ERR_INVALID_ARG
    finally:
        bipp_ss.bipp_ss_destroy(h)
