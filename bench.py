#!/usr/bin/env python
"""Benchmark of the standard-synthesis hot path on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--synthesis standard|nufft]

One bench step = one whole imaging job of the SKA-Low-like workload: 100 time
steps of (Gram matrix, generalised eigensolve, selection + levels, synthesis
of 1024^2 pixels from 512 stations with 64 eigenvectors in 4 levels). The
metric is synthesized pixel x eigvec x station products per second over the
whole path. Inputs (positions, 400 MB of visibilities) are resident in HBM
for `value` and are larger than L2, so every step streams them from DRAM;
`e2e` repeats the measurement through the host-buffer C ABI with the
host->device copies and the image read-back inside the timed region.

`--synthesis nufft` measures NUFFT synthesis (Sec. 3.4) on its own workload,
the one of the paper's NUFFT comparison: 512 stations, 50 steps over 6 hours,
1024^2 pixels of 4 arcsec, N_eig 64, 4 levels, tolerance 1e-5; the metric
counts the same products (the images are the same up to the tolerance).

`--impl reference` times the FP64 CPU oracle (the only other place this
script runs it) on a bounded sample of the same workload on the host cores.
Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "synthesized pixel*eigvec*station products/s"
UNIT = "products/s"

# Nominal FP64 and FP32 pipes of a B300 (148 SMs x 2 DFMA / 128 FFMA per clock x 2
# flop x 2.032 GHz): defaults only; the reported rooflines use the rates measured in
# the run by bipp_ss_measure_fma_rates.
SMS = 148
SM_MAX_GHZ = 2.032
FP64_PEAK_FLOPS = SMS * 2 * 2 * SM_MAX_GHZ * 1e9
FP32_PEAK_FLOPS = SMS * 128 * 2 * SM_MAX_GHZ * 1e9
# Issue slots: 4 warp instructions per SM per clock. k_synth_tc issues 30 thread
# instructions per pixel-station pair (ncu, profiles/k_synth_tc_ska_low_512st_1024px_10steps.md:
# phase, sincos, hi/lo split and stores of A in the producers, plus the epilogue).
ISSUE_THREAD_INSTR_PER_S = SMS * 4 * 32 * SM_MAX_GHZ * 1e9
SYNTH_TC_INSTR_PER_PAIR = 30


DTYPES = {"fp64": "f64", "fp32": "f64 eig + f32 synth",
          "split_bf16": "f64 eig + bf16x3 tensor synth (f32 acc)", "split_fp16": "f64 eig + f16x3 tensor synth (f32 acc)"}


EIG_DESC = {"jacobi64": "fp64 parallel-order Jacobi (off(C) <= 1e-13 ||C||_F)",
            "mixed": ("fp32 Householder tridiagonalisation, the n_eig+16 leading pairs of the tridiagonal form "
                      "(multisection, inverse iteration) back-transformed, then double-float Rayleigh-Ritz "
                      "refinement of those pairs (residual <= 1e-10 ||C||_F)")}


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one k_synth_tc launch of the
# default workload, from a single-pass ncu capture; reported only while the kernel sources
# hash to the captured ones and the workload is the captured one, else null.
SYNTH_TC_TRAFFIC = {
    "sha256": {"synth_tc.cu": "1c206790c91a6c6a14bcf205048ff7888efbef6a275d140962bce8f9e05822b1",
               "synth_tc.cuh": "3a72b4c84ea26409ffed4f45e9c21d3cca0fb257edb7d0006542fe4c601ec351"},
    "workload": {"n_st": 512, "n_pix": 1048576, "n_eig": 64, "n_level": 4, "n_t": 100, "precision": "split_fp16"},
    "bytes": 134725632 + 30382080,
}


def synth_tc_traffic(workload: dict):
    import hashlib
    csrc = os.path.join(ROOT, "paper_2310_09200_b300", "csrc")
    for name, digest in SYNTH_TC_TRAFFIC["sha256"].items():
        try:
            with open(os.path.join(csrc, name), "rb") as f:
                if hashlib.sha256(f.read()).hexdigest() != digest:
                    return None
        except OSError:
            return None
    return SYNTH_TC_TRAFFIC["bytes"] if workload == SYNTH_TC_TRAFFIC["workload"] else None


def tc_roofline(syn_flops: float, syn_ms: float, pairs: float, peaks: dict, traffic, sfu_rate: float) -> dict:
    """Roofline of the split tensor-core synthesis: 3 tensor products per real
    multiply-add, T_roof = max(T_tensor, T_sfu) for `frac` (sfu_rate: sincos
    pairs/s measured by bipp_ss_measure_sincos_rate in the same run); beside it
    the issue-slot time of the kernel's measured instruction count per pair and
    the name of the largest of the three."""
    r_tc = peaks.get("bf16_tflops_sustained", 1411.3) * 1e12
    t_tc = 3 * syn_flops / r_tc
    t_sfu = pairs / sfu_rate
    t_issue = SYNTH_TC_INSTR_PER_PAIR * pairs / ISSUE_THREAD_INSTR_PER_S
    t = {"tensor_split": t_tc * 1e3, "sfu_sincos": t_sfu * 1e3, "issue_slots": t_issue * 1e3}
    return {"kernel": "k_synth_tc", "bound": "tensor", "achieved": 3 * syn_flops / (syn_ms / 1e3) / 1e12,
            "peak": r_tc / 1e12, "unit": "TFLOP/s", "traffic": traffic,
            "frac": max(t_tc, t_sfu) / (syn_ms / 1e3),
            "frac_algorithmic_s1": (syn_flops / r_tc) / (syn_ms / 1e3),
            "frac_issue": t_issue / (syn_ms / 1e3),
            "t_roof_ms": t, "largest_bound": max(t, key=t.get),
            "peak_note": ("of measured: cuBLAS bf16 sustained (FP16 dense rate is the same nominal); "
                          "frac = max(T_tensor(s=3), T_sfu) / measured time; "
                          f"SFU rate {sfu_rate:.3g} sincos pairs/s measured in this run by "
                          "bipp_ss_measure_sincos_rate (__sincosf chains on every SM); issue_slots = "
                          f"{SYNTH_TC_INSTR_PER_PAIR} thread instructions per pair (ncu) at 4 warp "
                          "instructions per SM per clock, 148 SMs, 2.032 GHz")}


def eig_roofline(n: int, kp: int, n_t: int, eig_ms: float, fp32_rate: float, passes: int = 2) -> dict:
    """Roofline of the mixed eigensolve stage on the CUDA cores: the FP32
    Householder reduction (16/3 n^3 flops per step) and the three applications
    of the reflectors to kp columns (4 n^2 kp flops each) at the measured FP32
    FMA rate, plus `passes` refinement passes of double-float products at half
    that rate in operations (12 FP32 operations per real multiply-add, issued as
    6 packed FP32x2 instructions): per
    pass C X1 = L^{-1} (V (L^{-T} X1)) (6 n^2 kp real multiply-adds) and the
    five n x kp x kp products (20 n kp^2). frac = bound / measured stage time
    (the Sturm counts, solves and small Jacobi are latency chains, not in it)."""
    fp32_flops = (16.0 / 3.0 * n ** 3 + 3 * 4.0 * n ** 2 * kp) * n_t
    df_instr = passes * 12.0 * (6.0 * n ** 2 * kp + 20.0 * n * kp ** 2) * n_t
    t32, tdf = fp32_flops / fp32_rate, df_instr / (fp32_rate / 2)
    return {"kernel": "mixed eigensolve stage (FP32 tridiagonal form, kp leading pairs, double-float refinement)",
            "bound": "alu", "achieved": None, "peak": fp32_rate / 1e12, "unit": "TFLOP/s", "traffic": None,
            "frac": (t32 + tdf) / (eig_ms / 1e3),
            "t_roof_ms": {"fp32_stage": t32 * 1e3, "df_refinement": tdf * 1e3},
            "peak_note": ("of measured: FP32 FMA rate of this GPU (bipp_ss_measure_fma_rates, this run); "
                          "frac = (FP32 flops / rate + double-float instructions / instruction rate) / stage time")}


def synth_shape_of(get):
    """The tensor-core synthesis launch shape of the last collect (the autotuner's
    pick: ring stages, fused MMA, epilogue warps), or None if it cannot be read."""
    try:
        return get()
    except Exception:
        return None


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {"bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0, "hbm_gbs": 6400.0}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--mode", default="synthesis", choices=["synthesis", "grad"],
                    help="grad: forward + backward of the differentiable level images (configuration 4)")
    ap.add_argument("--precision", default="split_fp16", choices=["fp64", "fp32", "split_bf16", "split_fp16"])
    ap.add_argument("--n-t", type=int, default=0, help="time steps per imaging job (default 100; 50 for nufft)")
    ap.add_argument("--synthesis", default="standard", choices=["standard", "nufft"])
    ap.add_argument("--n-chan", type=int, default=64, help="channels of the batched workload")
    ap.add_argument("--workload", default="", choices=["", "ska_low_20deg", "nufft_4arcsec", "batch"],
                    help="inputs (default: the 20 deg SKA-Low job for standard synthesis, the 4 arcsec field "
                         "of the paper's NUFFT comparison for nufft)")
    ap.add_argument("--nufft-eps", type=float, default=1e-5)
    ap.add_argument("--nufft-partition", type=int, nargs=6, default=[1, 1, 1, 1, 1, 1],
                    help="NUFFT domain partitioning: input cells (x y z) then image cells (x y z)")
    ap.add_argument("--side", type=int, default=1024, help="image side in pixels")
    ap.add_argument("--n-st", type=int, default=0, help="keep only the first n stations (small profiling cases)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the side-by-side precision forms (FP32, split BF16, split FP16) after the timed region")
    ap.add_argument("--eig", default="mixed", choices=["jacobi64", "mixed"],
                    help="eigensolver: FP64 Jacobi, or FP32 Jacobi + FP64 refinement of the kept pairs")
    return ap.parse_args()


def workload_name(args):
    return args.workload or ("nufft_4arcsec" if args.synthesis == "nufft" else "ska_low_20deg")


def workload(args):
    from paper_2310_09200_b300 import inputs
    if workload_name(args) == "nufft_4arcsec":
        return inputs.make_nufft_config(n_t=args.n_t or 50, n_side=args.side, n_st=args.n_st or 512)
    inp = inputs.make_config(1, n_t=args.n_t or 100, n_side=args.side)
    if args.n_st:
        n = args.n_st
        inp.st_xyz = [p[:n] for p in inp.st_xyz]
        inp.vis = [V[:n, :n] for V in inp.vis]
    return inp


def config_dict(args, inp, precision):
    if workload_name(args) == "nufft_4arcsec":
        how = (f"NUFFT synthesis, type-3 NUFFT tolerance {args.nufft_eps:g}" if args.synthesis == "nufft"
               else f"standard synthesis ({precision})")
        return {
            "workload": (f"SKA-Low-like field of 4 arcsec pixels, {how}: {inp.st_xyz[0].shape[0]} stations "
                         f"(lognormal to 65 km), {args.side}^2 px, N_eig {inp.n_eig}, {inp.n_level} levels, "
                         f"{inp.n_t} time steps over 6 h per job, wl 2 m"),
            "n_st": int(inp.st_xyz[0].shape[0]), "n_pix": int(inp.n_pix), "n_eig": int(inp.n_eig),
            "n_level": int(inp.n_level), "n_t": int(inp.n_t),
            "synthesis": "nufft" if args.synthesis == "nufft" else precision,
            **({"nufft_eps": args.nufft_eps, "nufft_partition": list(args.nufft_partition)}
               if args.synthesis == "nufft" else {}),
            "eigensolve": EIG_DESC.get(getattr(args, "eig", "jacobi64"), "fp64 parallel-order Jacobi")
            if precision != "fp64 (oracle)" else "fp64 cyclic Jacobi (oracle)",
            "l2": "inputs larger than L2 (visibilities 200 MB per job)",
        }
    return {
        "workload": (f"SKA-Low-like standard synthesis: {inp.st_xyz[0].shape[0]} stations (lognormal to 65 km), "
                     f"{args.side}^2 px in a 20 deg cap, N_eig {inp.n_eig}, {inp.n_level} levels, "
                     f"{inp.n_t} time steps per job, wl 2 m"),
        "n_st": int(inp.st_xyz[0].shape[0]), "n_pix": int(inp.n_pix), "n_eig": int(inp.n_eig),
        "n_level": int(inp.n_level), "n_t": int(inp.n_t), "synthesis": precision,
        "eigensolve": EIG_DESC.get(getattr(args, "eig", "jacobi64"), "fp64 parallel-order Jacobi")
        if precision != "fp64 (oracle)" else "fp64 cyclic Jacobi (oracle)",
        "l2": "inputs larger than L2 (visibilities 400 MB per job)",
    }


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 7:
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dtype_label(args):
    if args.synthesis == "nufft":
        base = "f64 eig + f32 NUFFT grids (f64 coordinates and phase reduction)"
    else:
        base = DTYPES[args.precision]
    return base.replace("f64 eig", "f32+f64 eig") if args.eig == "mixed" else base


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def strided_subset(n_pix: int, n_sub_side: int = 64) -> np.ndarray:
    """Indices of a strided n_sub_side^2 subset of a square image (l fastest)."""
    side = int(round(math.sqrt(n_pix)))
    stride = max(1, side // n_sub_side)
    return (np.arange(0, side, stride)[:, None] * side + np.arange(0, side, stride)[None, :]).ravel()


def cpu_sample(inp, bounds, t: int = 0, n_sub_side: int = 64, eig: bool = True):
    """The oracle on a bounded sample of the job: Gram + eigensolve of time
    step t (single thread, as the oracle stands) and the synthesis of a
    strided n_sub_side^2 pixel subset with that step's kept eigenpairs (OpenMP
    over pixels). Returns the measured times, the products of exactly that
    synthesis and their rate over the whole sample, the subset's image, and,
    separately, the linear extrapolation of the step to all pixels and of the
    job to all steps. eig=False skips the eigensolve (random G-free
    eigenvectors of the same shape: a warm-up of the synthesis only)."""
    import oracle
    sel = strided_subset(inp.n_pix, n_sub_side)
    pix = inp.pix[sel]
    p, V = inp.st_xyz[t], inp.vis[t]
    t0 = time.perf_counter()
    if eig:
        G = oracle.gram(p, inp.wl)
        mu, A, _ = oracle.geneig(V, G)
    else:
        rng = np.random.default_rng(t)
        mu = np.sort(rng.normal(size=p.shape[0]))[::-1]
        A = rng.normal(size=(p.shape[0], p.shape[0])) + 0j
    t1 = time.perf_counter()
    d = mu[: inp.n_eig]
    lev = oracle.select_levels(d, bounds)
    img = oracle.synth_levels(pix, p, inp.wl, A[:, : inp.n_eig], d, lev, bounds.shape[0])
    t2 = time.perf_counter()
    t_eig, t_syn = t1 - t0, t2 - t1
    prods = float(len(sel)) * inp.n_eig * p.shape[0]
    return {"t_eig_s": t_eig, "t_synth_sub_s": t_syn, "wall_s": t2 - t0, "n_sub": int(len(sel)), "sel": sel,
            "img": img, "products": prods, "value": prods / (t2 - t0),
            "extrapolated_job_ms": inp.n_t * (t_eig + t_syn * inp.n_pix / len(sel)) * 1e3}


def cpu_sample_nufft(inp, bounds, eps, patch=128, t=0):
    """Oracle NUFFT synthesis on a bounded sample: time step t (FP64 Gram +
    Jacobi eigensolve, then the type-3 NUFFT of its level visibilities) onto
    the central patch^2 pixels of the image; measured time and products."""
    from oracle import nufft as onu
    side = int(round(math.sqrt(inp.n_pix)))
    c0 = side // 2 - patch // 2
    rows = np.arange(c0, c0 + patch)
    sel = (rows[:, None] * side + rows[None, :]).ravel()
    t0 = time.perf_counter()
    onu.nufft_levels(inp.pix[sel], inp.wl, bounds, inp.n_eig, inp.st_xyz[t], inp.vis[t], eps=eps)
    dt = time.perf_counter() - t0
    n_st = inp.st_xyz[t].shape[0]
    prods = float(len(sel)) * inp.n_eig * n_st
    return {"t_s": dt, "n_sub": int(len(sel)), "products": prods, "value": prods / dt}


def nufft_roofline(nt, n_level, n_pix, n_t, n_st, n_eig, hbm_gbs, fp32_rate=FP32_PEAK_FLOPS):
    """The dominant kernel of NUFFT synthesis (largest total time per job) and its
    HBM roofline: algorithmic bytes per launch / measured launch time."""
    M = nt["grid"]
    cells = M[0] * M[1] * M[2]
    cells2 = 8 * cells
    Lp = 1 if n_level == 1 else n_level + (n_level & 1)
    pts = nt["points"]
    kern = {  # name: (launches per job, ms per launch, algorithmic bytes per launch)
        "sort + strengths (k_nu_count, scans, k_nu_scatter)":
            (1, nt["sort_ms"], n_t * n_eig * n_st * 16 + n_t * n_st * 24 + pts * (32 + 8 * Lp) + cells * 12),
        "k_nu_spread": (1, nt["spread_ms"], pts * (32 + 8 * Lp) + cells * Lp * 8),
        "k_nu_pad": (n_level, nt["pad_ms"], cells * 8 + cells2 * 8),
        "cuFFT C2C (library)": (n_level, nt["fft_ms"], 2 * cells2 * 8),
        "k_nu_interp": (n_level, nt["interp_ms"], n_pix * (24 + 16 + 4)),
    }
    def roof(k):
        nl, ms, by = kern[k]
        if k == "k_nu_spread":  # arithmetic: w^3 cells x levels x (weight x complex strength, accumulated)
            flops = pts * nt["w"] ** 3 * n_level * 4.0
            ach = flops / (ms / 1e3) / 1e12
            return {"kernel": k, "bound": "alu", "achieved": ach, "peak": fp32_rate / 1e12, "unit": "TFLOP/s",
                    "frac": ach / (fp32_rate / 1e12)}
        ach = by / (ms / 1e3) / 1e9
        return {"kernel": k, "bound": "hbm", "achieved": ach, "peak": hbm_gbs, "unit": "GB/s", "frac": ach / hbm_gbs}

    name = max(kern, key=lambda k: kern[k][0] * kern[k][1])
    own = max((k for k in kern if "library" not in k), key=lambda k: kern[k][0] * kern[k][1])
    return {**roof(name), "traffic": None,
            "own_dominant": {**roof(own), "note": "largest of this library's kernels (the FFT is cuFFT)"},
            "kernels_ms_per_job": {k: v[0] * v[1] for k, v in kern.items()},
            "grid": list(M), "fine_grid_points": cells2,
            "peak_note": ("hbm: of measured STREAM-style copy; algorithmic bytes = eigenvectors and stations read, "
                          "sorted records and cell counts written (sort), one level read + fine grid written (pad), "
                          "fine grid read + written once (FFT), pixel coordinates + correction + image read/write "
                          "(interp); alu (spread): 4 flops per footprint cell and level of each baseline against "
                          "the FP32 FMA rate measured in this run")}


def main():
    args = parse()
    ws, rank, local = dist_setup(args)
    if args.impl == "reference":
        if args.mode == "grad" or args.workload == "batch":
            raise SystemExit("--impl reference times the oracle on the synthesis workloads only "
                             "(not --mode grad or --workload batch)")
        return reference_main(args, ws, rank)
    if args.mode == "grad":
        return grad_main(args, ws, rank, local)
    if args.workload == "batch":
        return batch_main(args, ws, rank, local)
    return ours_main(args, ws, rank, local)


def batch_main(args, ws, rank, local):
    """Batched form (configuration 3): n_chan channels (wl 1.5 to 3 m) x 20 steps,
    each step a random flagging of the 512-station layout (48 to 512 stations)
    with 8 to 64 eigenpairs, 512^2 px; the whole batch is one collect (the
    synthesis one persistent launch, the batch a replayed CUDA graph), level
    bounds per channel from the library's own pre-pass."""
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps({"impl": "reference", "unavailable": "the batched workload has no CPU reference arm; "
                              "its parity is checked in tests/test_gpu_batch.py"}), flush=True)
        return 0
    import torch

    from paper_2310_09200_b300 import bipp_ss, build, inputs
    from paper_2310_09200_b300.distributed import max_over_ranks
    build.build()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    cfg = inputs.make_batch_config(n_chan=args.n_chan, n_t=args.n_t or 20, n_side=args.side if args.side != 1024 else 512)
    pix, chans, L = cfg["pix"], cfg["channels"], cfg["n_level"]
    wls = np.array([c["wl"] for c in chans])
    bounds = np.stack([bipp_ss.estimate_level_bounds(c["st_xyz"][::4], c["vis"][::4], c["wl"], c["n_eig"][::4], L,
                                                     eig_mode=args.eig)[0] for c in chans])
    chan, st, vis, neig = [], [], [], []
    for ci, c in enumerate(chans):
        chan += [ci] * len(c["vis"])
        st += c["st_xyz"]
        vis += c["vis"]
        neig += c["n_eig"]
    nst, N, st_p, V_p = bipp_ss.pack_batch(st, vis)
    dev = f"cuda:{local}"
    d_st = torch.from_numpy(st_p).to(dev)
    d_V = torch.from_numpy(V_p).to(dev)
    stream = torch.cuda.Stream()
    h = bipp_ss.bipp_ss_create_channels(pix, wls, bounds, precision=args.precision, eig_mode=args.eig,
                                        device=local)
    n_pix = pix.shape[0]
    prods = float(sum(float(n_pix) * int(k) * int(n) for k, n in zip(neig, nst)))

    def one_step():
        bipp_ss.bipp_ss_collect_channels_device(h, chan, nst, d_st, d_V, n_eig=neig, stream=stream)
        return bipp_ss.bipp_ss_get_timings(h)

    for _ in range(args.warmup):
        one_step()
    sfu_rate = bipp_ss.bipp_ss_measure_sincos_rate(local, 5)  # the SFU bound's rate, on this GPU now
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = Clocks(local)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    stage = np.zeros(4)
    launches = 0
    e0.record(stream)
    for _ in range(args.steps):
        t = one_step()
        stage += [t["gram_reduce_ms"], t["eig_ms"], t["select_ms"], t["synth_ms"]]
        launches += t["launches"]
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms_total = e0.elapsed_time(e1)
    if dist:
        dist.barrier()
        ms_total = max_over_ranks(ms_total, device=dev)
    K = args.steps
    ms_step = ms_total / K
    syn_ms = stage[3] / K
    e2e = None
    if not args.no_e2e:
        st_h = torch.from_numpy(st_p).pin_memory()
        V_h = torch.from_numpy(V_p).pin_memory()
        img_t = torch.zeros((len(chans), L, n_pix), dtype=torch.float64).pin_memory()
        lib = bipp_ss.load()
        img_ptr = img_t.numpy().ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        ch = np.ascontiguousarray(chan, dtype=np.int32)
        ne = np.ascontiguousarray(neig, dtype=np.int32)
        nsv = np.ascontiguousarray(nst, dtype=np.int32)

        def host_step():
            rc = lib.bipp_ss_collect_channels(h, len(nsv), N, bipp_ss._ip(ch), bipp_ss._ip(nsv), bipp_ss._ip(ne),
                                              ctypes.c_void_p(st_h.data_ptr()), ctypes.c_void_p(V_h.data_ptr()),
                                              0, None)
            if rc != 0 or lib.bipp_ss_get_f64(h, img_ptr) != 0:
                raise RuntimeError(bipp_ss.bipp_ss_last_error(h))

        host_step()
        t0 = time.perf_counter()
        for _ in range(K):
            host_step()
        dt = (time.perf_counter() - t0) / K
        if dist:
            dt = max_over_ranks(dt, device=dev)
        e2e = {"value": prods * ws / dt, "unit": UNIT, "h2d_bytes_per_step": int(st_p.nbytes + V_p.nbytes),
               "d2h_bytes_per_step": int(img_t.numpy().nbytes)}
    synth_shape = synth_shape_of(lambda: bipp_ss.bipp_ss_get_synth_shape(h))
    bipp_ss.bipp_ss_destroy(h)
    if rank == 0:
        peaks = measured_peaks()
        r_tc = peaks.get("bf16_tflops_sustained", 1411.3) * 1e12
        pairs = float(sum(float(n_pix) * int(n) for n in nst))
        t_tc, t_sfu = 3 * 8.0 * prods / r_tc, pairs / sfu_rate
        roof = {"kernel": "k_synth_tc", "bound": "tensor", "achieved": 3 * 8.0 * prods / (syn_ms / 1e3) / 1e12,
                "peak": r_tc / 1e12, "unit": "TFLOP/s", "traffic": None, "frac": max(t_tc, t_sfu) / (syn_ms / 1e3),
                "t_roof_ms": {"tensor_split": t_tc * 1e3, "sfu_sincos": t_sfu * 1e3},
                "sfu_sincos_pairs_per_s": sfu_rate,
                "peak_note": ("of measured: cuBLAS bf16 sustained; frac = max(T_tensor(s=3), T_sfu) / measured "
                              "time; SFU rate measured in this run by bipp_ss_measure_sincos_rate")}
        line = {"metric": METRIC, "value": prods * ws / (ms_step / 1e3), "unit": UNIT, "n_gpus": ws,
                "steps": K, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": dtype_label(args), "data": "synthetic",
                "config": {"workload": (f"batched: {len(chans)} channels (wl 1.5-3 m) x {len(vis) // len(chans)} "
                                        f"steps, 48-512 stations and N_eig 8-64 per step, "
                                        f"{int(round(math.sqrt(n_pix)))}^2 px, {L} levels, one collect"),
                           "problems": len(vis), "n_pix": int(n_pix), "synthesis": args.precision,
                           "eigensolve": EIG_DESC.get(args.eig), "l2": "inputs larger than L2"},
                "stage_ms_per_step": {"gram_chol_reduce": stage[0] / K, "jacobi": stage[1] / K,
                                      "select_pack": stage[2] / K, "synthesis": syn_ms},
                "roofline": roof, "cpu_baseline": None, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
                **({"synth_shape": synth_shape} if synth_shape and synth_shape["stages"] else {})}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def grad_main(args, ws, rank, local):
    """Differentiation (configuration 4): loss = ||I_levels - I_target||^2 over 4
    levels of 512^2 pixels from 256 stations, 16 steps, N_eig 32. One bench step
    = the forward and backward of the whole 16-step loss in --precision (split
    FP16 by default: the tensor-core forward and adjoint; "fp32": the CUDA-core
    kernels). Eigenvectors, weights and levels are synthetic of the same
    shapes (their values do not change the work). Beside the timed region the
    plain FP32 path is timed the same way (forward alone, forward + backward),
    the comparison the metric names."""
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps({"impl": "reference", "unavailable": "the grad mode has no CPU reference arm; "
                              "the FP64 oracle gradient is checked in tests/test_gpu_adjoint.py"}), flush=True)
        return 0
    import torch

    from paper_2310_09200_b300 import build, inputs
    from paper_2310_09200_b300.autograd import synth_levels
    from paper_2310_09200_b300.distributed import max_over_ranks
    build.build()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    prec = args.precision if args.precision in ("fp32", "split_fp16", "split_bf16") else "split_fp16"
    inp = inputs.make_config(4)
    T, n_st, K, L = inp.n_t, inp.st_xyz[0].shape[0], inp.n_eig, inp.n_level
    rng = np.random.default_rng(1004)
    st = np.stack(inp.st_xyz)
    W = (rng.normal(size=(T, n_st, K)) + 1j * rng.normal(size=(T, n_st, K))) / np.sqrt(n_st)
    d = np.abs(rng.normal(size=(T, K))) * 50.0 + 1.0
    lev = rng.integers(0, L, size=(T, K)).astype(np.int32)
    g = inputs.gains(n_st, 0.05, rng)
    dev = torch.device(f"cuda:{local}")
    t_pix = torch.tensor(inp.pix, device=dev)
    t_st = torch.tensor(st, device=dev)
    t_d = torch.tensor(d, device=dev)
    t_lev = torch.tensor(lev, device=dev)
    target = torch.tensor(np.abs(rng.normal(size=(inp.n_pix, L))) * 1e3, device=dev)
    tW = torch.tensor(W, device=dev, requires_grad=True)
    tg = torch.tensor(g, device=dev, requires_grad=True)
    stream = torch.cuda.current_stream(dev)

    def step(precision, marks=None, backward=True):
        tW.grad = None
        tg.grad = None
        if marks:
            marks[0].record(stream)
        img = synth_levels(t_pix, t_st, tW, t_d, t_lev, tg, inp.wl, L, precision)
        if marks:
            marks[1].record(stream)
        loss = ((img - target) ** 2).sum()
        if backward:
            loss.backward()
        if marks:
            marks[2].record(stream)
        return loss

    def timed(precision, n, backward=True):
        marks = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(n)]
        for k in range(n):
            step(precision, marks[k], backward)
        torch.cuda.synchronize()
        return (statistics.mean(m[0].elapsed_time(m[1]) for m in marks),
                statistics.mean(m[1].elapsed_time(m[2]) for m in marks))

    for _ in range(args.warmup):
        step(prec)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = Clocks(local)
    marks = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.steps):
        step(prec, marks[k])
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms_total = e0.elapsed_time(e1)
    fwd = statistics.mean(m[0].elapsed_time(m[1]) for m in marks)
    bwd = statistics.mean(m[1].elapsed_time(m[2]) for m in marks)
    if dist:
        dist.barrier()
        ms_total = max_over_ranks(ms_total, device=dev)
    ms_step = ms_total / args.steps
    # the plain FP32 path beside it (outside the timed region)
    for _ in range(2):
        step("fp32")
    f32_fwd, _ = timed("fp32", 3, backward=False)
    f32_fwd_b, f32_bwd = timed("fp32", 3)
    pairs = float(inp.n_pix) * n_st * T
    prods = pairs * K
    if prec == "fp32":
        fp32_rate, _ = bipp_ss_fma(local)
        flops_bwd = pairs * (16.0 * K)  # recomputed z plus the gradient sums, complex
        ach = flops_bwd / (bwd / 1e3) / 1e12
        roof = {"kernel": "k_adjoint", "bound": "alu", "achieved": ach, "peak": fp32_rate / 1e12,
                "unit": "TFLOP/s", "traffic": None, "frac": ach / (fp32_rate / 1e12),
                "peak_note": "16 K flops per pixel-station pair and step (recomputed z and the gradient sums) "
                             "against the FP32 FMA rate measured in this run"}
    else:
        # backward: z recomputed (8 P real flops, x3 split) and grad_W' = 2 sum_r Phi Y as the real GEMM
        # [cos; sin] (2 n_st rows) x [Re Y, Im Y] (2 K columns) over pixels (x3 split); two Phi generations
        sfu = bipp_ss_rate(local)
        peaks = measured_peaks()
        r_tc = peaks.get("bf16_tflops_sustained", 1411.3) * 1e12
        flops = 3 * (8.0 * prods + 2.0 * (2 * n_st) * (2 * K) * inp.n_pix * T)
        t_tc, t_sfu = flops / r_tc, 2 * pairs / sfu
        roof = {"kernel": "adjoint on the tensor cores (k_synth_tc Y stage + k_adjoint_tc)", "bound": "tensor",
                "achieved": flops / (bwd / 1e3) / 1e12, "peak": r_tc / 1e12, "unit": "TFLOP/s", "traffic": None,
                "frac": max(t_tc, t_sfu) / (bwd / 1e3),
                "t_roof_ms": {"tensor_split": t_tc * 1e3, "sfu_sincos": t_sfu * 1e3},
                "peak_note": ("of measured: cuBLAS bf16 sustained; the backward's split tensor flops (z recomputed, "
                              "then Phi^T Y over pixels) and its two sincos passes against the SFU rate measured "
                              "in this run; frac = max(T_tensor, T_sfu) / measured backward time")}
    if rank == 0:
        line = {"metric": "fwd+bwd ms per step of the differentiable level images (vs the plain FP32 forward)",
                "value": ms_step, "unit": "ms", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp32": "f32 (f64 image and gradients)",
                          "split_fp16": "f16x3 tensor forward, bf16x3 tensor adjoint (f32 acc; f64 image, gradients)",
                          "split_bf16": "bf16x3 tensor forward and adjoint (f32 acc; f64 image, gradients)"}[prec],
                "data": "synthetic",
                "config": {"workload": (f"differentiation: {n_st} stations, {int(round(math.sqrt(inp.n_pix)))}^2 px, "
                                        f"{T} time steps, N_eig {K}, {L} levels, gains 1 + N(0, 0.05)"),
                           "n_st": n_st, "n_pix": int(inp.n_pix), "n_t": T, "n_eig": K, "n_level": L,
                           "precision": prec},
                "fwd_ms": fwd, "bwd_ms": bwd,
                "fp32_path": {"fwd_ms": f32_fwd, "fwd_bwd_ms": f32_fwd_b + f32_bwd, "bwd_ms": f32_bwd},
                "fwd_bwd_over_fp32_forward": (fwd + bwd) / f32_fwd,
                "speedup_vs_fp32_fwd_bwd": (f32_fwd_b + f32_bwd) / (fwd + bwd),
                "roofline": roof, "cpu_baseline": None, "e2e": None, "gpu_launches": None, "clocks": clocks}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def bipp_ss_fma(local):
    from paper_2310_09200_b300 import bipp_ss
    return bipp_ss.bipp_ss_measure_fma_rates(local, 5)


def bipp_ss_rate(local):
    from paper_2310_09200_b300 import bipp_ss
    return bipp_ss.bipp_ss_measure_sincos_rate(local, 5)


def reference_main(args, ws, rank):
    """The reference arm: the FP64 CPU oracle, as it stands, on bounded samples
    of the same workload (one time step's Gram + eigensolve and the synthesis
    of a strided pixel subset per bench step). value = the products of the
    timed samples / their measured wall time; ms_per_step = the measured wall
    time of one sample; the linear extrapolation to the whole job is reported
    apart (extrapolated_job_ms), never as the value."""
    if rank != 0:
        return 0
    import oracle
    from oracle import estimate as oest
    inp = workload(args)
    # level bounds from the oracle's own pre-pass over a few steps (no GPU, no library)
    pooled = []
    for t in range(0, inp.n_t, max(1, inp.n_t // 2))[:2]:
        mu, _, _ = oracle.geneig(inp.vis[t], oracle.gram(inp.st_xyz[t], inp.wl))
        pooled.extend(mu[: inp.n_eig])
    bounds = np.array(oest.quantile_bounds(pooled, inp.n_level))
    cores = os.cpu_count()
    n_st = inp.st_xyz[0].shape[0]
    if args.synthesis == "nufft":
        for _ in range(args.warmup):
            cpu_sample_nufft(inp, bounds, args.nufft_eps, patch=32)  # warm-up: a small patch
        samples = [cpu_sample_nufft(inp, bounds, args.nufft_eps, t=k % inp.n_t) for k in range(args.steps)]
        wall = sum(x["t_s"] for x in samples)
        value = sum(x["products"] for x in samples) / wall
        sample = (f"per bench step one time step of the job (steps 0..{args.steps - 1}): FP64 Gram + Jacobi "
                  f"eigensolve of {n_st} stations and the FP64 numpy type-3 NUFFT of its {inp.n_level} level "
                  f"visibilities onto the central {samples[0]['n_sub']} pixels; value = products of those pixels / "
                  f"measured wall time; warm-up: the same on 32^2 pixels")
        extra = {}
    else:
        for k in range(args.warmup):
            cpu_sample(inp, bounds, t=k % inp.n_t, eig=False)  # warm-up: synthesis of the subset only
        samples = [cpu_sample(inp, bounds, t=k % inp.n_t) for k in range(args.steps)]
        wall = sum(x["wall_s"] for x in samples)
        value = sum(x["products"] for x in samples) / wall
        sample = (f"per bench step one time step of the job (steps 0..{args.steps - 1}): FP64 Gram + Jacobi "
                  f"eigensolve of {n_st} stations (single thread, mean {statistics.mean(x['t_eig_s'] for x in samples):.1f} s) "
                  f"and the synthesis of a strided {samples[0]['n_sub']}-pixel subset with its {inp.n_eig} kept "
                  f"eigenpairs (OpenMP over pixels, mean {statistics.mean(x['t_synth_sub_s'] for x in samples):.2f} s); "
                  f"value = products of that subset / measured wall time of the sample; warm-up steps run the "
                  f"subset synthesis only")
        extra = {"extrapolated_job_ms": statistics.median(x["extrapolated_job_ms"] for x in samples),
                 "extrapolation_note": ("the whole job (all pixels, all steps) scaled linearly from the samples: "
                                        "context only, not the value")}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "gpu_used": False, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": wall / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": config_dict(args, inp, args.precision),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}, **extra}
    print(json.dumps(line), flush=True)
    return 0


def ours_main(args, ws, rank, local):
    import torch

    from paper_2310_09200_b300 import bipp_ss, build
    from paper_2310_09200_b300.distributed import max_over_ranks
    build.build()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    inp = workload(args)
    n_st = inp.st_xyz[0].shape[0]
    # level bounds: the library's own parameter-estimation pre-pass on every 10th step
    bounds, _ = bipp_ss.estimate_level_bounds(inp.st_xyz[::10], inp.vis[::10], inp.wl, inp.n_eig, inp.n_level,
                                              eig_mode=args.eig)
    nst, N, st, V = bipp_ss.pack_batch(inp.st_xyz, inp.vis)
    d_st = torch.from_numpy(st).to(f"cuda:{local}")
    d_V = torch.from_numpy(V).to(f"cuda:{local}")
    stream = torch.cuda.Stream()
    nufft = args.synthesis == "nufft"
    extra = ({"synthesis": "nufft", "nufft_eps": args.nufft_eps, "nufft_partition": args.nufft_partition}
             if nufft else {})
    ss = bipp_ss.StandardSynthesis(inp.pix, inp.wl, bounds, n_eig=inp.n_eig, precision=args.precision,
                                   device=local, eig_mode=args.eig, **extra)

    def one_step():
        bipp_ss.bipp_ss_collect_device(ss.h, nst, d_st, d_V, stream=stream)
        return ss.timings()

    for _ in range(args.warmup):
        one_step()
    sfu_rate = bipp_ss.bipp_ss_measure_sincos_rate(local, 5)  # the SFU bound's rate, on this GPU now
    fp32_rate, fp64_rate = bipp_ss.bipp_ss_measure_fma_rates(local, 5)  # CUDA-core FMA rates (flop/s)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = Clocks(local)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    stage = np.zeros(4)
    nu_ms = np.zeros(6)
    nu_last = None
    sweeps = 0
    launches = 0
    e0.record(stream)
    for _ in range(args.steps):
        t = one_step()
        stage += [t["gram_reduce_ms"], t["eig_ms"], t["select_ms"], t["synth_ms"]]
        sweeps += t["sweeps_total"]
        launches += t["launches"]
        if nufft:
            nu_last = ss.nufft_timings()
            nu_ms += [nu_last["sort_ms"], nu_last["spread_ms"], nu_last["pad_ms"], nu_last["fft_ms"],
                      nu_last["interp_ms"], nu_last["levels_ms"]]
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    if dist:
        dist.barrier()
    ms_total = e0.elapsed_time(e1)
    if dist:
        ms_total = max_over_ranks(ms_total, device=f"cuda:{local}")
    ms_step = ms_total / args.steps
    prods = inp.n_pix * inp.n_eig * n_st * inp.n_t
    value = prods * ws / (ms_step / 1e3)

    # ---- roofline of the dominant kernel and of the synthesis kernel
    K = args.steps
    eig_ms, syn_ms = stage[1] / K, stage[3] / K
    jac_flops = 20.0 * n_st ** 2 * (n_st - 1) * (sweeps / K)  # Hermitian two-sided rotations + Q, per launch
    syn_flops = 8.0 * prods  # one complex multiply-add per product
    if args.eig == "jacobi64":
        roof_jacobi = {"kernel": "k_jacobi_t<double>", "bound": "alu",
                       "achieved": jac_flops / (eig_ms / 1e3) / 1e12, "peak": fp64_rate / 1e12,
                       "unit": "TFLOP/s", "traffic": None,
                       "peak_note": "of measured: FP64 FMA rate of this GPU (bipp_ss_measure_fma_rates, this run)"}
        roof_jacobi["frac"] = roof_jacobi["achieved"] / roof_jacobi["peak"]
    else:
        roof_jacobi = eig_roofline(n_st, min(n_st, inp.n_eig + 16), inp.n_t, eig_ms, fp32_rate)
    if nufft:
        nt = dict(nu_last)
        for i, k in enumerate(["sort_ms", "spread_ms", "pad_ms", "fft_ms", "interp_ms", "levels_ms"]):
            nt[k] = nu_ms[i] / K
        roof_synth = nufft_roofline(nt, inp.n_level, inp.n_pix, inp.n_t, n_st, inp.n_eig,
                                    measured_peaks().get("hbm_gbs", 6400.0), fp32_rate)
    elif args.precision in ("fp32", "fp64"):
        peak = fp32_rate if args.precision == "fp32" else fp64_rate
        roof_synth = {"kernel": f"k_synth_{args.precision[-2:]}", "bound": "alu",
                      "achieved": syn_flops / (syn_ms / 1e3) / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
                      "traffic": None,
                      "peak_note": "of measured: CUDA-core FMA rate of this GPU (bipp_ss_measure_fma_rates, this run)"}
        roof_synth["frac"] = roof_synth["achieved"] / roof_synth["peak"]
    else:
        traffic = synth_tc_traffic({"n_st": int(n_st), "n_pix": int(inp.n_pix), "n_eig": int(inp.n_eig),
                                    "n_level": int(inp.n_level), "n_t": int(inp.n_t), "precision": args.precision})
        roof_synth = tc_roofline(syn_flops, syn_ms, inp.n_pix * n_st * inp.n_t, measured_peaks(), traffic,
                                 sfu_rate)
    # the dominant single kernel: the FP64 Jacobi when it runs, else the synthesis (the mixed
    # eigensolve is a stage of ~60 launches, the largest of which is well below the synthesis)
    dominant = roof_jacobi if (args.eig == "jacobi64" and eig_ms >= syn_ms) else roof_synth

    # ---- end to end through the host-buffer C ABI (pinned host inputs, images read back)
    e2e = None
    if not args.no_e2e:
        st_h = torch.from_numpy(st).pin_memory()
        V_h = torch.from_numpy(V).pin_memory()
        img_t = torch.zeros((inp.n_level, inp.n_pix), dtype=torch.float64).pin_memory()  # pinned, like the inputs
        img_h = img_t.numpy()
        bipp_ss.bipp_ss_collect_batch_packed(ss.h, nst, N, st_h.data_ptr(), V_h.data_ptr())
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        lib = bipp_ss.load()
        img_ptr = img_h.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        for _ in range(args.steps):
            bipp_ss.bipp_ss_collect_batch_packed(ss.h, nst, N, st_h.data_ptr(), V_h.data_ptr())
            if lib.bipp_ss_get_f64(ss.h, img_ptr) != 0:
                raise RuntimeError(bipp_ss.bipp_ss_last_error(ss.h))
        dt = (time.perf_counter() - t0) / args.steps
        if dist:
            dt = max_over_ranks(dt, device=f"cuda:{local}")
        e2e = {"value": prods * ws / dt, "unit": UNIT, "h2d_bytes_per_step": int(st.nbytes + V.nbytes),
               "d2h_bytes_per_step": int(img_h.nbytes)}
    synth_shape = synth_shape_of(ss.synth_shape)
    ss.close()

    cpu = None
    ref = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and nufft:
        s = cpu_sample_nufft(inp, bounds, args.nufft_eps)
        cpu = {"value": s["value"], "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": (f"one time step: FP64 Gram + Jacobi of {n_st} stations and the FP64 numpy type-3 NUFFT "
                          f"of its level visibilities onto the central {s['n_sub']} pixels ({s['t_s']:.1f} s); "
                          f"products of those pixels / measured time")}
    elif rank == 0 and ws == 1 and not args.no_cpu_baseline:
        ref = cpu_sample(inp, bounds)
        cpu = {"value": ref["value"], "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": (f"time step 0: FP64 Gram + Jacobi of {n_st} stations (single thread, "
                          f"{ref['t_eig_s']:.1f} s) + synthesis of a strided {ref['n_sub']}-pixel subset "
                          f"(OpenMP, {ref['t_synth_sub_s']:.2f} s); products of that subset / measured wall time "
                          f"of the sample"),
               "extrapolated_job_ms": ref["extrapolated_job_ms"]}
    forms = None
    if rank == 0 and not nufft and not args.no_forms:
        forms = precision_forms(args, inp, bounds, d_st, d_V, nst, local, ref)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": dtype_label(args), "data": "synthetic",
                "config": config_dict(args, inp, args.precision),
                "stage_ms_per_step": {"gram_chol_reduce": stage[0] / K, "jacobi": eig_ms,
                                      "select_pack": stage[2] / K, "synthesis": syn_ms},
                **({"nufft_ms_per_step": {"sort": nu_ms[0] / K, "spread": nu_ms[1] / K,
                                          "pad_per_level": nu_ms[2] / K, "fft_per_level": nu_ms[3] / K,
                                          "interp_per_level": nu_ms[4] / K, "levels": nu_ms[5] / K}}
                   if nufft else {}),
                "synthesis_only_value": prods / (syn_ms / 1e3),
                "roofline": dominant, "roofline_synthesis": roof_synth, "roofline_jacobi": roof_jacobi,
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
                **({"synth_shape": synth_shape} if synth_shape and synth_shape["stages"] else {}),
                **({"precision_forms": forms} if forms else {})}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def precision_forms(args, inp, bounds, d_st, d_V, nst, local, ref):
    """The precision forms side by side on the same job (outside the timed
    region): the synthesis stage of its first 10 steps on all pixels in the
    plain FP32 CUDA-core path and the two split tensor-core forms (best of two
    collects after one that autotunes and captures the graph), and, when the
    oracle sample `ref` of step 0 is at hand, each form's per-level relative L2
    error on that sample's pixels against the FP64 oracle."""
    from paper_2310_09200_b300 import bipp_ss
    n10 = min(10, inp.n_t)
    n_st = inp.st_xyz[0].shape[0]
    prods = float(inp.n_pix) * inp.n_eig * n_st * n10
    out = {"note": (f"synthesis stage of steps 0..{n10 - 1} on all {inp.n_pix} pixels (CUDA events in the library, "
                    "best of 2 after a warm-up collect); level_rel_l2_vs_oracle: step 0 on the strided "
                    "pixel subset of the CPU sample, GPU eigensolve and synthesis against the FP64 oracle's")}
    for prec in ("fp32", "split_bf16", "split_fp16"):
        with bipp_ss.StandardSynthesis(inp.pix, inp.wl, bounds, n_eig=inp.n_eig, precision=prec, device=local,
                                       eig_mode=args.eig) as ss:
            ms = []
            for k in range(3):
                bipp_ss.bipp_ss_collect_device(ss.h, nst[:n10], d_st[:n10], d_V[:n10])
                if k:
                    ms.append(ss.timings()["synth_ms"])
        entry = {"synth_ms": min(ms), "synth_products_per_s": prods / (min(ms) / 1e3)}
        if ref is not None:
            with bipp_ss.StandardSynthesis(inp.pix[ref["sel"]], inp.wl, bounds, n_eig=inp.n_eig, precision=prec,
                                           device=local, eig_mode=args.eig) as ss:
                ss.collect(inp.st_xyz[0], inp.vis[0])
                got = ss.get()
            want = ref["img"]
            entry["level_rel_l2_vs_oracle"] = [
                float(np.linalg.norm(got[:, l] - want[:, l]) / max(np.linalg.norm(want[:, l]), 1e-300))
                for l in range(want.shape[1])]
        out[prec] = entry
    return out


if __name__ == "__main__":
    sys.exit(main())
