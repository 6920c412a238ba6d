#!/usr/bin/env python
"""Throughput of the GB300 linear elliptical slice sampler.

Metric: chain-iterations per second at d = 1000, m = 2000, 8192 chains (the
unit-norm Gaussian polytope family, b ~ U[0.05, 0.5], X0 = 0), for the mixed
form (FP16x3 tensor-core GEMM, FP32 step, FP64 checks) -- the headline value --
and the plain FP64 form, each with its roofline fraction.

A "step" is one pass of the whole hot path over all chains: nu draw, q = A nu,
roots + sort + sweep + theta draw + move (+ the A x refresh every refresh_k
steps, at its natural frequency).  Inputs are resident in HBM when the timed
region starts; the per-step working set (~300 MB) exceeds the 126 MB L2, so no
explicit flush is needed.  Timing: W warm-up steps, then K steps bracketed by
CUDA events on the run's stream (barrier + synchronize on both sides, max over
ranks).  Under torchrun each rank runs its own 8192 chains (weak scaling, no
collective on the data path).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
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
sys.path.insert(0, ROOT)

METRIC = "ESS chain-iter/s at d=1000,m=2000,8192 chains: mixed vs FP64, % of roofline"
UNIT = "chain-iter/s"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--fp64-steps", type=int, default=32)
    ap.add_argument("--fp64-split-steps", type=int, default=64)
    ap.add_argument("--chains", type=int, default=8192)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--chain-kernel", choices=["auto", "warp", "stream"], default="auto",
                    help="float chain-step kernel (ess_set_chain_kernel)")
    ap.add_argument("--mixed-only", action="store_true",
                    help="time only the mixed form (profiling runs)")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the short runs of the other configurations")
    ap.add_argument("--case", choices=sorted(CASES), default=None,
                    help="run one small named case and exit (the command profiles/ "
                         "summaries capture under ncu); prints one JSON line")
    return ap.parse_args()


def _case_chains(ess, torch, inst, C, prec, steps, seed=7):
    s = ess.Sampler(inst.A, inst.b, precision=prec)
    try:
        X = torch.tensor(inst.X0[0], dtype=torch.float64, device="cuda").repeat(C, 1).contiguous()
        ess.ess_chains_init(s.state, X, C, 0)
        ess.ess_chains_step(s.state, steps, seed)
        torch.cuda.synchronize()
        st = s.stats()
    finally:
        s.close()
    return {k: st[k] / max(1, st["steps"]) for k in ("residual_rechecks", "tangent_fp64",
                                                     "sort_keys", "rejections")}


def run_case(name):
    """Small single cases for ncu captures (each a few hundred MB on the
    device, a few launches of the kernel of interest)."""
    import torch
    import paper_2407_10449_gb300 as ess
    import workloads
    if name == "wide_metric":
        # metric family at m = 16384 (> 8192: the wide-row kernel), 1216 chains
        inst = workloads.metric(n_chains=1, m=16384)
        out = _case_chains(ess, torch, inst, 1216, ess.ESS_PREC_MIXED, 4)
    elif name == "wide_probit":
        inst = workloads.probit_features(n_chains=1)
        out = _case_chains(ess, torch, inst, 1216, ess.ESS_PREC_MIXED, 4)
    elif name == "probit":
        # the probit orthant of App. A (d = m = 2000, b = 0), 4096 chains:
        # the warp kernel with the long-arc union
        from types import SimpleNamespace
        import numpy as np
        pb = workloads.probit(n_chains=1)
        Aw, bw = ess.ess_whiten(pb["A0"], pb["b"], pb["mu"], np.linalg.cholesky(pb["K"]))
        inst = SimpleNamespace(A=Aw, b=bw, X0=pb["X0"])
        out = _case_chains(ess, torch, inst, 4096, ess.ESS_PREC_MIXED, 4)
    elif name == "batched":
        # 512 uneven polytopes, mixed form: refresh periods as graphs of
        # per-step launches and as one persistent launch each
        insts = workloads.batched()
        peaks = load_peaks()
        out = {}
        for persistent in (False, True):
            r = time_batch(ess, torch, insts, "mixed", 96, 4, 0, peaks, persistent=persistent,
                           per_step_graphs=not persistent)
            out["persistent" if persistent else "graphs"] = {
                "ms_per_step": r["ms_per_step"], "value": r["value"],
                "graph_launches": r["graph_launches"], "stats": r["stats"]}
    elif name == "paper_hd":
        # the Sec. 4.2 family with 1 and 10 chains through ess_run_few
        out = time_paper_hd(ess, torch, workloads, load_peaks(), 0)
    elif name == "hdr_box":
        inst = workloads.rotated_box()
        s = ess.Sampler(inst.A, inst.b, precision=ess.ESS_PREC_MIXED)
        try:
            r = ess.ess_hdr(s.state, 2048, 0.5, 4, 3)
        finally:
            s.close()
        out = {"levels": len(r["shifts"]), "log_z": r["log_z"], "exact": inst.meta["log_z"]}
    print(json.dumps({"case": name, **out}))
    return 0


CASES = ("wide_metric", "wide_probit", "hdr_box", "batched", "probit", "paper_hd")


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return {"hbm_gbs": p["hbm_gbs"], "bf16_tflops": p["bf16_tflops"],
                "bf16_tflops_sustained": p.get("bf16_tflops_sustained", p["bf16_tflops"]),
                "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "source": "fallback"}


# FP64 throughput, the denominator of the FP64 phases: measured in the run by
# measure_fp64_peak (cuBLAS DGEMM); this value stands in only if that fails.
FP64_TFLOPS_MEASURED = 1.19
FP64_PEAK_SOURCE = "fallback: earlier DFMA microbenchmark on this pool"


def measure_fp64_peak(torch, n=4096, reps=3):
    """FP64 dense throughput of this GPU in this run: the best of `reps`
    cuBLAS DGEMMs of n x n x n (2 n^3 flops), timed with CUDA events."""
    global FP64_TFLOPS_MEASURED, FP64_PEAK_SOURCE
    a = torch.randn((n, n), dtype=torch.float64, device="cuda")
    b = torch.randn((n, n), dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    best = float("inf")
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    del a, b
    FP64_TFLOPS_MEASURED = 2.0 * n**3 / (best * 1e-3) / 1e12
    FP64_PEAK_SOURCE = f"measured in this run: cuBLAS DGEMM {n}^3, best of {reps}"
    return FP64_TFLOPS_MEASURED


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.25)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        power = [num(r[3]) for r in rows if num(r[3]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(power) if power else None,
                "samples": len(rows), "reasons": reasons}


def dist_setup(n_gpus):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, value):
    """Largest value over the ranks (the job's time is its slowest rank's)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_seed(seed, rank):
    """Seed of a rank's replica: the replicas draw disjoint Philox streams."""
    return seed + 1000003 * rank


def job_throughput(world, chains_per_rank, steps, ms_max):
    """Whole-job chain-iterations per second from the slowest rank's time."""
    return world * chains_per_rank * steps / (ms_max / 1e3)


def source_hash(*names):
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_2407_10449_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


def ncu_counters(kernel_key, src_hash):
    """(DRAM bytes, warp instructions) per launch from the committed ncu
    summary, if it was taken on the current source of that kernel (else
    (None, None))."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.md")
    if not os.path.exists(path):
        return None, None
    with open(path) as f:
        for line in f:
            # | kernel_key | src_hash | dram bytes per launch | warp instructions | ... |
            parts = [p.strip() for p in line.strip().strip("|").split("|")]
            if len(parts) >= 4 and parts[0] == kernel_key and parts[1] == src_hash:
                def num(v):
                    try:
                        return float(v)
                    except ValueError:
                        return None
                return num(parts[2]), num(parts[3])
    return None, None


def step_roofline(roof, ms_per_step):
    """The whole step's roofline: the sum over its phases of each phase's
    lower bound (its algorithmic work at its peak; the chain kernel at the
    larger of its HBM and issue bounds; the refresh amortised over refresh_k
    steps), against the measured time per step.  The draw runs beside the q
    GEMM on a side stream and is left out."""
    parts = {}
    for ph, r in roof.items():
        if ph == "draw":
            continue
        scale = 1e6 if r["unit"] == "GB/s" else 1e9
        t = r["work_per_launch"] / (r["peak"] * scale)
        if ph == "chain" and r.get("issue"):
            t = max(t, r["issue"]["issue_limited_ms"])
        if ph == "refresh":
            t /= REFRESH_K
        parts[ph] = t
    bound = sum(parts.values())
    if not parts or not ms_per_step:
        return None
    return {"bound_ms_per_step": bound, "ms_per_step": ms_per_step, "frac": bound / ms_per_step,
            "phase_bound_ms": parts}


def issue_roofline(torch, inst_per_launch, ms_per_launch, sm_mhz):
    """The SM issue bound of a kernel: warp instructions per launch (ncu) over
    its live launch time, against one instruction per clock per scheduler
    (SM count x 4 schedulers x the median SM clock under load)."""
    if not inst_per_launch or not ms_per_launch:
        return None
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = sm_mhz or 2070.0
    peak = sms * 4 * mhz * 1e6
    ach = inst_per_launch / (ms_per_launch * 1e-3)
    return {"bound": "issue", "unit": "warp-inst/s", "achieved": ach, "peak": peak,
            "frac": ach / peak, "inst_per_launch": inst_per_launch, "sm_mhz": mhz,
            "issue_limited_ms": inst_per_launch / peak * 1e3}


def phase_rooflines(inst, n_chains, timing, precision, peaks):
    """Achieved vs peak for each phase of the timed region (per launch)."""
    d, m, C = inst.d, inst.m, n_chains
    mixed = precision == "mixed"
    split = precision == "fp64_split"
    esz = 4 if mixed else 8
    out = {}

    def slice_pairs(bits):
        # exact split: K (K + 1) / 2 bf16 slice products of w-bit slices,
        # (2^w - 1)^2 d <= 2^24, K = ceil(bits / w)
        w = 8
        while w > 1 and (2 ** w - 1) ** 2 * d > 2 ** 24:
            w -= 1
        K = min(-(-bits // w), 12)
        return K * (K + 1) / 2

    steps = timing.get("draw", {}).get("launches", 0)
    for phase, t in timing.items():
        if t["launches"] == 0 or t["ms"] <= 0:
            continue
        # the chain phase is one warp-per-chain launch plus the (usually empty)
        # CTA-per-chain launch for overflow chains: time it per step
        units = steps if phase == "chain" and steps else t["launches"]
        ms = t["ms"] / units
        if phase == "gemm":
            if mixed:
                # three fp16 slice products issued (FP16x3); the fp16 dense rate
                # equals the bf16 one (nominal ratio 1:1), so the measured bf16
                # peak is the denominator
                flops = 3 * 2.0 * m * d * C
                peak = peaks["bf16_tflops_sustained"]
                out[phase] = dict(bound="tensor", unit="TFLOP/s", achieved=flops / ms / 1e9,
                                  peak=peak, work_per_launch=flops, useful_flops=flops / 3)
            elif split:
                # FP64 products from 56-bit splits: the slice products issued
                flops = slice_pairs(56) * 2.0 * m * d * C
                out[phase] = dict(bound="tensor", unit="TFLOP/s", achieved=flops / ms / 1e9,
                                  peak=peaks["bf16_tflops_sustained"], work_per_launch=flops,
                                  useful_flops=2.0 * m * d * C)
            else:
                flops = 2.0 * m * d * C
                out[phase] = dict(bound="fp64", unit="TFLOP/s", achieved=flops / ms / 1e9,
                                  peak=FP64_TFLOPS_MEASURED, work_per_launch=flops)
        elif phase == "refresh":
            if mixed or split:
                # exact split (35 bits mixed, 56 bits for the FP64 form; K = 5
                # and 8 slices per operand at d = 1000)
                flops = slice_pairs(35 if mixed else 56) * 2.0 * m * d * C
                out[phase] = dict(bound="tensor", unit="TFLOP/s", achieved=flops / ms / 1e9,
                                  peak=peaks["bf16_tflops_sustained"], work_per_launch=flops,
                                  useful_flops=2.0 * m * d * C)
            else:
                flops = 2.0 * m * d * C
                out[phase] = dict(bound="fp64", unit="TFLOP/s", achieved=flops / ms / 1e9,
                                  peak=FP64_TFLOPS_MEASURED, work_per_launch=flops)
        elif phase == "chain":
            # read p, q (m each), write p; read x, nu, write x (d each)
            byts = float(C) * esz * (3 * m + 3 * d)
            out[phase] = dict(bound="hbm", unit="GB/s", achieved=byts / ms / 1e6,
                              peak=peaks["hbm_gbs"], work_per_launch=byts)
        elif phase == "draw":
            byts = float(C) * d * (esz + (4 if mixed else 0))  # nu (+ two fp16 slices)
            out[phase] = dict(bound="hbm", unit="GB/s", achieved=byts / ms / 1e6,
                              peak=peaks["hbm_gbs"], work_per_launch=byts)
        out[phase]["ms_per_launch"] = ms
        out[phase]["launches"] = t["launches"]
        out[phase]["units"] = units
        out[phase]["share"] = t["ms"] / sum(v["ms"] for v in timing.values())
        out[phase]["frac"] = out[phase]["achieved"] / out[phase]["peak"]
    return out


REFRESH_K = 32


def aligned_warmup(warmup, refresh_k=REFRESH_K):
    """Warm-up steps that end on a refresh boundary (at least `warmup`), so
    that the timed window starts with a refresh and holds the refreshes of
    its steps at their natural frequency (one every refresh_k steps)."""
    return warmup + (-warmup) % refresh_k


def refreshes_in(t0, steps, refresh_k=REFRESH_K):
    return sum(1 for t in range(t0, t0 + steps) if t % refresh_k == 0)


CHAIN_KERNEL = "auto"


def time_form(ess, torch, inst, precision, n_chains, steps, warmup, seed, world, rank,
              clocks=None, phase_steps=None, keep=0):
    """Exactly `steps` steps through ess_chains_step on the run's stream as a
    user runs them (refresh periods replayed from CUDA graphs), starting on a
    refresh boundary, timed by CUDA events; then a second pass with per-phase
    events (plain launches) for the phase table.  keep > 0: also returns the
    states of `keep` chains after the timed steps (host, float64)."""
    prec = ess.ESS_PREC_MIXED if precision == "mixed" else ess.ESS_PREC_FP64
    cfg = {"fp64_products": ess.ESS_PRODUCTS_SPLIT} if precision == "fp64_split" else {}
    s = ess.Sampler(inst.A, inst.b, precision=prec, refresh_k=REFRESH_K, **cfg)
    if CHAIN_KERNEL != "auto":
        ess.ess_set_chain_kernel(s.state, {"warp": ess.ESS_CHAIN_WARP,
                                           "stream": ess.ESS_CHAIN_STREAM}[CHAIN_KERNEL])
    stream = torch.cuda.Stream()
    x0 = torch.as_tensor(inst.X0[0], dtype=torch.float64)
    X = x0.to("cuda").repeat(n_chains, 1).contiguous()
    w = aligned_warmup(warmup)
    ess.ess_chains_init(s.state, X, n_chains, 0, stream)
    ess.ess_chains_step(s.state, w, seed, stream=stream)
    ess.ess_chains_get(s.state, None, stream)
    ess.ess_reset_timing(s.state)
    s.reset_stats()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    e0.record(stream)
    ess.ess_chains_step(s.state, steps, seed, stream=stream)
    e1.record(stream)
    e1.synchronize()
    clk = clocks.stop() if clocks else None
    torch.cuda.synchronize()
    barrier(world)
    kept = None
    if keep:
        out = torch.empty_like(X)
        ess.ess_chains_get(s.state, out, stream)
        torch.cuda.synchronize()
        kept = out[:keep].cpu().numpy().astype("float64")
    else:
        ess.ess_chains_get(s.state, None, stream)
    ms = e0.elapsed_time(e1)
    ms_max = max_over_ranks(world, ms)
    launches = sum(t["launches"] for t in ess.ess_get_timing(s.state).values())
    graphs = ess.ess_graph_launches(s.state)
    stats = s.stats()
    # phase table: per-phase events around plain launches
    ps = phase_steps or steps
    ess.ess_reset_timing(s.state)
    ess.ess_set_timing(s.state, True)
    ess.ess_chains_step(s.state, ps, seed, stream=stream)
    ess.ess_chains_get(s.state, None, stream)
    timing = ess.ess_get_timing(s.state)
    s.close()
    window = {"t0": w, "steps": steps, "refreshes": refreshes_in(w, steps),
              "refresh_k": REFRESH_K}
    return ms_max, timing, stats, clk, {"gpu_launches": launches, "graph_launches": graphs,
                                        "window": window, "states": kept}


# FP32 FMA peak of the GPU at the maximum SM clock (152 SMs x 128 FMA/clk x 2
# flops x 2.07 GHz on GB300); the batched GEMM runs on the FP32 pipe.
def fp32_peak_tflops(torch):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    return sms * 128 * 2 * 2.07e9 / 1e12


def batch_phase_rooflines(insts, timing, precision, torch, peaks):
    """Phase rooflines of the batched sampler (work summed over problems)."""
    mixed = precision == "mixed"
    esz = 4 if mixed else 8
    mdC = sum(i.m * i.d * i.n_chains for i in insts)
    steps = timing.get("draw", {}).get("launches", 0)
    fp = fp32_peak_tflops(torch) if mixed else FP64_TFLOPS_MEASURED
    work = {
        "draw": ("hbm", "GB/s", float(sum(i.d * i.n_chains for i in insts) * esz),
                 peaks["hbm_gbs"]),
        # mixed: the tcgen05 grouped GEMM streams each problem's fp16 A splits
        # once (4 B per element of A), its chains' nu splits once per 128-row
        # tile and writes Q: HBM-bound (arithmetic intensity ~1.5 N flops per
        # byte of A for N chains); FP64 form: DFMAs
        "gemm": (("hbm", "GB/s",
                  float(sum(4 * i.m * i.d + 4 * i.n_chains * i.d * (-(-i.m // 128))
                            + 4 * i.n_chains * i.m for i in insts)),
                  peaks["hbm_gbs"]) if mixed else ("fp64", "TFLOP/s", 2.0 * mdC, fp)),
        "chain": ("hbm", "GB/s", float(sum(i.n_chains * esz * (3 * i.m + 3 * i.d) for i in insts)),
                  peaks["hbm_gbs"]),
        # double-float refresh: ~11 FP32 operations per multiply-add
        "refresh": ("fp32" if mixed else "fp64", "TFLOP/s", 2.0 * mdC,
                    fp / 5.5 if mixed else fp),
    }
    out = {}
    total = sum(v["ms"] for v in timing.values()) or 1.0
    for phase, t in timing.items():
        if t["launches"] == 0 or t["ms"] <= 0:
            continue
        bound, unit, w, peak = work[phase]
        units = steps if phase == "chain" and steps else t["launches"]
        ms = t["ms"] / units
        scale = 1e6 if unit == "GB/s" else 1e9
        ach = w / ms / scale
        out[phase] = dict(bound=bound, unit=unit, achieved=ach, peak=peak, frac=ach / peak,
                          ms_per_launch=ms, work_per_launch=w, launches=t["launches"],
                          share=t["ms"] / total)
    return out


def time_batch(ess, torch, insts, precision, steps, warmup, seed, peaks, persistent=False,
               per_step_graphs=False):
    """Batched problems: value from a timed run (refresh periods replayed as
    CUDA graphs: in the mixed form by default one persistent cooperative launch
    each, with `per_step_graphs` a graph of per-step launches), phases from a
    second run with per-phase events (plain launches; skipped when `persistent`
    or `per_step_graphs` is set)."""
    prec = ess.ESS_PREC_MIXED if precision == "mixed" else ess.ESS_PREC_FP64
    As = [i.A for i in insts]
    bs = [i.b for i in insts]
    nc = [i.n_chains for i in insts]
    s = ess.BatchSampler(As, bs, precision=prec, refresh_k=REFRESH_K)
    if persistent or per_step_graphs:
        ess.ess_batch_set_persistent(s.batch, not per_step_graphs)
    X = s.pack([i.X0 for i in insts])
    stream = torch.cuda.current_stream()
    warmup = aligned_warmup(warmup)
    s.run(nc, X, warmup, seed)
    s.reset_stats()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    s.run(nc, X, steps, seed, t0=warmup)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    stats = s.stats()
    info = ess.ess_batch_info(s.batch)
    phases = {}
    if not (persistent or per_step_graphs):
        ess.ess_batch_set_timing(s.batch, True)
        ess.ess_batch_reset_timing(s.batch)
        s.run(nc, X, steps, seed, t0=warmup + steps)
        timing = ess.ess_batch_get_timing(s.batch)
        phases = batch_phase_rooflines(insts, timing, precision, torch, peaks)
    s.close()
    n = sum(nc)
    return {"value": n * steps / (ms / 1e3), "unit": UNIT, "steps": steps,
            "ms_per_step": ms / steps, "chains": n, "graph_launches": info["graph_launches"],
            "window": {"t0": warmup, "steps": steps, "refreshes": refreshes_in(warmup, steps),
                       "refresh_k": REFRESH_K},
            "phases": phases, "stats": stats}


def time_unwhiten(ess, torch, pb, n, peaks, reps=10):
    """App. A map x = L u + mu on the GPU for one record of n samples (d x d L)."""
    d = pb["L"].shape[0]
    w = ess.Whitener(pb["L"], pb["mu"])
    out = {}
    g = torch.Generator(device="cuda").manual_seed(0)
    for name, dt in (("float", torch.float32), ("double", torch.float64)):
        U = torch.randn((n, d), generator=g, device="cuda", dtype=dt)
        X = torch.empty_like(U)
        for _ in range(3):
            ess.ess_whitener_apply(w._w, U, X)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            ess.ess_whitener_apply(w._w, U, X)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / reps
        if dt == torch.float32:
            flops = 3 * 2.0 * n * d * d  # three fp16 products (FP16x3)
            peak = peaks["bf16_tflops_sustained"]
        else:
            flops = 2.0 * n * d * d
            peak = FP64_TFLOPS_MEASURED
        ach = flops / ms / 1e9
        out[name] = {"ms": ms, "samples_per_s": n / (ms / 1e3), "achieved_tflops": ach,
                     "peak_tflops": peak, "frac": ach / peak}
    w.close()
    return out


def time_cholesky(ess, torch, K, reps=3):
    """L = chol(K) on the GPU (ess_cholesky, FP64): the best of `reps` timed
    factorisations (CUDA events; the matrix copied in before each); n^3 / 3
    multiply-adds against the FP64 peak measured in the run."""
    n = K.shape[0]
    src = torch.tensor(np.ascontiguousarray(K), dtype=torch.float64, device="cuda")
    A = torch.empty_like(src)
    best = float("inf")
    for _ in range(reps + 1):
        A.copy_(src)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        ess.ess_cholesky(A)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    flops = n ** 3 / 3.0
    L = torch.tril(A).cpu().numpy()
    return {"n": n, "ms": best, "achieved_tflops": flops / (best * 1e-3) / 1e12,
            "peak_tflops": FP64_TFLOPS_MEASURED,
            "frac": flops / (best * 1e-3) / 1e12 / FP64_TFLOPS_MEASURED, "L": L}


def time_configs(ess, torch, workloads, peaks, seed, errors=True):
    """The other configurations, both forms, short runs (parity-tested
    elsewhere; reported here with their phase rooflines)."""
    from types import SimpleNamespace
    out = {}
    singles = [("small_d10_m20_c16", workloads.small(n_chains=1), 16, (192, 192)),
               ("medium_d100_m200_c1024", workloads.medium(n_chains=1), 1024, (192, 96))]
    pb = workloads.probit(n_chains=1)
    # App. A's factor of K on the GPU (FP64 blocked Cholesky), then the whitening
    chol = time_cholesky(ess, torch, pb["K"])
    pb["L"] = chol.pop("L")
    Aw, bw = ess.ess_whiten(pb["A0"], pb["b"], pb["mu"], pb["L"])
    singles.append(("probit_n2000_c4096",
                    SimpleNamespace(A=Aw, b=bw, X0=pb["X0"], d=Aw.shape[1], m=Aw.shape[0]),
                    4096, (64, 32)))
    for name, inst, C, (st_mixed, st_fp64) in singles:
        entry = {}
        for form, steps in (("mixed", st_mixed), ("fp64", st_fp64),
                            ("fp64_split", max(st_fp64, min(st_mixed, 64)))):
            ms, timing, stats, _, lc = time_form(ess, torch, inst, form, C, steps, 3, seed, 1, 0,
                                                 keep=ERR_SAMPLE if errors else 0)
            ph = phase_rooflines(inst, C, timing, form, peaks)
            dom = max(ph, key=lambda k: ph[k]["share"]) if ph else None
            entry[form] = {"value": C * steps / (ms / 1e3), "unit": UNIT, "steps": steps,
                           "ms_per_step": ms / steps, "window": lc["window"],
                           "dominant": dom, "dominant_frac": ph[dom]["frac"] if dom else None,
                           "phases": ph, "graph_launches": lc["graph_launches"],
                           "rejections": stats["rejections"],
                           "numeric_errors": stats["numeric_errors"]}
            if errors:
                entry[form]["error_vs_oracle"] = oracle_errors(ess, torch, inst.A, inst.b,
                                                               lc["states"], form, seed)
        if C <= 16:
            # the few-chain FP64 path: every step of the run in one cooperative kernel
            entry["fp64_few"] = time_few(ess, torch, inst, C, 1000, seed)
        out[name] = entry
    out["probit_n2000_c4096"]["unwhiten"] = time_unwhiten(ess, torch, pb, 4096, peaks)
    out["probit_n2000_c4096"]["cholesky"] = chol
    insts = workloads.batched()
    entry = {}
    for form, steps in (("mixed", 64), ("fp64", 32)):
        # mixed: refresh periods as one persistent launch each (the default);
        # phases from plain per-step launches
        r = time_batch(ess, torch, insts, form, steps, 4, seed, peaks)
        ph = r["phases"]
        dom = max(ph, key=lambda k: ph[k]["share"]) if ph else None
        r["dominant"] = dom
        r["dominant_frac"] = ph[dom]["frac"] if dom else None
        if errors:
            r["error_vs_oracle"] = batch_oracle_errors(ess, torch, insts, form, seed)
        entry[form] = r
    # the same mixed run with refresh periods as graphs of per-step launches
    r = time_batch(ess, torch, insts, "mixed", 64, 4, seed, peaks, persistent=False,
                   per_step_graphs=True)
    entry["mixed_per_step_graphs"] = {k: r[k] for k in ("value", "unit", "ms_per_step",
                                                        "graph_launches", "window")}
    out["batched_512_problems"] = entry
    out.update(time_paper_hd(ess, torch, workloads, peaks, seed))
    out.update(time_wide(ess, torch, workloads, peaks, seed, errors))
    out.update(time_hdr(ess, torch, workloads, seed))
    return out


def time_hdr(ess, torch, workloads, seed):
    """Normal probability of a rotated box (d = 200, m = 400, exact log Z =
    200 log(Phi(1.5) - Phi(-1))) by ess_hdr: 8192 samples per level, rho =
    1/2, 8 chain steps between levels, both stages; the whole call timed by
    CUDA events, its chain steps counted for a throughput in the metric's unit."""
    inst = workloads.rotated_box()
    want = inst.meta["log_z"]
    n, rho, kb = 8192, 0.5, 8
    out = {}
    for form, prec in (("mixed", ess.ESS_PREC_MIXED), ("fp64", ess.ESS_PREC_FP64)):
        s = ess.Sampler(inst.A, inst.b, precision=prec)
        try:
            ess.ess_hdr(s.state, 1024, rho, 2, seed + 7)  # warm-up (allocations, kernels)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            r = ess.ess_hdr(s.state, n, rho, kb, seed)
            e1.record()
            e1.synchronize()
            ms = e0.elapsed_time(e1)
        finally:
            s.close()
        T = len(r["shifts"])
        # chain steps: stage 1 runs T - 1 level transitions, stage 2 as many
        steps = 2 * (T - 1) * kb
        p = r["counts"] / n
        se = float(np.sqrt(np.sum((1 - p) / (n * p))))
        out[form] = {"ms_per_estimate": ms, "levels": T, "log_z": r["log_z"],
                     "log_z_ss": r["log_z_ss"], "log_z_exact": want,
                     "error": r["log_z"] - want, "naive_se": se,
                     "chain_iter_per_s": n * steps / (ms / 1e3), "unit": UNIT}
    return {"hdr_rotated_box_d200_m400": out}


def time_wide(ess, torch, workloads, peaks, seed, errors=True):
    """m beyond the CTA kernel's 8192 arcs: the metric family at m = 16384
    (the warp kernel keeps nearly every chain) and a probit-style orthant at
    m = 16384, d = 256 (every arc survives the prune: every chain goes to the
    wide-row kernel), both forms, with the phase rooflines of time_configs."""
    out = {}
    cases = [("metric_d1000_m16384_c8192", workloads.metric(n_chains=1, m=16384), 8192,
              (("mixed", 64), ("fp64", 32))),
             ("probit_features_d256_m16384_c2048", workloads.probit_features(n_chains=1), 2048,
              (("mixed", 64), ("fp64", 32)))]
    for name, inst, C, forms in cases:
        entry = {"m": inst.m, "d": inst.d, "chains": C}
        for form, steps in forms:
            ms, timing, stats, _, lc = time_form(ess, torch, inst, form, C, steps, 3, seed, 1, 0,
                                                 keep=ERR_SAMPLE if errors else 0)
            ph = phase_rooflines(inst, C, timing, form, peaks)
            dom = max(ph, key=lambda k: ph[k]["share"]) if ph else None
            entry[form] = {"value": C * steps / (ms / 1e3), "unit": UNIT, "steps": steps,
                           "ms_per_step": ms / steps, "window": lc["window"],
                           "dominant": dom, "dominant_frac": ph[dom]["frac"] if dom else None,
                           "phases": ph, "rejections": stats["rejections"],
                           "numeric_errors": stats["numeric_errors"],
                           "arcs_per_chain_step": stats["sort_keys"] / max(1, stats["steps"])}
            if errors:
                entry[form]["error_vs_oracle"] = oracle_errors(ess, torch, inst.A, inst.b,
                                                               lc["states"], form, seed)
        out[name] = entry
    return out


def time_few(ess, torch, inst, C, steps, seed):
    """C <= 16 FP64 chains through ess_run_few (all steps in one persistent
    cooperative kernel), timed with CUDA events after an 8-step warm-up."""
    s = ess.Sampler(inst.A, inst.b, precision=ess.ESS_PREC_FP64)
    try:
        X = torch.tensor(inst.X0[0], dtype=torch.float64, device="cuda").repeat(C, 1).contiguous()
        ess.ess_run_few(s.state, X, C, 0, 8, seed)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        ess.ess_run_few(s.state, X, C, 8, steps, seed)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        st = s.stats()
    finally:
        s.close()
    return {"value": C * steps / (ms / 1e3), "unit": UNIT, "steps": steps,
            "us_per_step": 1e3 * ms / steps, "dtype": "f64", "call": "ess_run_few",
            "rejections": st["rejections"], "numeric_errors": st["numeric_errors"]}


def time_paper_hd(ess, torch, workloads, peaks, seed):
    """Sec. 4.2 family (A d x d iid N(0, 1), b = A x0 + U[0, 1], m = d) with 1
    and 10 chains: the few-chain FP64 path (ess_run_few, one persistent
    kernel per run), with A read once per step (8 m d bytes) against the HBM
    peak, and the generic mixed path on the same chains for context."""
    out = {}
    for d in (1000, 2000, 4000):
        for C, steps in ((1, 200), (10, 50)):
            inst = workloads.paper_hd(d=d, n_chains=C)
            s = ess.Sampler(inst.A, inst.b, precision=ess.ESS_PREC_FP64)
            X = torch.tensor(inst.X0, dtype=torch.float64, device="cuda")
            ess.ess_run_few(s.state, X, C, 0, 8, seed)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            ess.ess_run_few(s.state, X, C, 8, steps, seed)
            e1.record()
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            st = s.stats()
            s.close()
            a_gbs = 8.0 * d * d / (ms / steps * 1e-3) / 1e9
            entry = {"value": C * steps / (ms / 1e3), "unit": UNIT, "steps": steps,
                     "us_per_step": 1e3 * ms / steps, "dtype": "f64", "call": "ess_run_few",
                     "roofline": {"bound": "hbm", "achieved": a_gbs, "peak": peaks["hbm_gbs"],
                                  "unit": "GB/s", "frac": a_gbs / peaks["hbm_gbs"],
                                  "work_per_step": 8.0 * d * d},
                     "arcs_per_chain_step": st["sort_keys"] / max(1, st["steps"])}
            # the generic path's mixed form on the same chains
            sm = ess.Sampler(inst.A, inst.b, precision=ess.ESS_PREC_MIXED)
            Xm = torch.tensor(inst.X0, dtype=torch.float64, device="cuda")
            ess.ess_chains_init(sm.state, Xm, C, 0)
            ess.ess_chains_step(sm.state, 32, seed)
            torch.cuda.synchronize()
            e0.record()
            ess.ess_chains_step(sm.state, steps, seed)
            e1.record()
            e1.synchronize()
            msm = e0.elapsed_time(e1)
            sm.close()
            entry["generic_mixed"] = {"value": C * steps / (msm / 1e3),
                                      "us_per_step": 1e3 * msm / steps}
            out[f"paper_hd_d{d}_c{C}"] = entry
    return out


def time_e2e(ess, torch, inst, n_chains, steps, seed, record_every=10):
    """One user call through the C ABI with host buffers: pinned X0 in, K steps,
    samples (every record_every steps) and final states out."""
    s = ess.Sampler(inst.A, inst.b, precision=ess.ESS_PREC_MIXED)
    X = torch.zeros((n_chains, inst.d), dtype=torch.float64).pin_memory()
    n_rec = steps // record_every
    S = torch.zeros((n_chains, max(n_rec, 1), inst.d), dtype=torch.float32).pin_memory()
    Xn = X.numpy()
    # warm-up call (module load, work buffers)
    ess.ess_run_host(s.state, Xn, n_chains, 0, 2, seed, S.numpy(), 1 if n_rec else 0)
    X.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ess.ess_run_host(s.state, Xn, n_chains, 0, steps, seed, S.numpy(),
                     record_every if n_rec else 0)
    dt = time.perf_counter() - t0
    s.close()
    h2d = n_chains * inst.d * 8
    d2h = n_chains * inst.d * 8 + n_rec * n_chains * inst.d * 4
    return {"value": n_chains * steps / dt, "unit": UNIT,
            "h2d_bytes_per_step": h2d / steps, "d2h_bytes_per_step": d2h / steps,
            "seconds": dt, "call": "ess_run_host", "record_every": record_every}


ERR_SAMPLE = 32


def _step_errors(theta_g, x_g, rej_g, refs):
    """Largest and median angle error (rad) and largest relative iterate error
    of the GPU's one-step map against the oracle's, plus rejection mismatches."""
    import numpy as np
    th_o = np.array([r.theta for r in refs])
    x_o = np.stack([r.x_next for r in refs])
    rej_o = np.array([r.rejected for r in refs])
    dth = np.abs(theta_g - th_o)
    dx = np.max(np.abs(x_g - x_o) / np.maximum(1.0, np.abs(x_o)), axis=1)
    return {"chains": int(len(refs)), "max_theta_err_rad": float(dth.max()),
            "median_theta_err_rad": float(np.median(dth)), "max_x_rel_err": float(dx.max()),
            "median_x_rel_err": float(np.median(dx)),
            "rejection_mismatches": int(np.sum(rej_o != (rej_g != 0)))}


def oracle_errors(ess, torch, A, b, states, form, seed, n=ERR_SAMPLE):
    """Part of the CPU-baseline (oracle) leg: one step of `n` chains taken from
    the states after the timed run, with given draws (seeded numpy normals
    and uniforms), through ess_step_with_draws on the GPU and through the
    oracle's one-step map; the mixed form's inputs are rounded to float on
    both sides, as the mixed form stores them."""
    import numpy as np
    import oracle
    rng = np.random.default_rng(seed + 17)
    X = np.asarray(states[:n], dtype=np.float64)
    NU = rng.standard_normal(X.shape)
    U = rng.uniform(size=X.shape[0])
    if form == "mixed":
        X = X.astype(np.float32).astype(np.float64)
        NU = NU.astype(np.float32).astype(np.float64)
    prec = ess.ESS_PREC_MIXED if form == "mixed" else ess.ESS_PREC_FP64
    cfg = {"fp64_products": ess.ESS_PRODUCTS_SPLIT} if form == "fp64_split" else {}
    s = ess.Sampler(A, b, precision=prec, **cfg)
    try:
        cuda = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
        Xn, th, _, _, rej = s.step_with_draws(cuda(X), cuda(NU), cuda(U))
        Xn, th, rej = (t.cpu().numpy() for t in (Xn, th, rej))
    finally:
        s.close()
    t0 = time.perf_counter()
    refs = [oracle.step(A, b, X[c], NU[c], U[c]) for c in range(X.shape[0])]
    dt = time.perf_counter() - t0
    out = _step_errors(th, Xn.astype(np.float64), rej, refs)
    out["oracle_chain_iter_per_s_1core"] = X.shape[0] / dt
    return out


def batch_oracle_errors(ess, torch, insts, form, seed, n=ERR_SAMPLE):
    """As oracle_errors for the batched sampler: one step of every chain of
    the batch from its start state with given draws; `n` chains spread over
    the problems are compared with the oracle (each with its own A, b)."""
    import numpy as np
    import oracle
    rng = np.random.default_rng(seed + 29)
    prec = ess.ESS_PREC_MIXED if form == "mixed" else ess.ESS_PREC_FP64
    As = [i.A for i in insts]
    bs = [i.b for i in insts]
    nc = [i.n_chains for i in insts]
    Xs = [np.asarray(i.X0, dtype=np.float64) for i in insts]
    NUs = [rng.standard_normal(x.shape) for x in Xs]
    if form == "mixed":
        Xs = [x.astype(np.float32).astype(np.float64) for x in Xs]
        NUs = [v.astype(np.float32).astype(np.float64) for v in NUs]
    U = rng.uniform(size=sum(nc))
    s = ess.BatchSampler(As, bs, precision=prec)
    try:
        Xn, th, rej = s.step_with_draws(nc, s.pack(Xs), s.pack(NUs),
                                        torch.tensor(U, dtype=torch.float64, device="cuda"))
        Xn = s.unpack(Xn, nc)
        th, rej = th.cpu().numpy(), rej.cpu().numpy()
    finally:
        s.close()
    offs = np.concatenate([[0], np.cumsum(nc)])
    chains = [(p, c) for p in range(len(insts)) for c in range(nc[p])]
    pick = rng.choice(len(chains), size=min(n, len(chains)), replace=False)
    refs, thg, xg, rg = [], [], [], []
    for k in pick:
        p, c = chains[k]
        g = offs[p] + c
        refs.append(oracle.step(As[p], bs[p], Xs[p][c], NUs[p][c], U[g]))
        thg.append(th[g])
        xg.append(np.asarray(Xn[p][c], dtype=np.float64))
        rg.append(rej[g])
    dth = np.abs(np.array(thg) - np.array([r.theta for r in refs]))
    dx = np.array([np.max(np.abs(x - r.x_next) / np.maximum(1.0, np.abs(r.x_next)))
                   for x, r in zip(xg, refs)])
    return {"chains": int(len(refs)), "max_theta_err_rad": float(dth.max()),
            "median_theta_err_rad": float(np.median(dth)), "max_x_rel_err": float(dx.max()),
            "median_x_rel_err": float(np.median(dx)),
            "rejection_mismatches": int(sum(bool(r.rejected) != bool(x) for r, x in zip(refs, rg)))}


def cpu_baseline(inst_small_fn, n_chains=256, n_iter=4):
    """The FP64 oracle, as it stands, on the host cores (bounded sample)."""
    import oracle
    inst = inst_small_fn(n_chains)
    cores = os.cpu_count() or 1
    oracle.run(inst.A, inst.b, inst.X0[:cores], 1, seed=0, n_threads=cores)  # warm-up
    t0 = time.perf_counter()
    oracle.run(inst.A, inst.b, inst.X0, n_iter, seed=0, n_threads=cores)
    dt = time.perf_counter() - t0
    return {"value": n_chains * n_iter / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n_chains} chains x {n_iter} steps of the d=1000, m=2000 workload "
                      f"({dt:.1f} s wall)"}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    import workloads
    per_step = 128
    inst = workloads.metric(n_chains=per_step)
    cores = os.cpu_count() or 1
    X = inst.X0.copy()
    for w in range(args.warmup):
        X, _, _ = oracle.run(inst.A, inst.b, X, 1, seed=args.seed, t0=w, n_threads=cores)
    t0 = time.perf_counter()
    for k in range(args.steps):
        X, _, _ = oracle.run(inst.A, inst.b, X, 1, seed=args.seed, t0=args.warmup + k,
                             n_threads=cores)
    dt = time.perf_counter() - t0
    value = per_step * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "metric_d1000_m2000", "d": 1000, "m": 2000,
                       "chains_per_step": per_step, "note": "FP64 CPU oracle, bounded sample"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} chains per step, {args.steps} steps"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse_args()
    if args.case:
        return run_case(args.case)
    if args.impl == "reference":
        return run_reference(args)
    if args.warmup < 3:
        print("warm-up must be >= 3 steps", file=sys.stderr)
        return 2
    import torch
    import paper_2407_10449_gb300 as ess
    import workloads

    global CHAIN_KERNEL
    CHAIN_KERNEL = args.chain_kernel
    world, rank, local = dist_setup(args.gpus)
    peaks = load_peaks()
    fp64_peak = measure_fp64_peak(torch)
    C = args.chains
    inst = workloads.metric(n_chains=1)
    seed = rank_seed(args.seed, rank)

    clocks = ClockSampler(local) if rank == 0 else None
    keep = ERR_SAMPLE if (not args.no_cpu and rank == 0) else 0
    ms, timing, stats, clk, lc = time_form(ess, torch, inst, "mixed", C, args.steps, args.warmup,
                                           seed, world, rank, clocks, keep=keep)
    value = job_throughput(world, C, args.steps, ms)
    if args.mixed_only:
        ms64, timing64, stats64, value64 = float("nan"), {}, {}, None
    else:
        ms64, timing64, stats64, _, lc64 = time_form(ess, torch, inst, "fp64", C,
                                                     args.fp64_steps, 3, seed, world, rank,
                                                     None, keep=keep)
        value64 = job_throughput(world, C, args.fp64_steps, ms64)
        ms64s, timing64s, stats64s, _, lc64s = time_form(ess, torch, inst, "fp64_split", C,
                                                         args.fp64_split_steps, 3, seed, world,
                                                         rank, None, keep=keep)
        value64s = job_throughput(world, C, args.fp64_split_steps, ms64s)

    if rank != 0:
        barrier(world)
        return 0

    roof = phase_rooflines(inst, C, timing, "mixed", peaks)
    roof64 = phase_rooflines(inst, C, timing64, "fp64", peaks) if timing64 else {}
    roof64s = phase_rooflines(inst, C, timing64s, "fp64_split", peaks) if timing64 else {}
    dominant = max(roof, key=lambda k: roof[k]["share"])
    dom = roof[dominant]
    kernel_src = {"gemm": ("k_gemm_tc.cu", "tc_ptx.cuh"),
                  # the counters are chain_warp_kernel's (the CTA-per-chain
                  # fallback beside it is empty at this size)
                  "chain": ("k_chain_warp.cu", "chain_warp_step.cuh", "chain_math.cuh",
                            "chain_warp_ops.cuh"),
                  "draw": ("k_draw.cu", "ess_common.cuh"), "refresh": ("k_gemm_tc.cu", "tc_ptx.cuh")}
    src = source_hash(*kernel_src[dominant])
    traffic, inst_count = ncu_counters(f"{dominant}_mixed", src)
    roofline = {"bound": dom["bound"], "kernel": dominant, "achieved": dom["achieved"],
                "peak": dom["peak"], "unit": dom["unit"], "frac": dom["frac"],
                "traffic": traffic, "work_per_launch": dom["work_per_launch"],
                "peak_source": peaks["source"] if dom["bound"] in ("hbm", "tensor") else
                FP64_PEAK_SOURCE}
    # the chain kernel against its other bound, the SM issue rate (instructions
    # counted by ncu on the current source, time live)
    if "chain" in roof:
        c_src = source_hash(*kernel_src["chain"])
        _, c_inst = ncu_counters("chain_mixed", c_src)
        iss = issue_roofline(torch, c_inst, roof["chain"]["ms_per_launch"],
                             (clk or {}).get("sm_mhz"))
        roof["chain"]["issue"] = iss
        if dominant == "chain":
            roofline["issue"] = iss
    launches = lc["gpu_launches"]

    e2e = None
    if not args.no_e2e:
        e2e = time_e2e(ess, torch, inst, C, args.steps, seed)
    cpu = None
    errors = {}
    if not args.no_cpu and world >= 1:
        cpu = cpu_baseline(lambda n: workloads.metric(n_chains=n))
        # the same leg compares the oracle's one-step map with the GPU's on
        # sampled chains of each form (angle and iterate error)
        errors["mixed"] = oracle_errors(ess, torch, inst.A, inst.b, lc["states"], "mixed", seed)
        if not args.mixed_only:
            errors["fp64"] = oracle_errors(ess, torch, inst.A, inst.b, lc64["states"], "fp64",
                                           seed)
            errors["fp64_split"] = oracle_errors(ess, torch, inst.A, inst.b, lc64s["states"],
                                                 "fp64_split", seed)
    configs = None
    if not args.no_configs and not args.mixed_only:
        configs = time_configs(ess, torch, workloads, peaks, seed, errors=not args.no_cpu)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+fp16x3", "data": "synthetic",
        "config": {"workload": "metric_d1000_m2000_c8192", "d": 1000, "m": 2000,
                   "chains_per_gpu": C, "precision": "mixed", "refresh_k": REFRESH_K,
                   "window": lc["window"],
                   "l2": "working set per step ~300 MB > 126 MB L2 (no flush needed)",
                   "parallelism": f"replicas{world}"},
        "error_vs_oracle": errors.get("mixed"),
        "fp64": None if args.mixed_only else {
            "value": value64, "unit": UNIT, "steps": args.fp64_steps,
            "ms_per_step": ms64 / args.fp64_steps, "dtype": "f64", "window": lc64["window"],
            "phases": roof64, "stats": stats64, "error_vs_oracle": errors.get("fp64"),
            "step_roofline": step_roofline(roof64, ms64 / args.fp64_steps)},
        # the FP64 form with q = A nu and p = A x from exact 56-bit splits on the
        # tensor cores (FP64-class products, ess_config.fp64_products = 1)
        "fp64_split": None if args.mixed_only else {
            "value": value64s, "unit": UNIT, "steps": args.fp64_split_steps,
            "ms_per_step": ms64s / args.fp64_split_steps, "dtype": "f64 (products: bf16 slices)",
            "window": lc64s["window"], "phases": roof64s, "stats": stats64s,
            "error_vs_oracle": errors.get("fp64_split"),
            "step_roofline": step_roofline(roof64s, ms64s / args.fp64_split_steps)},
        "roofline": roofline,
        "step_roofline": step_roofline(roof, ms / args.steps),
        "phases": roof,
        "fp64_peak": {"tflops": fp64_peak, "source": FP64_PEAK_SOURCE},
        "e2e": e2e,
        "cpu_baseline": cpu,
        "clocks": clk,
        "gpu_launches": launches,
        "graph_launches": lc["graph_launches"],
        "stats": stats,
        "configs": configs,
    }
    print(json.dumps(line), flush=True)
    barrier(world)
    return 0


if __name__ == "__main__":
    sys.exit(main())
