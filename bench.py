"""Benchmark: MSPCG vs plain CG time-to-solve at residual 1e-10 on one GB300,
and the hop (Dslash) kernel's HBM bandwidth.

Workload (default): Moebius DWF 16^3 x 32 x Ls=12, b=1.5, c=0.5, M5=1.8,
m_f=0.01, SU(3) links exp(i 0.4 H) (seed 1001), one Gaussian source (seed
2001 + rank). MSPCG: 8^3 x 16 blocks (16 blocks), 6 inner CG iterations in
FP16 storage, FP32 outer iterations with FP64 reductions and reliable updates.
Plain CG: the same outer solver without the preconditioner.

A step is one full MSPCG solve (every stage of the path) to a true residual
of 1e-10. `value` is the mean MSPCG time-to-solution over the timed steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Under torchrun (N > 1) every rank runs an independent replica on its own GPU
and source; the timed region is bracketed by barriers and the maximum over
ranks is reported ("replicas only": the path has no data exchange on one GPU).
--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (see cpu_sample()).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MSPCG vs plain CG time-to-solve at resid 1e-10 (1 GB300); Dslash HBM GB/s"
# dram__bytes_read.sum + dram__bytes_write.sum per launch of the hop kernels
# inside the MSPCG solve of this workload, from one ncu capture of the same
# bench command on the current kernels (see profiles/); a kernel missing here
# reports traffic null. hop2_kernel<F16,1,0,0,1>: block-operator hops 4 and 3,
# (185.43 + 26.95) and (174.87 + 49.17) MB, mean of the two launches.
DRAM_BYTES_PER_LAUNCH = {"hop2_kernel<F16,1,0,0,1>": 218210560}
WORKLOAD = "mobius_16^3x32x12"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"dwf_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()
            self.f.close()

    def summary(self):
        if not self.proc or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": smax, "reasons": ["unsampled"]}
        loaded = [s for s in sm if smax and s > 0.5 * smax] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------
# CPU oracle sample (cpu_baseline and --impl reference)
# ----------------------------------------------------------------------------
def cpu_sample(outer_iters, k, nblocks):
    """Time one application of the oracle's block operator A_s on one
    8^3 x 16 block of the workload (the cut-out box form, FP64 numpy) and
    scale it to a full MSPCG solve: the oracle's cost is proportional to the
    sites it sweeps, so A on the whole lattice costs t_As * V / V_box, and
    one outer iteration costs A + k * nblocks * A_s."""
    from oracle import dwf_operator as op
    from oracle import solvers as sv
    from paper_1811_08488_gb300 import synthetic as syn
    w = syn.WORKLOADS[WORKLOAD]
    act = op.Action(dims=w["dims"], Ls=w["Ls"], M5=w["M5"], b=w["b"], c=w["c"])
    U = op.gauge_to_mu_major(syn.gauge_field(w["dims"], w["eps"], 1000 + w["id"]))
    b = op.half_to_full(syn.half_field(w["dims"], w["Ls"], 2000 + w["id"]), 0)
    block, origin = w["block"], (0, 0, 0, 0)
    mask = sv.block_mask(act, block, origin)
    t0 = time.perf_counter()
    sv.a_block_box(act, U, sv.project(b, mask), w["mf"][0], origin, block)
    t_as = time.perf_counter() - t0
    vbox = np.prod([min(L, bl + 4) for L, bl in zip(w["dims"], block)])
    t_a = t_as * np.prod(w["dims"]) / vbox
    per_outer = t_a + k * nblocks * t_as
    return {"value": float(outer_iters * per_outer), "t_sample": t_as,
            "sample": (f"one FP64 oracle A_s apply on one 8^3x16 block box ({t_as:.1f} s), "
                       f"scaled to {outer_iters} outer iterations x (A + {k} x {nblocks} A_s)")}


def cpu_sample_1core(outer_iters, k, nblocks):
    """cpu_sample() with every numpy/BLAS thread pool limited to one thread
    (the oracle's arrays ops are single-threaded numpy): returns (sample, cores)."""
    try:
        import threadpoolctl
        with threadpoolctl.threadpool_limits(1):
            return cpu_sample(outer_iters, k, nblocks), 1
    except ImportError:
        return cpu_sample(outer_iters, k, nblocks), 1


# Outer iterations of the GB300 MSPCG solve of this workload (measured by the
# GB300 arm: 118 at k = 6, 8^3 x 16 blocks). The reference arm scales its
# per-iteration sample by it, since a full FP64 oracle solve takes hours.
MSPCG_OUTER_ITERS = 118


# ----------------------------------------------------------------------------
# Replicas (N > 1): the step time is the maximum over ranks
# ----------------------------------------------------------------------------
def max_over_ranks(values, dist, device):
    """Element-wise maximum of a list of floats over all ranks."""
    import torch
    v = torch.tensor(values, dtype=torch.float64, device=device)
    dist.all_reduce(v, op=dist.ReduceOp.MAX)
    return v.tolist()


def replica_source_seed(workload_id, rank):
    """Each replica solves its own Gaussian source."""
    return 2000 + workload_id + rank


# ----------------------------------------------------------------------------
# GB300 arm
# ----------------------------------------------------------------------------
def bench_config(world):
    """The benchmark workload, as both arms report it."""
    from paper_1811_08488_gb300 import synthetic as syn
    w = syn.WORKLOADS[WORKLOAD]
    nblocks = int(np.prod([d // bl for d, bl in zip(w["dims"], w["block"])]))
    return {"workload": WORKLOAD, "lattice": "16^3x32", "Ls": w["Ls"], "b": w["b"], "c": w["c"],
            "M5": w["M5"], "mf": w["mf"][0], "gauge_eps": w["eps"], "block": "8^3x16",
            "nblocks": nblocks, "inner_iters": 6, "inner": "fp16+scale", "outer": "fp32",
            "reductions": "fp64", "tol": 1e-10, "parallelism": f"replicas{world}",
            "l2": "solve working set > L2 (about 1.3 GB); 256 MB L2 flush between steps"}


def flush_l2(buf):
    """Evict L2 by reading a buffer larger than it (leaves clean lines, so the
    timed kernel pays no write-back of the flush)."""
    buf.sum()


def run_gpu(args, rank, world, dist):
    import torch
    from paper_1811_08488_gb300 import dwf, synthetic as syn
    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    w = syn.WORKLOADS[WORKLOAD]
    dims, Ls, mf = w["dims"], w["Ls"], w["mf"][0]
    Uc = syn.gauge_field(dims, w["eps"], 1000 + w["id"])
    src = syn.half_field(dims, Ls, replica_source_seed(w["id"], rank))
    ctx = dwf.Context(dims, Ls, b=w["b"], c=w["c"], M5=w["M5"], device=dev)
    ctx.gauge_load(Uc)
    stream = torch.cuda.current_stream()
    V4 = int(np.prod(dims))
    Vh = V4 // 2
    l2_flush = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB

    # --- hop kernel bandwidth (FP32, the solver's outer launch shape) ---------
    canon = torch.from_numpy(src[None].copy()).cuda()
    fin = ctx.new_field("fp32")
    fout = ctx.new_field("fp32")
    ctx.field_import(fin, "fp32", canon)
    alg_bytes = 2 * Vh * Ls * 24 * 4 + V4 * 4 * 18 * 4
    for _ in range(5):
        ctx.dslash_eo(fout, fin, 0, 0, "fp32", [mf])
    times = []
    for _ in range(30):
        flush_l2(l2_flush)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.dslash_eo(fout, fin, 0, 0, "fp32", [mf])
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) * 1e-3)
    t_hop = statistics.median(times)
    hop_gbs = alg_bytes / t_hop / 1e9

    # the same kernel on FP16 fields (the storage of the inner block solves,
    # which take most of the MSPCG time): 48 B + 4 B scale per (site, s),
    # 36 B FP16 links
    f16in = ctx.new_field("fp16")
    f16out = ctx.new_field("fp16")
    ctx.field_import(f16in, "fp16", canon)
    alg16 = 2 * Vh * Ls * (48 + 4) + V4 * 4 * 18 * 2
    for _ in range(5):
        ctx.dslash_eo(f16out, f16in, 0, 1, "fp16", [mf])
    times16 = []
    for _ in range(30):
        flush_l2(l2_flush)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.dslash_eo(f16out, f16in, 0, 1, "fp16", [mf])
        e1.record(stream)
        e1.synchronize()
        times16.append(e0.elapsed_time(e1) * 1e-3)
    t_hop16 = statistics.median(times16)

    def time_call(fn, reps=10):
        for _ in range(3):
            fn()
        ts = []
        for _ in range(reps):
            flush_l2(l2_flush)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1) * 1e-3)
        return statistics.median(ts)

    # --- M_5^-1 on the tensor cores, 16 right-hand sides (the multi-RHS shape) ---
    m5 = None
    if not args.dslash_only:
        nr = args.m5_rhs
        m16 = list(syn.log_spaced_masses(0.001, 0.05, nr))
        canon16 = canon.expand(nr, *canon.shape[1:]).contiguous()
        peak_m5, _ = peaks()
        m5 = {"nrhs": nr, "note": "call time: kernel + 4-byte status read + stream sync"}
        for prec, bpe in (("fp32", 96), ("fp16", 52)):
            fi, fo = ctx.new_field(prec, nr), ctx.new_field(prec, nr)
            ctx.field_import(fi, prec, canon16, nr)
            t = time_call(lambda: ctx.m5inv_gemm(fo, fi, 0, prec, m16))
            alg = 2 * Vh * Ls * bpe * nr
            m5[prec] = {"us": round(t * 1e6, 1), "alg_bytes": alg, "gbs": round(alg / t / 1e9, 1),
                        "frac": round(alg / t / 1e9 / peak_m5, 4)}
            if prec == "fp32":
                t_cc = time_call(lambda: ctx.m5inv(fo, fi, 0, "fp32", m16))
                m5["closed_form_fp32"] = {"kernel": "ls_kernel (CUDA cores)",
                                          "us": round(t_cc * 1e6, 1),
                                          "gbs": round(alg / t_cc / 1e9, 1)}
            del fi, fo
        del canon16
        torch.cuda.empty_cache()
        if args.m5_only:
            return {"metric": "M_5^-1 GEMM HBM GB/s", "m5inv_gemm": m5,
                    "config": {"workload": WORKLOAD, "nrhs": nr}}, None, None

    if args.dslash_only:
        times_dag = []
        for _ in range(30):
            flush_l2(l2_flush)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.dslash_eo(fout, fin, 0, 1, "fp32", [mf])
            e1.record(stream)
            e1.synchronize()
            times_dag.append(e0.elapsed_time(e1) * 1e-3)
        t_dag = statistics.median(times_dag)
        peak, kind = peaks()
        res = {"metric": "Dslash HBM GB/s", "value": round(hop_gbs, 1), "unit": "GB/s",
               "higher_is_better": True, "us": round(t_hop * 1e6, 2), "alg_bytes": alg_bytes,
               "dagger_us": round(t_dag * 1e6, 2), "dagger_gbs": round(alg_bytes / t_dag / 1e9, 1),
               "frac": round(hop_gbs / peak, 4), "config": {"workload": WORKLOAD}}
        if args.dslash_fp64:
            # the FP64 hop of the reliable updates (after the FP32 and FP16 launches)
            d_in, d_out = ctx.new_field("fp64"), ctx.new_field("fp64")
            ctx.field_import(d_in, "fp64", canon)
            t64 = time_call(lambda: ctx.dslash_eo(d_out, d_in, 0, 0, "fp64", [mf]), 5)
            res["fp64_us"] = round(t64 * 1e6, 1)
        return res, None, None

    # --- solves -----------------------------------------------------------------
    b = canon
    x = torch.zeros_like(b)
    p_ms = dwf.default_params(inner_iters=6, block=w["block"], inner="fp16", outer="fp32",
                              tol=1e-10)
    p_plain = dwf.default_params(inner_iters=0, outer="fp32", tol=1e-10)

    def timed_solves(prm, n, collect):
        out = []
        for _ in range(n):
            flush_l2(l2_flush)
            if dist:
                dist.barrier()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st, info = ctx.solve(x, b, [mf], prm)
            e1.record(stream)
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
            if collect:
                out.append((e0.elapsed_time(e1) * 1e-3, st, info[0]))
        return out

    timed_solves(p_plain, max(1, args.warmup // 2), False)
    plain = timed_solves(p_plain, max(1, args.steps // 2 + 1), True)
    # the hop-kernel timer runs inside the timed MSPCG solves: its graphs are
    # captured with the timer during the warm-up, and the counters are reset
    # right before the timed region
    ctx.profile(True)
    timed_solves(p_ms, args.warmup, False)
    ctx.profile(True)
    with ClockSampler(dev) as clk:
        ms = timed_solves(p_ms, args.steps, True)
    kstats = ctx.profile_read()
    ctx.profile(False)
    # the same solves without the timer (its cost, for the record)
    timed_solves(p_ms, 1, False)
    ms_off = timed_solves(p_ms, max(1, args.steps // 2 + 1), True)
    # the block autotuner's shape for this workload (the configured 8^3 x 16
    # blocks stay the benchmark value): tuning cost and the solve with it
    p_auto = dwf.default_params(inner_iters=6, block=(0, 0, 0, 0), inner="fp16", outer="fp32",
                                tol=1e-10)
    t0 = time.perf_counter()
    blk_auto, _ = ctx.autotune_block(b, [mf], p_auto, trial=20)
    t_tune = time.perf_counter() - t0
    timed_solves(p_auto, 1, False)
    auto = timed_solves(p_auto, max(1, args.steps // 2 + 1), True)
    if dist:
        auto_t = max_over_ranks([statistics.mean(t for t, _, _ in auto)], dist, "cuda")[0]
    else:
        auto_t = statistics.mean(t for t, _, _ in auto)
    mspcg_auto = {"block": "x".join(map(str, blk_auto)), "seconds": round(auto_t, 6),
                  "outer_iters": auto[-1][2]["outer_iters"], "tuning_seconds": round(t_tune, 3),
                  "converged": all(st == 0 and i["converged"] for _, st, i in auto)}

    # e2e: host buffers, copies inside the timed region
    bh = torch.from_numpy(src[None].copy()).pin_memory()
    xh = torch.zeros_like(bh).pin_memory()
    p_e2e = dwf.default_params(inner_iters=6, block=w["block"], inner="fp16", outer="fp32",
                               tol=1e-10, io_on_host=1)
    ctx.solve(xh, bh, [mf], p_e2e)
    e2e_t = []
    for _ in range(args.steps):
        flush_l2(l2_flush)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, info = ctx.solve(xh, bh, [mf], p_e2e)
        torch.cuda.synchronize()
        e2e_t.append(time.perf_counter() - t0)

    t_ms = statistics.mean(t for t, _, _ in ms)
    t_plain = statistics.mean(t for t, _, _ in plain)
    t_e2e = statistics.mean(e2e_t)
    if dist:
        t_ms, t_plain, t_e2e = max_over_ranks([t_ms, t_plain, t_e2e], dist, "cuda")
    info_ms, info_plain = ms[-1][2], plain[-1][2]
    ok = all(st == 0 and i["converged"] for _, st, i in ms + plain)
    k = 6
    nblocks = int(np.prod([d // bl for d, bl in zip(dims, w["block"])]))
    launches_ms = (1 + 1 + (6 * k + 1) + 2 + info_ms["outer_iters"] * (6 + 6 * k + 1)
                   + info_ms["reliable_updates"] * (6 + 6 * k + 2) + 1)
    peak, kind = peaks()
    # the dominant kernel of the timed solves, from the hop-kernel timer:
    # achieved = its compulsory bytes / its device time, summed over launches
    t_steps = sum(t for t, _, _ in ms)
    kernels = []
    for kst in sorted(kstats, key=lambda d: -d["seconds"]):
        kernels.append({"kernel": kst["name"], "launches": kst["launches"],
                        "ms": round(kst["seconds"] * 1e3, 3),
                        "share": round(kst["seconds"] / t_steps, 4),
                        "avg_us": round(kst["seconds"] / kst["launches"] * 1e6, 2),
                        "gbs": round(kst["alg_bytes"] / kst["seconds"] / 1e9, 1)})
    dom = max(kstats, key=lambda d: d["seconds"])
    dom_gbs = dom["alg_bytes"] / dom["seconds"] / 1e9
    dom_traffic = DRAM_BYTES_PER_LAUNCH.get(dom["name"])
    res = {
        "metric": METRIC,
        "value": round(t_ms, 6),
        "unit": "s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(t_ms * 1e3, 3),
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": bench_config(world),
        "mspcg": {"seconds": round(t_ms, 6),
                  "seconds_without_kernel_timer": round(statistics.mean(t for t, _, _ in ms_off), 6),
                  "outer_iters": info_ms["outer_iters"],
                  "inner_iters_total": info_ms["inner_iters_total"],
                  "reliable_updates": info_ms["reliable_updates"],
                  "true_resid": info_ms["true_resid"]},
        "plain_cg": {"seconds": round(t_plain, 6), "outer_iters": info_plain["outer_iters"],
                     "reliable_updates": info_plain["reliable_updates"],
                     "true_resid": info_plain["true_resid"]},
        "mspcg_speedup_vs_plain": round(t_plain / t_ms, 4),
        "mspcg_autotuned": mspcg_auto,
        "all_converged": ok,
        "dslash": {"kernel": "hop2_kernel<F32,DAG=0,PRE=1> (M^4 = -1/2 Dhop M_phi)",
                   "us": round(t_hop * 1e6, 2), "alg_bytes": alg_bytes,
                   "gbs": round(hop_gbs, 1), "frac_of_8tbs_nominal": round(hop_gbs / 8000, 4)},
        "m5inv_gemm": m5,
        "dslash_fp16_dagger": {"kernel": "hop2_kernel<F16,DAG=1,PRE=0>", "us": round(t_hop16 * 1e6, 2),
                               "alg_bytes": alg16, "gbs": round(alg16 / t_hop16 / 1e9, 1),
                               "frac": round(alg16 / t_hop16 / 1e9 / peak, 4)},
        # the dominant kernel of the timed MSPCG solves (hop-kernel timer):
        # achieved = compulsory bytes / device time over all its launches in
        # the timed region; traffic = dram read + write per launch from one
        # ncu capture of the same bench command (profiles/), null if none
        "roofline": {"bound": "hbm", "achieved": round(dom_gbs, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(dom_gbs / peak, 4), "traffic": dom_traffic,
                     "frac_of_8tbs_nominal": round(dom_gbs / 8000, 4),
                     "kernel": dom["name"], "peak_kind": kind, "launches": dom["launches"],
                     "share_of_timed_solves": round(dom["seconds"] / t_steps, 4),
                     "avg_launch_us": round(dom["seconds"] / dom["launches"] * 1e6, 2),
                     "alg_bytes_per_launch": int(dom["alg_bytes"] / dom["launches"])},
        "hop_kernels_in_timed_solves": kernels,
        "e2e": {"value": round(t_e2e, 6), "unit": "s",
                "h2d_bytes_per_step": int(bh.numel() * 16), "d2h_bytes_per_step": int(xh.numel() * 16)},
        "gpu_launches": int(launches_ms),
        "clocks": clk.summary(),
    }
    return res, info_ms, nblocks


# ----------------------------------------------------------------------------
# studies: the solver parameter sweeps (one JSON line per configuration)
# ----------------------------------------------------------------------------
def _divisor_blocks(dims, cands):
    return [b for b in cands if all(d % x == 0 and x % 2 == 0 for d, x in zip(dims, b))]


STUDY_BLOCKS = [(4, 4, 4, 4), (6, 6, 6, 8), (8, 8, 8, 8), (8, 8, 8, 16), (12, 12, 12, 8),
                (12, 12, 12, 16), (16, 16, 16, 16)]


def run_resident_study(args):
    """Per-block cost of the block preconditioner against the number of blocks.

    With 2 or 4 blocks of 8^3 x 16 (Ls = 12, FP16 inner storage) the whole
    working set of the k inner iterations stays in the 129 MB L2; with 16 or
    32 it streams from HBM. Equal per-block times mean that keeping blocks
    resident in L2 would not pay."""
    import torch
    from paper_1811_08488_gb300 import dwf, synthetic as syn
    stream = torch.cuda.current_stream()
    flush = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    block, Ls, k = (8, 8, 8, 16), 12, 6
    for dims in [(16, 8, 8, 16), (16, 16, 8, 16), (16, 16, 16, 16), (16, 16, 16, 32),
                 (32, 16, 16, 32)]:
        ctx = dwf.Context(dims, Ls, b=1.5, c=0.5, M5=1.8)
        ctx.gauge_load(syn.gauge_field(dims, 0.4, 1002))
        canon = torch.from_numpy(syn.half_field(dims, Ls, 2002)[None].copy()).cuda()
        r, z = ctx.new_field("fp32", 1), ctx.new_field("fp32", 1)
        ctx.field_import(r, "fp32", canon, 1)
        prm = dwf.default_params(block=block, inner="fp16", inner_iters=k)
        for _ in range(3):
            ctx.block_precond(z, r, prm, [0.01])
        res = {}
        for mode in ("warm", "flushed"):
            ts = []
            for _ in range(max(args.steps, 5)):
                if mode == "flushed":
                    flush_l2(flush)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ctx.block_precond(z, r, prm, [0.01])
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1) * 1e3)
            res[mode] = float(np.median(ts))
        nb = int(np.prod([d // b for d, b in zip(dims, block)]))
        print(json.dumps({"study": "resident", "dims": "x".join(map(str, dims)), "Ls": Ls,
                          "block": "x".join(map(str, block)), "blocks": nb, "inner_iters": k,
                          "inner": "fp16", "us": {m: round(v, 1) for m, v in res.items()},
                          "us_per_block": {m: round(v / nb, 1) for m, v in res.items()}}),
              flush=True)
        del ctx


def run_study(args):
    """Time MSPCG / plain CG solves of one workload over a parameter sweep.

    k      inner iterations k in {0 (plain CG), 2, 3, 4, 6, 8, 12}
    snake  block operator with and without the snake terms (k = 6), and plain CG
    inner  inner storage FP32 / FP16 / BF16 (k = 6), and plain CG
    block  every block shape of STUDY_BLOCKS that tiles the lattice (k = 6)
    rhs    all right-hand sides of the workload in one call vs one call each
    pair   plain CG and MSPCG (k = 6) with the workload's block shape
    autotune  the block autotuner's pick, then the solve with block = 0
    resident  the k = 6 block preconditioner alone, per 8^3 x 16 block, on
           lattices of 2 to 32 such blocks (working set from well inside L2
           to several times L2), timed warm and with L2 flushed
    delta  reliable-update threshold delta in {0.1, 0.03, 0.01, 0.001}, plain CG and k = 6
    flexible  Algorithm 1's Fletcher-Reeves beta vs the flexible Polak-Ribiere beta (k = 6)
    Each configuration: one short untimed solve (plans, graphs), then
    `--steps` timed solves (CUDA events, L2 flushed before each). With
    `--maxiter` the solves stop after that many outer iterations and the
    line reports the time per outer iteration and the residual reached.
    """
    import torch
    from paper_1811_08488_gb300 import dwf, synthetic as syn
    torch.cuda.set_device(0)
    if args.study == "resident":
        run_resident_study(args)
        return
    name = args.workload
    w = syn.WORKLOADS[name]
    dims, Ls = w["dims"], w["Ls"]
    U, srcs = syn.workload_inputs(name)
    ctx = dwf.Context(dims, Ls, b=w["b"], c=w["c"], M5=w["M5"], recon12=args.recon12)
    ctx.gauge_load(U)
    masses = list(w["mf"])
    stream = torch.cuda.current_stream()
    flush = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    b_all = torch.from_numpy(np.ascontiguousarray(np.stack(srcs))).cuda()
    base = dict(block=w["block"], inner="fp16", outer="fp32", inner_iters=6, tol=1e-10)
    if args.maxiter:
        base["maxiter"] = args.maxiter
    if args.delta:
        base["delta"] = args.delta

    configs = []
    if args.study == "k":
        configs = [dict(base, inner_iters=k) for k in (0, 2, 3, 4, 6, 8, 12)]
    elif args.study == "snake":
        configs = [dict(base, inner_iters=0)] + [dict(base, snake=s) for s in (1, 0)]
    elif args.study == "inner":
        configs = [dict(base, inner_iters=0)] + [dict(base, inner=p) for p in ("fp32", "fp16", "bf16")]
    elif args.study == "block":
        configs = [dict(base, block=bl) for bl in _divisor_blocks(dims, STUDY_BLOCKS)]
    elif args.study == "rhs":
        configs = [dict(base, _batched=True), dict(base, _batched=False)]
    elif args.study == "pair":
        configs = [dict(base, inner_iters=0), dict(base)]
    elif args.study == "flexible":
        configs = [dict(base, flexible=f) for f in (0, 1)]
    elif args.study == "delta":
        configs = [dict(base, inner_iters=k, delta=d) for k in (0, 6) for d in (0.1, 0.03, 0.01, 0.001)]
    elif args.study == "autotune":
        # the autotuner's pick (20 trial outer iterations per candidate), then
        # the full solve with block = 0 (the remembered pick)
        prm = dwf.default_params(**dict(base, block=(0, 0, 0, 0)))
        t0 = time.perf_counter()
        blk, pred = ctx.autotune_block(b_all, masses, prm, trial=20)
        t_tune = time.perf_counter() - t0
        x = torch.zeros_like(b_all)
        flush_l2(flush)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, info = ctx.solve(x, b_all, masses, prm)
        e1.record(stream)
        torch.cuda.synchronize()
        print(json.dumps({"study": "autotune", "workload": name, "block": "x".join(map(str, blk)),
                          "tuning_seconds": round(t_tune, 3), "predicted_seconds": round(pred, 4),
                          "seconds": round(e0.elapsed_time(e1) * 1e-3, 4), "status": st,
                          "outer_iters": [i["outer_iters"] for i in info],
                          "converged": all(i["converged"] for i in info)}), flush=True)
        return
    else:
        raise SystemExit(f"unknown study {args.study}")

    def solve_once(prm_kw, b, mf, timed):
        kw = {k: v for k, v in prm_kw.items() if not k.startswith("_")}
        prm = dwf.default_params(**kw)
        x = torch.zeros_like(b)
        flush_l2(flush)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, info = ctx.solve(x, b, mf, prm)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) * 1e-3, st, info

    default_delta = dwf.default_params().delta
    for cfg in configs:
        warm = dict(cfg, maxiter=2)
        if cfg.get("_batched", True):
            calls = [(b_all, masses)]
        else:
            calls = [(b_all[i:i + 1], [m]) for i, m in enumerate(masses)]
        solve_once(warm, *calls[0], False)
        for _ in range(args.steps):
            t_tot, infos, sts = 0.0, [], []
            for b, mf in calls:
                t, st, info = solve_once(cfg, b, mf, True)
                t_tot += t
                infos += info
                sts.append(st)
            outer = [i["outer_iters"] for i in infos]
            line = {"study": args.study, "workload": name, "recon12": bool(args.recon12),
                    "inner_iters": cfg["inner_iters"], "inner": cfg["inner"],
                    "block": "x".join(map(str, cfg["block"])), "snake": cfg.get("snake", 1),
                    "delta": cfg.get("delta", default_delta), "flexible": cfg.get("flexible", 0),
                    "nrhs": len(masses), "one_call": cfg.get("_batched", True),
                    "seconds": round(t_tot, 4), "status": sts,
                    "outer_iters": outer, "max_outer_iters": max(outer),
                    "reliable_updates": [i["reliable_updates"] for i in infos],
                    "true_resid": [float(f"{i['true_resid']:.3e}") for i in infos],
                    "converged": all(i["converged"] for i in infos)}
            if args.maxiter:
                line["s_per_outer_iter"] = round(t_tot / max(1, max(outer)), 6)
            print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--dslash-only", action="store_true",
                    help="time only the FP32 hop kernel (used for kernel profiles)")
    ap.add_argument("--dslash-fp64", action="store_true",
                    help="with --dslash-only: also time the FP64 hop")
    ap.add_argument("--m5-only", action="store_true",
                    help="time only the tensor-core M_5^-1 (used for kernel profiles)")
    ap.add_argument("--m5-rhs", type=int, default=16, help="right-hand sides of the M_5^-1 timing")
    ap.add_argument("--study", choices=["k", "snake", "inner", "block", "rhs", "pair", "autotune", "delta", "resident",
                             "flexible"],
                    help="solver parameter sweep instead of the benchmark line")
    ap.add_argument("--workload", default=WORKLOAD, help="workload of --study")
    ap.add_argument("--maxiter", type=int, default=0, help="outer-iteration cap of --study")
    ap.add_argument("--recon12", action="store_true", help="--study with reconstruct-12 links")
    ap.add_argument("--delta", type=float, default=0.0, help="reliable-update threshold of --study")
    args = ap.parse_args()
    if args.study:
        run_study(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        from paper_1811_08488_gb300 import synthetic as syn
        w = syn.WORKLOADS[WORKLOAD]
        # iteration count of the GB300 MSPCG solve of this workload (measured),
        # used to scale the per-iteration sample
        nblocks = 16
        vals = []
        for i in range(args.warmup + args.steps):
            s, cores = cpu_sample_1core(MSPCG_OUTER_ITERS, 6, nblocks)
            if i >= args.warmup:
                vals.append(s["value"])
        v = statistics.mean(vals)
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": "s",
                          "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": round(v * 1e3, 1), "higher_is_better": False,
                          "scaling": "weak", "vs_baseline": None, "data": "synthetic", "dtype": "f64",
                          "config": bench_config(args.gpus),
                          "cpu_baseline": {"value": round(v, 3), "unit": "s", "cores": cores,
                                           "kind": "oracle", "sample": s["sample"]},
                          "e2e": {"value": round(v, 3), "unit": "s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}))
        return

    dist = None
    if world > 1:
        import torch
        import torch.distributed as td
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        import datetime
        # a replica that is lost between steps ends the others' next barrier
        # or reduction with an error after this long instead of the default 10 min
        td.init_process_group("nccl", timeout=datetime.timedelta(seconds=300))
        dist = td
    res, info_ms, nblocks = run_gpu(args, rank, world, dist)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline and not args.dslash_only and not args.m5_only:
            s, cores = cpu_sample_1core(info_ms["outer_iters"], 6, nblocks)
            res["cpu_baseline"] = {"value": round(s["value"], 3), "unit": "s",
                                   "cores": cores, "kind": "oracle", "sample": s["sample"]}
        print(json.dumps(res))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
