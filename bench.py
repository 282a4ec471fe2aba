"""Benchmark: MSPCG vs plain CG time-to-solve at residual 1e-10 on one GB300,
and the hop (Dslash) kernel's HBM bandwidth.

Headline workload: Moebius DWF 24^3 x 64 x Ls=16, b=1.5, c=0.5, M5=1.8,
m_f=0.003, SU(3) links exp(i 0.45 H) (seed 1002), one Gaussian source (seed
2002 + rank). MSPCG: 12^3 x 16 blocks (32 blocks), 6 inner CG iterations in
FP16 storage, FP32 outer iterations with FP64 reductions and reliable updates.
Plain CG: the same outer solver without the preconditioner. This is the
largest workload whose solves fit the benchmark's step count in a few minutes
(one MSPCG solve of the 32^3 x 64 x 12 workload with 4 right-hand sides takes
about a minute); that workload is measured once per solver as an extra key.

A step is one full MSPCG solve (every stage of the path) to a true residual
of 1e-10. `value` is the mean MSPCG time-to-solution over the timed steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Under torchrun (N > 1) every rank runs an independent replica on its own GPU
and source; the timed region is bracketed by barriers and the maximum over
ranks is reported ("replicas only": the path has no data exchange on one GPU).
--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (see reference_sample()).
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import hashlib
import json
import multiprocessing as mp
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MSPCG vs plain CG time-to-solve at resid 1e-10 (1 GB300); Dslash HBM GB/s"
WORKLOAD = "mobius_24^3x64x16"          # headline
LARGE = "mobius_32^3x64x12_4rhs"        # extra key: one timed solve per solver
SMALL = "mobius_16^3x32x12"             # extra key: the 16^3 x 32 x 12 solves
MULTI = "mobius_16^3x32x12_16rhs"       # tensor-core M_5^-1 with 16 right-hand sides
INNER_K = 6

# Outer iterations of the GB300 MSPCG solve of the headline workload (k = 6,
# 12^3 x 16 blocks), recorded from the GB300 arm. The reference arm cannot
# solve the workload (hours of CPU time), so it scales its sample by this
# count and says so; the GB300 arm's own cpu_baseline uses the count it
# measured in the same run.
MSPCG_OUTER_ITERS_RECORDED = 192

# dram__bytes_read.sum + dram__bytes_write.sum per launch of the dominant kernel
# of the timed MSPCG solves, from one ncu capture of the headline workload;
# valid only while the hop kernel sources hash to `source_sha` (otherwise the
# line reports traffic null).
KNOWN_TRAFFIC = {
    # one-pass ncu capture of 4 launches inside the timed solve of the bench
    # command (profiles/hop_fp16_block_adjoint_mobius_24x24x24x64_Ls16.md):
    # dram__bytes_read.sum + dram__bytes_write.sum, mean per launch
    "hop2_kernel<F16,1,0,0,1> [block]": {"bytes": 1799313536, "source_sha": "a5428b9e50878f1d"},
}
HOP_SOURCES = ["paper_1811_08488_gb300/csrc/hop.cu", "paper_1811_08488_gb300/csrc/device_common.cuh",
               "paper_1811_08488_gb300/csrc/dwf_internal.cuh"]


def hop_source_sha() -> str:
    h = hashlib.sha256()
    for p in HOP_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def nsites5(name):
    from paper_1811_08488_gb300 import synthetic as syn
    w = syn.WORKLOADS[name]
    return int(np.prod(w["dims"])) // 2 * w["Ls"]


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
# CPU oracle: measured timings (cpu_baseline) and the reference arm's sample
# ----------------------------------------------------------------------------
def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


ONE_THREAD_ENV = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def one_thread():
    """Limit numpy's BLAS thread pools to one thread (threadpoolctl when it is
    installed; the worker processes also start with the thread-count variables
    set to 1). The oracle's elementwise numpy arithmetic is single-threaded."""
    try:
        import threadpoolctl
        return threadpoolctl.threadpool_limits(1)
    except ImportError:
        import contextlib
        return contextlib.nullcontext()


def _oracle_inputs(name):
    from oracle import dwf_operator as op
    from paper_1811_08488_gb300 import synthetic as syn
    w = syn.WORKLOADS[name]
    act = op.Action(dims=w["dims"], Ls=w["Ls"], M5=w["M5"], b=w["b"], c=w["c"])
    Uc = syn.gauge_field(w["dims"], w["eps"], 1000 + w["id"])
    src = syn.half_field(w["dims"], w["Ls"], 2000 + w["id"])
    return w, act, Uc, src


def oracle_block_inputs(name):
    from oracle import dwf_operator as op
    w, act, Uc, src = _oracle_inputs(name)
    return w, act, op.gauge_to_mu_major(Uc), op.half_to_full(src, 0)


def oracle_block_sample(name, block, inputs=None):
    """Seconds of one oracle A_s application (the box form, FP64 numpy) on the
    block at the origin of workload `name`, and the 5D sites of its box."""
    from oracle import solvers as sv
    w, act, U, x = inputs or oracle_block_inputs(name)
    mask = sv.block_mask(act, block, (0, 0, 0, 0))
    t0 = time.perf_counter()
    sv.a_block_box(act, U, sv.project(x, mask), w["mf"][0], (0, 0, 0, 0), block)
    t = time.perf_counter() - t0
    box = int(np.prod([sv.box_extent(L, b) for L, b in zip(w["dims"], block)])) // 2 * w["Ls"]
    return t, box


def oracle_one_core_jobs():
    """The oracle's single-core measurements (run in a worker process while the
    GPU part of the benchmark runs; numpy's arithmetic here is single-threaded):
    * a full FP64 plain-CG solve of the Shamir 8^4 x 8 workload to 1e-10;
    * one A = D_PC^+ D_PC application on the 16^3 x 32 x 12 lattice;
    * one A_s application on a 6^3 x 8 block box of the headline workload."""
    from oracle import dwf_operator as op
    from oracle import solvers as sv
    out = {}
    with one_thread():
        w, act, Uc, src = _oracle_inputs("shamir_8^4x8")
        U = op.gauge_to_mu_major(Uc)
        b = op.half_to_full(src, 0)
        t0 = time.perf_counter()
        _, it, res = sv.cg(lambda v: op.mdagm(act, U, v, w["mf"][0]), b, 1e-10)
        out["c1_plain_cg"] = {"seconds": time.perf_counter() - t0, "iters": it, "true_resid": res}
        w, act, Uc, src = _oracle_inputs(SMALL)
        U = op.gauge_to_mu_major(Uc)
        x = op.half_to_full(src, 0)
        t0 = time.perf_counter()
        op.mdagm(act, U, x, w["mf"][0])
        out["c2_A"] = {"seconds": time.perf_counter() - t0, "sites5": nsites5(SMALL)}
        t, box = oracle_block_sample(WORKLOAD, (6, 6, 6, 8))
        out["headline_As_box"] = {"seconds": t, "sites5": box, "block": "6^3x8"}
    return out


def oracle_all_cores_A():
    """One A application on the 16^3 x 32 x 12 lattice with every host core:
    the oracle evaluates A in time slabs in worker processes (oracle/slabs.py)."""
    from oracle import dwf_operator as op
    from oracle import slabs
    w, act, Uc, src = _oracle_inputs(SMALL)
    n = os.cpu_count() or 1
    t0 = time.perf_counter()
    slabs.mdagm_half(act, Uc, src, w["mf"][0], slab=4, workers=n)
    return {"seconds": time.perf_counter() - t0, "cores": n}


def extrapolate(t_site_A, t_site_As, name, block, outer_iters, k=INNER_K):
    """Oracle seconds of one solve of `name`: per outer iteration one A on the
    lattice plus k A_s on every block's box, each scaled from a measured
    per-5D-site cost."""
    from oracle import solvers as sv
    from paper_1811_08488_gb300 import synthetic as syn
    w = syn.WORKLOADS[name]
    nblocks = int(np.prod([d // b for d, b in zip(w["dims"], block)]))
    box = int(np.prod([sv.box_extent(L, b) for L, b in zip(w["dims"], block)])) // 2 * w["Ls"]
    per_outer = t_site_A * nsites5(name) + k * nblocks * t_site_As * box
    return outer_iters * per_outer, per_outer


def cpu_baseline(one_core, all_cores, outer_ms, outer_plain):
    """The oracle as it stands on this host's cores (measured), and the
    headline solve extrapolated from those measurements by the GPU arm's
    iteration counts of this run."""
    from paper_1811_08488_gb300 import synthetic as syn
    block = syn.WORKLOADS[WORKLOAD]["block"]
    t_A = one_core["c2_A"]["seconds"] / one_core["c2_A"]["sites5"]
    t_As = one_core["headline_As_box"]["seconds"] / one_core["headline_As_box"]["sites5"]
    ms, _ = extrapolate(t_A, t_As, WORKLOAD, block, outer_ms)
    plain = outer_plain * t_A * nsites5(WORKLOAD)
    return {"value": round(ms, 1), "unit": "s", "cores": 1, "kind": "oracle",
            "value_is": "extrapolated: measured per-site oracle costs x the GB300 arm's outer "
                        "iterations of this run",
            "sample": (f"measured on 1 core: one A on 16^3x32x12 ({one_core['c2_A']['seconds']:.1f} s), "
                       f"one A_s on a 6^3x8 block box of {WORKLOAD} "
                       f"({one_core['headline_As_box']['seconds']:.1f} s); scaled per 5D site to "
                       f"{outer_ms} MSPCG outer iterations x (A + {INNER_K} x nblocks x A_s on "
                       f"12^3x16 block boxes)"),
            "plain_cg_extrapolated_s": round(plain, 1),
            "measured": {
                "shamir_8^4x8_plain_cg_fp64": {
                    "1_core": {"seconds": round(one_core["c1_plain_cg"]["seconds"], 2),
                               "iters": one_core["c1_plain_cg"]["iters"],
                               "true_resid": one_core["c1_plain_cg"]["true_resid"]},
                    "all_cores": "same as 1 core: the oracle's numpy arithmetic is single-threaded"},
                "A_16^3x32x12": {"1_core_s": round(one_core["c2_A"]["seconds"], 2),
                                 "all_cores_s": round(all_cores["seconds"], 2) if all_cores else None,
                                 "all_cores": all_cores["cores"] if all_cores else None},
                "A_s_6^3x8_box_of_headline": {"1_core_s": round(one_core["headline_As_box"]["seconds"], 2)},
            },
            "host": {"nproc": os.cpu_count(), "cpu": cpu_model(), "machine": platform.machine()}}


def reference_sample(inputs):
    """One step of the reference arm: one oracle A_s application on a 6^3 x 8
    block box of the headline workload on one core (measured), scaled per 5D
    site to the headline MSPCG solve with the recorded GB300 outer-iteration
    count. `inputs` (oracle_block_inputs) are drawn once, outside the steps."""
    with one_thread():
        t, box = oracle_block_sample(WORKLOAD, (6, 6, 6, 8), inputs)
    from paper_1811_08488_gb300 import synthetic as syn
    block = syn.WORKLOADS[WORKLOAD]["block"]
    per_site = t / box
    total, per_outer = extrapolate(per_site, per_site, WORKLOAD, block, MSPCG_OUTER_ITERS_RECORDED)
    return t, total


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
    return {"workload": WORKLOAD, "lattice": "24^3x64", "Ls": w["Ls"], "b": w["b"], "c": w["c"],
            "M5": w["M5"], "mf": w["mf"][0], "gauge_eps": w["eps"], "block": "12^3x16",
            "nblocks": nblocks, "inner_iters": INNER_K, "inner": "fp16+scale", "outer": "fp32",
            "reductions": "fp64", "tol": 1e-10, "parallelism": f"replicas{world}",
            "l2": "solve working set > L2 (about 10 GB); 256 MB L2 flush between steps"}


def flush_l2(buf):
    """Evict L2 by reading a buffer larger than it (leaves clean lines, so the
    timed kernel pays no write-back of the flush)."""
    buf.sum()


class Timer:
    def __init__(self, stream, flush):
        self.stream, self.flush = stream, flush

    def call(self, fn, reps=20, warm=3):
        """Median device time of fn() (CUDA events on the launching stream, L2
        flushed before each repetition)."""
        import torch
        for _ in range(warm):
            fn()
        ts = []
        for _ in range(reps):
            flush_l2(self.flush)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            fn()
            e1.record(self.stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1) * 1e-3)
        return statistics.median(ts)

    def solves(self, ctx, x, b, masses, prm, n, dist=None, defl=None):
        """n solves, each bracketed by (barrier +) synchronize and CUDA events;
        defl = (V, lambda, coarse): mspcg_solve_deflated."""
        import torch
        out = []
        for _ in range(n):
            flush_l2(self.flush)
            if dist:
                dist.barrier()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            if defl is None:
                st, info = ctx.solve(x, b, masses, prm)
            else:
                st, info = ctx.solve_deflated(x, b, masses, prm, *defl)
            e1.record(self.stream)
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
            out.append((e0.elapsed_time(e1) * 1e-3, st, info))
        return out


def dslash_line(ctx, T, canon, mf, prec, dagger, nrhs=1):
    """One hop launch (dwf_dslash_eo, even output) on native fields of `prec`:
    device time, compulsory bytes (every input and output element once, the
    links of both parities once) and their ratio."""
    fin, fout = ctx.new_field(prec, nrhs), ctx.new_field(prec, nrhs)
    ctx.field_import(fin, prec, canon, nrhs)
    V4 = int(np.prod(ctx.dims))
    eb = {"fp32": 96, "fp16": 52, "bf16": 52, "fp64": 192}[prec]
    lb = {"fp32": 72, "fp16": 36, "bf16": 36, "fp64": 144}[prec]
    alg = 2 * (V4 // 2) * ctx.Ls * eb * nrhs + V4 * 4 * lb
    masses = [mf] * nrhs
    t = T.call(lambda: ctx.dslash_eo(fout, fin, 0, dagger, prec, masses))
    peak, kind = peaks()
    del fin, fout
    return {"us": round(t * 1e6, 2), "alg_bytes": alg, "gbs": round(alg / t / 1e9, 1),
            "frac": round(alg / t / 1e9 / peak, 4), "frac_of_8tbs_nominal": round(alg / t / 8e12, 4)}


def kernel_table(kstats, t_steps):
    rows = []
    for k in sorted(kstats, key=lambda d: -d["seconds"]):
        rows.append({"kernel": k["name"], "launches": k["launches"], "ms": round(k["seconds"] * 1e3, 3),
                     "share": round(k["seconds"] / t_steps, 4),
                     "avg_us": round(k["seconds"] / k["launches"] * 1e6, 2),
                     "gbs": round(k["alg_bytes"] / k["seconds"] / 1e9, 1)})
    return rows


def run_gpu(args, rank, world, dist):
    import torch
    from paper_1811_08488_gb300 import dwf, synthetic as syn
    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    T = Timer(stream, torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device="cuda"))  # 256 MB
    peak, peak_kind = peaks()
    res = {}

    # --- headline workload ------------------------------------------------------
    w = syn.WORKLOADS[WORKLOAD]
    dims, Ls, mf = w["dims"], w["Ls"], w["mf"][0]
    Uc = syn.gauge_field(dims, w["eps"], 1000 + w["id"])
    src = syn.half_field(dims, Ls, replica_source_seed(w["id"], rank))
    ctx = dwf.Context(dims, Ls, b=w["b"], c=w["c"], M5=w["M5"], device=dev)
    ctx.gauge_load(Uc)
    del Uc
    b = torch.from_numpy(src[None]).cuda()
    x = torch.zeros_like(b)

    # the hop kernel on this lattice (fields ~10x L2): the "Dslash HBM GB/s"
    dsl = dslash_line(ctx, T, b, mf, "fp32", 0)
    dsl["kernel"] = "hop2_kernel<F32,0,1,0,0> (M^4 = -1/2 Dhop M_phi, M_phi on load)"
    dsl_dag = dslash_line(ctx, T, b, mf, "fp32", 1)
    dsl16 = dslash_line(ctx, T, b, mf, "fp16", 1)

    loop = dict(use_graph=0) if args.eager else {}
    p_ms = dwf.default_params(inner_iters=INNER_K, block=w["block"], inner="fp16", outer="fp32",
                              tol=1e-10, **loop)
    p_plain = dwf.default_params(inner_iters=0, outer="fp32", tol=1e-10, **loop)
    T.solves(ctx, x, b, [mf], p_plain, max(1, args.warmup // 2), dist)
    plain = T.solves(ctx, x, b, [mf], p_plain, max(1, args.steps // 2 + 1), dist)
    # the hop-kernel timer runs inside the timed MSPCG solves: its graphs are
    # captured with the timer during the warm-up, and the counters are reset
    # right before the timed region
    ctx.profile(True)
    T.solves(ctx, x, b, [mf], p_ms, args.warmup, dist)
    ctx.profile(True)
    with ClockSampler(dev) as clk:
        torch.cuda.nvtx.range_push("mspcg_timed")  # the range profilers select
        ms = T.solves(ctx, x, b, [mf], p_ms, args.steps, dist)
        torch.cuda.nvtx.range_pop()
    kstats = ctx.profile_read()
    ctx.profile(False)
    ms_off = T.solves(ctx, x, b, [mf], p_ms, 1, dist)

    # e2e: host buffers, copies inside the timed region (the solve copies b in
    # and x out through mspcg_solve's io_on_host path)
    bh = torch.from_numpy(src[None]).pin_memory()
    xh = torch.zeros_like(bh).pin_memory()
    p_e2e = dwf.default_params(inner_iters=INNER_K, block=w["block"], inner="fp16", outer="fp32",
                               tol=1e-10, io_on_host=1)
    ctx.solve(xh, bh, [mf], p_e2e)
    e2e_t = []
    for _ in range(max(1, min(args.steps, 3))):
        flush_l2(T.flush)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, info = ctx.solve(xh, bh, [mf], p_e2e)
        torch.cuda.synchronize()
        e2e_t.append(time.perf_counter() - t0)
    h2d, d2h = int(bh.numel() * 16), int(xh.numel() * 16)
    del bh, xh, b, x
    ctx.close()
    torch.cuda.empty_cache()

    t_ms = statistics.mean(t for t, _, _ in ms)
    t_plain = statistics.mean(t for t, _, _ in plain)
    t_e2e = statistics.mean(e2e_t)
    if dist:
        t_ms, t_plain, t_e2e = max_over_ranks([t_ms, t_plain, t_e2e], dist, "cuda")
    info_ms, info_plain = ms[-1][2][0], plain[-1][2][0]
    ok = all(st == 0 and i[0]["converged"] for _, st, i in ms + plain)
    t_steps = sum(t for t, _, _ in ms)
    dom = max(kstats, key=lambda d: d["seconds"])
    dom_gbs = dom["alg_bytes"] / dom["seconds"] / 1e9
    known = KNOWN_TRAFFIC.get(dom["name"])
    sha = hop_source_sha()
    dom_traffic = known["bytes"] if known and known["source_sha"] == sha else None
    nblocks = int(np.prod([d // bl for d, bl in zip(dims, w["block"])]))
    hop_launches = sum(k["launches"] for k in kstats)
    # BLAS / gather / scatter launches per outer iteration besides the hops:
    # outer axpy_xr, xpay_p; inner gather, scatter, k x (xr) + (k - 1) x p
    blas_per_iter = 2 + 2 + INNER_K + (INNER_K - 1)
    launches = hop_launches + args.steps * (info_ms["outer_iters"] * blas_per_iter +
                                            info_ms["reliable_updates"] * (4 + blas_per_iter) + 8)
    res.update({
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
                  "seconds_without_kernel_timer": round(ms_off[0][0], 6),
                  "outer_iters": info_ms["outer_iters"],
                  "inner_iters_total": info_ms["inner_iters_total"],
                  "reliable_updates": info_ms["reliable_updates"],
                  "true_resid": info_ms["true_resid"],
                  "dslash_gbs": round(info_ms["dslash_gbs"], 1)},
        "plain_cg": {"seconds": round(t_plain, 6), "outer_iters": info_plain["outer_iters"],
                     "reliable_updates": info_plain["reliable_updates"],
                     "true_resid": info_plain["true_resid"]},
        "mspcg_speedup_vs_plain": round(t_plain / t_ms, 4),
        "all_converged": ok,
        "dslash": dsl,
        "dslash_fp32_dagger": dsl_dag,
        "dslash_fp16_dagger": dsl16,
        # the dominant kernel of the timed MSPCG solves (hop-kernel timer):
        # achieved = compulsory bytes / device time over all its launches in
        # the timed region; traffic = dram read + write per launch from one ncu
        # capture of this workload on the same kernel sources, else null
        "roofline": {"bound": "hbm", "achieved": round(dom_gbs, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(dom_gbs / peak, 4), "traffic": dom_traffic,
                     "frac_of_8tbs_nominal": round(dom_gbs / 8000, 4),
                     "kernel": dom["name"], "peak_kind": peak_kind, "launches": dom["launches"],
                     "share_of_timed_solves": round(dom["seconds"] / t_steps, 4),
                     "avg_launch_us": round(dom["seconds"] / dom["launches"] * 1e6, 2),
                     "alg_bytes_per_launch": int(dom["alg_bytes"] / dom["launches"]),
                     "hop_source_sha": sha},
        "hop_kernels_in_timed_solves": kernel_table(kstats, t_steps),
        "e2e": {"value": round(t_e2e, 6), "unit": "s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
    })

    if not args.headline_only:
        res["small"] = run_small(args, T, rank, dist)
        if not args.no_large:
            res["large"] = run_large(args, T, rank, dist)
    return res, info_ms, info_plain


def m5_timings(ctx, T, b, dims, Ls, nr):
    """dwf_m5inv_gemm (tensor cores) on nr right-hand sides (the first nr
    log-spaced masses of the 16-rhs workload) in FP32 and FP16, and the
    CUDA-core closed form dwf_m5inv in FP32; b: one canonical source."""
    from paper_1811_08488_gb300 import synthetic as syn
    masses = list(syn.WORKLOADS[MULTI]["mf"])[:nr]
    canon = b[:1].expand(nr, *b.shape[1:]).contiguous()
    peak, _ = peaks()
    m5 = {"nrhs": nr, "note": "call time: kernel + 4-byte status read + stream sync"}
    Vh = int(np.prod(dims)) // 2
    for prec, bpe in (("fp32", 96), ("fp16", 52)):
        fi, fo = ctx.new_field(prec, nr), ctx.new_field(prec, nr)
        ctx.field_import(fi, prec, canon, nr)
        t = T.call(lambda: ctx.m5inv_gemm(fo, fi, 0, prec, masses), reps=10)
        alg = 2 * Vh * Ls * bpe * nr
        m5[prec] = {"us": round(t * 1e6, 1), "alg_bytes": alg, "gbs": round(alg / t / 1e9, 1),
                    "frac": round(alg / t / 1e9 / peak, 4)}
        if prec == "fp32":
            t_cc = T.call(lambda: ctx.m5inv(fo, fi, 0, "fp32", masses), reps=10)
            m5["closed_form_fp32"] = {"kernel": "ls_kernel (CUDA cores)", "us": round(t_cc * 1e6, 1),
                                      "gbs": round(alg / t_cc / 1e9, 1)}
        del fi, fo
    return m5


def deflation_timings(ctx, T, x, b, w, dist, n_ev=24):
    """Low modes of A (dwf_eig_lowmodes: n_ev wanted, m = n_ev + 8, Chebyshev
    degree 30, Ritz residuals <= 1e-5 lambda_max, seeded start vectors), then
    plain CG and MSPCG deflated with them (start and coarse correction), three
    timed solves each after an untimed two-iteration call."""
    import torch
    from paper_1811_08488_gb300 import dwf, synthetic as syn
    dims, Ls, mf = w["dims"], w["Ls"], float(w["mf"][0])
    m = n_ev + 8
    V = ctx.new_field("fp32", m)
    rs = ctx.field_bytes("fp32", 1)
    for b0 in range(0, m, 16):
        k = min(16, m - b0)
        start = torch.from_numpy(np.stack([syn.half_field(dims, Ls, 5000 + b0 + j)
                                           for j in range(k)])).cuda()
        ctx.field_import(V[b0 * rs:(b0 + k) * rs], "fp32", start, k)
        del start
    prm_e = dwf.default_eig_params(n_ev=n_ev, degree=30, max_passes=60, tol=1e-5)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    theta, resid, einfo = ctx.eig_lowmodes(V, m, mf, prm_e)
    t_eig = time.perf_counter() - t0
    out = {"n_ev": n_ev, "m": m, "degree": 30,
           "eig_seconds_wall": round(t_eig, 3), "eig_passes": einfo["passes"],
           "eig_matvecs": einfo["matvecs"], "eig_converged": bool(einfo["converged"]),
           "gap_theta_n_ev_over_theta_n_ev_minus_1": round(float(theta[n_ev] / theta[n_ev - 1]), 3)}
    defl = (V[:n_ev * rs], theta[:n_ev], True)
    for name, kw in (("plain_cg_deflated", dict(inner_iters=0)),
                     ("mspcg_deflated", dict(inner_iters=INNER_K, block=w["block"]))):
        T.solves(ctx, x, b, [mf], dwf.default_params(tol=1e-10, maxiter=2, **kw), 1, dist, defl)
        r = T.solves(ctx, x, b, [mf], dwf.default_params(tol=1e-10, **kw), 3, dist, defl)
        out[name] = {"seconds": round(statistics.mean(t for t, _, _ in r), 6),
                     "outer_iters": r[-1][2][0]["outer_iters"],
                     "converged": all(st == 0 and i[0]["converged"] for _, st, i in r)}
    del V
    return out


def run_small(args, T, rank, dist):
    """The 16^3 x 32 x 12 workload: MSPCG (configured and autotuned blocks) and
    plain CG, the tensor-core M_5^-1 with 16 right-hand sides, and the
    deflated solves with 24 low modes."""
    import torch
    from paper_1811_08488_gb300 import dwf, synthetic as syn
    w = syn.WORKLOADS[SMALL]
    dims, Ls, mf = w["dims"], w["Ls"], w["mf"][0]
    ctx = dwf.Context(dims, Ls, b=w["b"], c=w["c"], M5=w["M5"],
                      device=int(os.environ.get("LOCAL_RANK", 0)))
    ctx.gauge_load(syn.gauge_field(dims, w["eps"], 1000 + w["id"]))
    b = torch.from_numpy(syn.half_field(dims, Ls, replica_source_seed(w["id"], rank))[None]).cuda()
    x = torch.zeros_like(b)
    out = {"workload": SMALL, "dslash": dslash_line(ctx, T, b, mf, "fp32", 0)}
    for name, prm in (("plain_cg", dwf.default_params(inner_iters=0, tol=1e-10)),
                      ("mspcg", dwf.default_params(inner_iters=INNER_K, block=w["block"], tol=1e-10))):
        T.solves(ctx, x, b, [mf], prm, 1, dist)
        r = T.solves(ctx, x, b, [mf], prm, 3, dist)
        out[name] = {"seconds": round(statistics.mean(t for t, _, _ in r), 6),
                     "outer_iters": r[-1][2][0]["outer_iters"],
                     "converged": all(st == 0 and i[0]["converged"] for _, st, i in r)}
    p_auto = dwf.default_params(inner_iters=INNER_K, block=(0, 0, 0, 0), tol=1e-10)
    t0 = time.perf_counter()
    blk, _ = ctx.autotune_block(b, [mf], p_auto, trial=20)
    t_tune = time.perf_counter() - t0
    T.solves(ctx, x, b, [mf], p_auto, 1, dist)
    r = T.solves(ctx, x, b, [mf], p_auto, 3, dist)
    out["mspcg_autotuned"] = {"block": "x".join(map(str, blk)), "tuning_seconds": round(t_tune, 3),
                              "seconds": round(statistics.mean(t for t, _, _ in r), 6),
                              "outer_iters": r[-1][2][0]["outer_iters"],
                              "converged": all(st == 0 and i[0]["converged"] for _, st, i in r)}
    # tensor-core M_5^-1, 16 right-hand sides of log-spaced masses (one call)
    out["m5inv_gemm_16rhs"] = m5_timings(ctx, T, b, dims, Ls, len(syn.WORKLOADS[MULTI]["mf"]))
    out["deflation"] = deflation_timings(ctx, T, x, b, w, dist)
    del b, x
    ctx.close()
    torch.cuda.empty_cache()
    return out


def run_large(args, T, rank, dist):
    """The 32^3 x 64 x 12 workload with 4 right-hand sides (m_f 0.0008): the
    hop kernel on fields ~20x L2, and one timed solve per solver (all four
    right-hand sides in one call) after an untimed two-iteration solve that
    builds the plans and graphs."""
    import torch
    from paper_1811_08488_gb300 import dwf, synthetic as syn
    w = syn.WORKLOADS[LARGE]
    dims, Ls, masses = w["dims"], w["Ls"], list(w["mf"])
    ctx = dwf.Context(dims, Ls, b=w["b"], c=w["c"], M5=w["M5"],
                      device=int(os.environ.get("LOCAL_RANK", 0)))
    ctx.gauge_load(syn.gauge_field(dims, w["eps"], 1000 + w["id"]))
    srcs = [syn.half_field(dims, Ls, replica_source_seed(w["id"], rank) + r) for r in range(len(masses))]
    b = torch.from_numpy(np.stack(srcs)).cuda()
    del srcs
    x = torch.zeros_like(b)
    out = {"workload": LARGE, "dslash": dslash_line(ctx, T, b[:1], masses[0], "fp32", 0)}
    for name, kw in (("plain_cg", dict(inner_iters=0)),
                     ("mspcg", dict(inner_iters=INNER_K, block=w["block"]))):
        T.solves(ctx, x, b, masses, dwf.default_params(tol=1e-10, maxiter=2, **kw), 1, dist)
        r = T.solves(ctx, x, b, masses, dwf.default_params(tol=1e-10, **kw), 1, dist)
        t, st, info = r[0]
        out[name] = {"seconds": round(t, 4), "outer_iters": [i["outer_iters"] for i in info],
                     "true_resid": [float(f"{i['true_resid']:.3e}") for i in info],
                     "converged": st == 0 and all(i["converged"] for i in info)}
    out["mspcg_speedup_vs_plain"] = round(out["plain_cg"]["seconds"] / out["mspcg"]["seconds"], 4)
    del b, x
    ctx.close()
    torch.cuda.empty_cache()
    return out


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


def run_deflation_study(args):
    """Low modes and deflated solves on one workload (one mass, `--nrhs`
    seeded sources): the eigensolver's time, then plain CG and MSPCG (k = 6)
    without deflation, with the deflated start only, and with the start plus
    the coarse correction; every solve call takes all sources at once and is
    timed with CUDA events after an untimed two-iteration call, L2 flushed."""
    import torch
    from paper_1811_08488_gb300 import dwf, synthetic as syn
    name = args.workload
    w = syn.WORKLOADS[name]
    dims, Ls = w["dims"], w["Ls"]
    mf = float(w["mf"][0])
    U, _ = syn.workload_inputs(name)
    ctx = dwf.Context(dims, Ls, b=w["b"], c=w["c"], M5=w["M5"])
    ctx.gauge_load(U)
    stream = torch.cuda.current_stream()
    flush = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    n_ev = args.n_ev
    m = min(dwf.MAX_EIG, n_ev + max(8, n_ev // 4))
    V = ctx.new_field("fp32", m)
    rs = ctx.field_bytes("fp32", 1)
    for b0 in range(0, m, 16):
        k = min(16, m - b0)
        start = torch.from_numpy(np.stack([syn.half_field(dims, Ls, 5000 + b0 + j)
                                           for j in range(k)])).cuda()
        ctx.field_import(V[b0 * rs:(b0 + k) * rs], "fp32", start, k)
        del start
    prm_e = dwf.default_eig_params(n_ev=n_ev, degree=args.degree, max_passes=60, tol=args.eig_tol)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    theta, resid, einfo = ctx.eig_lowmodes(V, m, mf, prm_e)
    t_eig = time.perf_counter() - t0
    print(json.dumps({"study": "deflate", "workload": name, "step": "eig_lowmodes", "m": m,
                      "n_ev": n_ev, "degree": args.degree, "tol": args.eig_tol,
                      "seconds": round(t_eig, 3), **einfo,
                      "theta_over_lambda_max": [float(f"{t / einfo['lambda_max']:.4e}")
                                                for t in theta[:n_ev + 1]],
                      "max_resid_over_lambda_max": float(f"{resid[:n_ev].max() / einfo['lambda_max']:.3e}")}),
          flush=True)
    srcs = np.stack([syn.half_field(dims, Ls, 6000 + r) for r in range(args.nrhs)])
    b = torch.from_numpy(srcs).cuda()
    masses = [mf] * args.nrhs
    Vd = V[:n_ev * rs]
    if args.vprec != "fp32":
        Vd = ctx.new_field(args.vprec, n_ev)
        ctx.field_convert(Vd, args.vprec, V, "fp32", n_ev)
    lam = theta[:n_ev]

    def timed(fn):
        flush_l2(flush)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) * 1e-3, out

    for k in (0, INNER_K):
        base = dict(block=w["block"], inner="fp16", outer="fp32", inner_iters=k, tol=1e-10)
        if args.eager:
            base["use_graph"] = 0
        for mode in ("none", "start", "coarse"):
            def call(maxiter=None):
                prm = dwf.default_params(**dict(base, **({"maxiter": maxiter} if maxiter else {})))
                x = torch.zeros_like(b)
                if mode == "none":
                    return ctx.solve(x, b, masses, prm, raise_on_error=False)
                return ctx.solve_deflated(x, b, masses, prm, Vd, lam, coarse=mode == "coarse",
                                          vprec=args.vprec, raise_on_error=False)
            call(maxiter=2)
            for _ in range(args.steps):
                t, (st, info) = timed(call)
                print(json.dumps({"study": "deflate", "workload": name, "solver":
                                  "plain_cg" if k == 0 else f"mspcg_k{k}", "deflation": mode,
                                  "vprec": args.vprec,
                                  "n_ev": n_ev, "nrhs": args.nrhs, "seconds": round(t, 4),
                                  "status": st, "outer_iters": [i["outer_iters"] for i in info],
                                  "true_resid": [float(f"{i['true_resid']:.3e}") for i in info],
                                  "converged": all(i["converged"] for i in info)}), flush=True)


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
    delta  reliable-update threshold delta in {0.1, 0.03, 0.01, 0.001, 0.0001}, plain CG and k = 6
    flexible  Algorithm 1's Fletcher-Reeves beta vs the flexible Polak-Ribiere beta (k = 6)
    deflate  low modes (dwf_eig_lowmodes) and deflated plain CG / MSPCG solves
    m5     M_5^-1 on --nrhs right-hand sides: tensor cores (FP32, FP16) and CUDA cores
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
    if args.study == "deflate":
        run_deflation_study(args)
        return
    if args.study == "m5":
        # M_5^-1 on the 16^3x32 x Ls=12 lattice for --nrhs right-hand sides
        w = syn.WORKLOADS[SMALL]
        ctx = dwf.Context(w["dims"], w["Ls"], b=w["b"], c=w["c"], M5=w["M5"])
        b = torch.from_numpy(syn.half_field(w["dims"], w["Ls"], 2002)[None].copy()).cuda()
        flush = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
        T = Timer(torch.cuda.current_stream(), flush)
        print(json.dumps({"study": "m5", "workload": SMALL,
                          **m5_timings(ctx, T, b, w["dims"], w["Ls"], args.nrhs)}), flush=True)
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
    if args.eager:
        base["use_graph"] = 0
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
        configs = [dict(base, inner_iters=k, delta=d) for k in (0, 6)
                   for d in (0.1, 0.03, 0.01, 0.001, 0.0001)]
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
    ap.add_argument("--headline-only", action="store_true",
                    help="only the headline workload (no 16^3x32 and 32^3x64 extra keys)")
    ap.add_argument("--no-large", action="store_true", help="skip the 32^3x64x12 extra key")
    ap.add_argument("--eager", action="store_true",
                    help="host-driven outer loop with eager launches (use_graph = 0), for "
                         "profilers that select kernels by launch")
    ap.add_argument("--study", choices=["k", "snake", "inner", "block", "rhs", "pair", "autotune", "delta",
                                        "resident", "flexible", "deflate", "m5"],
                    help="solver parameter sweep instead of the benchmark line")
    ap.add_argument("--workload", default=SMALL, help="workload of --study")
    ap.add_argument("--maxiter", type=int, default=0, help="outer-iteration cap of --study")
    ap.add_argument("--recon12", action="store_true", help="--study with reconstruct-12 links")
    ap.add_argument("--delta", type=float, default=0.0, help="reliable-update threshold of --study")
    ap.add_argument("--n-ev", type=int, default=24, help="low modes of --study deflate")
    ap.add_argument("--degree", type=int, default=30, help="Chebyshev degree of --study deflate")
    ap.add_argument("--eig-tol", type=float, default=1e-5, help="Ritz residual tolerance of --study deflate")
    ap.add_argument("--nrhs", type=int, default=4, help="sources of --study deflate / m5")
    ap.add_argument("--vprec", default="fp32", choices=["fp32", "fp16"],
                    help="storage of the low modes in the deflated solves of --study deflate")
    args = ap.parse_args()
    if args.study:
        run_study(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        steps, vals = [], []
        inputs = oracle_block_inputs(WORKLOAD)
        for i in range(args.warmup + args.steps):
            t, v = reference_sample(inputs)
            if i >= args.warmup:
                steps.append(t)
                vals.append(v)
        v = statistics.mean(vals)
        nb = bench_config(1)["nblocks"]
        sample = (f"per step: one FP64 oracle A_s application on a 6^3x8 block box of {WORKLOAD} on "
                  f"1 core ({statistics.mean(steps):.1f} s, measured), scaled per 5D site to one MSPCG "
                  f"solve: {MSPCG_OUTER_ITERS_RECORDED} outer iterations (the GB300 arm's recorded "
                  f"count) x (A + {INNER_K} x {nb} A_s on 12^3x16 block boxes)")
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": round(v, 1), "unit": "s",
                          "value_is": "extrapolated from the measured sample (ms_per_step is the "
                                      "sample's own time)",
                          "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": round(statistics.mean(steps) * 1e3, 1),
                          "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
                          "data": "synthetic", "dtype": "f64", "config": bench_config(args.gpus),
                          "cpu_baseline": {"value": round(v, 1), "unit": "s", "cores": 1,
                                           "kind": "oracle", "sample": sample},
                          "e2e": {"value": round(v, 1), "unit": "s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}))
        return

    # the oracle's single-core measurements run in a worker process (started
    # with "spawn" before the first GPU call) while the GPU part runs
    pool, fut = None, None
    want_cpu = world == 1 and not args.no_cpu_baseline
    if want_cpu:
        saved = {k: os.environ.get(k) for k in ONE_THREAD_ENV}
        os.environ.update({k: "1" for k in ONE_THREAD_ENV})
        pool = cf.ProcessPoolExecutor(1, mp_context=mp.get_context("spawn"))
        fut = pool.submit(oracle_one_core_jobs)
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v

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
    res, info_ms, info_plain = run_gpu(args, rank, world, dist)
    if rank == 0:
        if want_cpu:
            one = fut.result()
            pool.shutdown()
            all_c = oracle_all_cores_A()
            res["cpu_baseline"] = cpu_baseline(one, all_c, info_ms["outer_iters"],
                                               info_plain["outer_iters"])
        print(json.dumps(res))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
