#!/usr/bin/env python
"""Benchmark: IADM iterations per second of the GB300 TV/L2 solver.

Workload (the single-image binary32 configuration): n = 128 (N = 16384 pixels),
m = 4915 Gaussian measurements (ratio 0.3), A = 4915 x 16384 binary32 resident
in HBM (322 MB, larger than the 129 MB L2, so no L2 flush is needed), seeded
phantom of 12 ellipses plus a rectangle grid, noise 1e-3 RMS, mu = 1e3,
beta = 10, reconstructions of 300 iterations.  A step is one IADM iteration
(one pass of rows a1-a7: multiplier update, shrink, right-hand side, FFT
u-solve, stop norms, A u - f and A^T r).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun, one independent problem per rank (no collective on
the data path; weak scaling).  `--impl reference` times the FP64 CPU oracle on
the host cores instead (a bounded sample of the same workload).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ADM iter/s and recons/s at <=1e-4 rel err vs FP64 oracle; % of HBM/tensor roofline"
ITERS_PER_RECON = 300
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "k_products_n128_m4915.json")
PRODUCTS_SRC = os.path.join(ROOT, "paper_1001_1774_gb300", "csrc", "k_products.cu")
GEMM_SUMMARY = os.path.join(ROOT, "profiles", "k_gemm_bf16x3_pair_batch256_n128_m4915.json")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30000)
    ap.add_argument("--warmup", type=int, default=300)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-solves", type=int, default=5)
    ap.add_argument("--ref-budget", type=float, default=60.0,
                    help="seconds of oracle iterations the reference arm times")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sub-records", action="store_true",
                    help="skip the short batch256 and n256 segments of the default line")
    ap.add_argument("--workload", choices=["n128", "n32", "n256", "batch256", "batch256tol", "uneven64",
                                           "dct128", "products"],
                    default="n128",
                    help="n128: 128x128, m=4915, binary32 A (the benchmark workload); "
                         "n32: 32x32, m=307, to tol 1e-4; "
                         "n256: 256x256, m=13107, A stored per --precision; "
                         "batch256: 256 images of 128x128 sharing one A (bf16 hi/lo); "
                         "uneven64: 64 problems of n in {64..192}, A regenerated in the kernel; "
                         "dct128: 128x128 with the partial-DCT encoder of Sec. 3.2, to tol 5e-5; "
                         "batch256tol: the batch256 images, each to its own tol 1e-4 (compaction); "
                         "products: the product kernel alone for --n, --m, --precision (A generated "
                         "on the device), --steps back-to-back launches (for profiler captures)")
    ap.add_argument("--images", type=int, default=256,
                    help="images of --workload batch256 (one group up to 512; more run in groups of at most 512)")
    ap.add_argument("--gemm-shape", default=None,
                    help="--workload batch256: pin both batched GEMMs to 'BLOCKS,PAIR' (e.g. 152,1 for "
                         "76 CTA pairs) instead of the tuner's pick (profiling captures)")
    ap.add_argument("--n", type=int, default=256, help="image side of --workload products")
    ap.add_argument("--m", type=int, default=13107, help="measurements of --workload products")
    ap.add_argument("--algo", choices=["iadm", "ftvcs"], default="iadm",
                    help="Algorithm 2 (IADM, default) or Algorithm 1 (FTVCS: lambda = 0, the penalty model)")
    ap.add_argument("--precision", type=int, default=0,
                    help="storage of A: 0 binary32, 1 bf16 hi+lo, 2 fp8 e4m3 + bf16 correction")
    ap.add_argument("--host-loop", action="store_true",
                    help="launch the iteration kernels from the host instead of the loop graph "
                         "(same kernels; for per-kernel profiler launch lists)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return 6800.0, "fallback 6.8 TB/s"


STORAGE = {0: ("fp32", 4), 1: ("bf16x2", 4), 2: ("fp8e4m3+bf16", 3)}


def workload_spec(workload: str, rank: int) -> dict:
    """The problem rank `rank` solves: the named single-image configuration on
    rank 0 and, on the other ranks, the same configuration with seed + rank (an
    independent problem of the same shape: weak scaling, no data exchange)."""
    if workload == "n256":
        return dict(n=256, ratio=0.2, seed=2 + rank, n_ellipses=20, mu=5e2, beta=10.0, tol=0.0,
                    max_iter=ITERS_PER_RECON, noise_c=5e-3, rect_grid=False)
    if workload == "n32":
        return dict(n=32, ratio=0.3, seed=0 + rank, n_ellipses=6, mu=1e3, beta=10.0, tol=1e-4,
                    max_iter=500, noise_c=1e-3, rect_grid=False)
    return dict(n=128, ratio=0.3, seed=1 + rank, n_ellipses=12, mu=1e3, beta=10.0, tol=0.0,
                max_iter=ITERS_PER_RECON, noise_c=1e-3, rect_grid=True)


def make_workload(args, rank):
    import synth
    sp = workload_spec(args.workload, rank)
    return synth.make_problem(sp["n"], sp["ratio"], sp["seed"], sp["n_ellipses"], sp["mu"],
                              sp["beta"], sp["tol"], sp["max_iter"], sp["noise_c"],
                              rect_grid=sp["rect_grid"], name="%s_rank%d" % (args.workload, rank))


def max_over_ranks(x: float, ws: int, device: str = "cpu") -> float:
    """The largest of the ranks' values (a time: the job ends with its slowest rank)."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(ws: int, units_per_rank: float, ms: float) -> float:
    """Units all ranks processed per second, over the slowest rank's time."""
    return ws * units_per_rank / (ms / 1e3)


def workload_config(P, A_bytes, precision=0, algo="iadm"):
    name = "n%d_m%d_%s_single_image" % (P.n, P.m, STORAGE[precision][0])
    return {"workload": name, "n": P.n, "m": P.m, "N": P.N, "A_storage": STORAGE[precision][0],
            "mu": P.mu, "beta": P.beta, "iters_per_recon": ITERS_PER_RECON,
            "A_bytes": A_bytes, "algo": algo.upper(),
            "l2": ("inputs larger than L2 (A = %.0f MB > 129 MB); no flush" % (A_bytes / 1e6)
                   if A_bytes > 129e6 else
                   "A (%.1f MB) is L2-resident: latency-bound, no roofline claim" % (A_bytes / 1e6)),
            "parallelism": "one independent problem per GPU"}


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, local_rank: int):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        idx = str(local_rank)
        if vis:
            parts = [p.strip() for p in vis.split(",") if p.strip()]
            if local_rank < len(parts):
                idx = parts[local_rank]
        self.idx = idx
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", self.idx], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        with open(self.path) as fh:
            for line in fh:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    mx.append(float(p[2]))
                except ValueError:
                    continue
                for name, val in zip(self.NAMES, p[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------- traffic summary

def traffic_from_profile(summary=PROFILE_SUMMARY, key="dram_bytes_per_launch"):
    """dram bytes per launch (or launch pair) of a kernel from its committed ncu
    summary, or None when the kernel's source changed since it was taken."""
    try:
        with open(summary) as fh:
            d = json.load(fh)
        with open(os.path.join(ROOT, d["source"]), "rb") as fh:
            sha = hashlib.sha256(fh.read()).hexdigest()
        if d.get("source_sha256") != sha:
            return None
        return float(d[key])
    except Exception:
        return None


def batch_launch_iters(iters):
    """The same for the shared-A batch, whose loop body holds 4 iterations."""
    return -(-iters // 4) * 4


def batch_launches(iters, g_in_usolve=True):
    """Kernels one shared-A batched solve launches: u^0 = A^T F (bf16 split of F, GEMM,
    fix-up, split of u^0), the first products (GEMM, fix-up, GEMM and, unless the
    u-solve adds G's partial tiles itself as it does for 128 x 128 images, G's
    fix-up), per launched iteration the u-solve, two GEMMs, one or two fix-ups and
    the condition kernel, then G formed after the loop when the loop left it in
    partial tiles (split of R, GEMM, fix-up) and the end-of-run kernels (residual,
    its norm, the two final kernels)."""
    per_iter = 5 if g_in_usolve else 6
    fixed = 4 + (3 if g_in_usolve else 4) + (3 if g_in_usolve else 0) + 4
    return per_iter * batch_launch_iters(iters) + fixed


def loop_launch_iters(iters, max_iter=None):
    """Iterations whose kernels a single-image run launches: the run's first
    16 * (max_iter // 16) iterations go through a WHILE graph of 16-iteration
    bodies and the remaining max_iter % 16 through a graph of their own.  A
    fixed-count run (max_iter = iters) launches exactly its iterations; a run
    that stopped by tol after `iters` also launches the rest of its last body
    and the final graph, whose iterations skip their work."""
    if max_iter is None or iters >= max_iter:
        return iters if max_iter is None else max_iter
    body = 16
    nb, rest = max_iter // body, max_iter % body
    if iters <= nb * body:
        return -(-iters // body) * body + rest
    return max_iter


# ----------------------------------------------------------------------------- CPU oracle sample

def oracle_sample(P, tau, budget_s=20.0, want_u=False, algo=0, max_iters=None):
    """Times the FP64 oracle (as it stands) on this host: iterations/s measured on
    a bounded number of iterations of the same workload (at most max_iters, one
    300-iteration reconstruction by default, fewer when the time budget is short)."""
    import numpy as np
    import oracle
    t0 = time.perf_counter()
    oracle.solve(P.A, P.f, P.n, P.mu, P.beta, tau, max_iter=0, algo=algo)
    t_init = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.solve(P.A, P.f, P.n, P.mu, P.beta, tau, max_iter=2, algo=algo)
    per = max((time.perf_counter() - t0 - t_init) / 2, 1e-6)
    want = ITERS_PER_RECON if max_iters is None else max(1, max_iters)
    iters = want if per * want <= budget_s else max(2, min(want, int(budget_s / per)))
    t0 = time.perf_counter()
    res = oracle.solve(P.A, P.f, P.n, P.mu, P.beta, tau, max_iter=iters, algo=algo)
    elapsed = time.perf_counter() - t0 - t_init
    return {"iters": iters, "seconds": elapsed, "value": iters / elapsed,
            "cores": oracle.num_threads(), "u": res.u if want_u else None}


# ----------------------------------------------------------------------------- our arm

def sub_records(tv, args, stream, main):
    """The other configurations of the benchmark, short: the 256-image shared-A
    batch (tensor-core GEMMs) and the 256 x 256 image with A stored as binary32,
    bf16 hi+lo and fp8 + bf16 correction (product kernels against HBM)."""
    steps = ITERS_PER_RECON   # one whole reconstruction per timed call
    out = {}
    b = batch_segment(tv, steps, 3, stream, want_parity=not args.no_cpu_baseline)
    for k in ("_A", "_F", "_mus"):
        b.pop(k)
    # against the single-image binary32 path: its 300-iteration reconstructions end
    # to end through tvcs_solve, and its device-timed iteration rate
    single_e2e = main["e2e"]["value"] / ITERS_PER_RECON
    b["vs_single_image_fp32"] = {"recons_per_s_single_e2e": single_e2e,
                                 "ratio_e2e": b["e2e"]["value"] / ITERS_PER_RECON / single_e2e,
                                 "recons_per_s_single_device": main["recons_per_s"],
                                 "ratio_device": b["recons_per_s"] / main["recons_per_s"]}
    out["batch256"] = b
    for p in (0, 1, 2):
        out["n256_" + STORAGE[p][0]] = n256_segment(tv, p, steps, stream)
    return out



def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import synth
    import __graft_entry__
    ws, rank, local = dist_env()
    dev = "cuda"
    if ws > 1:
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
        dev = "cuda" if backend == "nccl" else "cpu"
    torch.cuda.set_device(local)
    if rank == 0:
        __graft_entry__.build()
    if ws > 1:
        dist.barrier()
    import paper_1001_1774_gb300 as tv

    P = make_workload(args, rank)
    stream = torch.cuda.Stream()
    opt = tv.tvcs_default_options()
    opt.max_iter = ITERS_PER_RECON
    opt.precision = args.precision
    opt.stream = ctypes_stream(stream)
    opt.host_loop = 1 if args.host_loop else 0
    opt.algo = 1 if args.algo == "ftvcs" else 0
    with torch.cuda.stream(stream):
        A_dev = torch.from_numpy(P.A).cuda()
        f_dev = torch.from_numpy(P.f).cuda()
        u_dev = torch.empty(P.N, dtype=torch.float32, device="cuda")
    stream.synchronize()
    h = tv.tvcs_create(A_dev, 0, P.m, P.n, P.mu, P.beta, 0.0, opt)
    del A_dev
    tau = tv.tvcs_get_tau(h)
    # first reconstruction: builds the loop graph and the state
    tv.tvcs_solve(h, f_dev, u_dev)
    tv.tvcs_iterate(h, max(args.warmup, 3))

    def barrier():
        if ws > 1:
            dist.barrier()

    sampler = ClockSampler(local)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.2)
    torch.cuda.nvtx.range_push("timed")
    ev0.record(stream)
    res = tv.tvcs_iterate(h, args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    clocks = sampler.stop()
    barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1), ws, dev)
    assert res.iters == args.steps, res.iters

    # Dominant kernel (products, one pass over A, with the reduction of its
    # partials into g): launches back to back on the same stream.
    reps = 400
    k0 = torch.cuda.Event(enable_timing=True)
    k1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("products")
    k0.record(stream)
    tv.tvcs_time_stage(h, 2, reps)
    k1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    prod_us = k0.elapsed_time(k1) * 1e3 / reps
    stage_us = {"products": prod_us,
                "usolve_cluster": tv.tvcs_time_stage(h, 1, 400) * 1e3 / 400}
    # restore a clean state after the timing runs
    tv.tvcs_solve(h, f_dev, u_dev)

    # End to end through the C ABI with pinned host buffers: each call copies f in
    # and the image out and runs one 300-iteration reconstruction.
    f_host = torch.from_numpy(P.f).pin_memory()
    u_host = torch.empty(P.N, dtype=torch.float32).pin_memory()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_solves):
        r = tv.tvcs_solve(h, f_host, u_host)
        assert r.iters == ITERS_PER_RECON
    e2e_s = max_over_ranks(time.perf_counter() - t0, ws, dev)
    u_gpu = u_host.numpy().copy()
    # relative error of the reconstruction against the phantom (Sec. 3.1)
    ub = P.ubar.ravel().astype(np.float64)
    rel_err_ubar = float(np.linalg.norm(u_gpu.astype(np.float64) - ub) / np.linalg.norm(ub))

    out = None
    if rank == 0:
        peak, peak_src = hbm_peak()
        A_bytes = P.m * P.N * STORAGE[args.precision][1] + (4 * P.m if args.precision == 2 else 0)
        alg_bytes = A_bytes + 4 * (P.N + 2 * P.m)
        achieved = alg_bytes / (prod_us * 1e-6) / 1e9
        traffic = traffic_from_profile() if args.workload == "n128" else None
        value = whole_job_rate(ws, args.steps, ms)
        e2e_iters = ws * args.e2e_solves * ITERS_PER_RECON
        out = {
            "metric": METRIC, "value": value, "unit": "iter/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic (seeded phantom, Philox Gaussian A)",
            "recons_per_s": value / ITERS_PER_RECON,
            "config": workload_config(P, A_bytes, args.precision, args.algo),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": "k_products (fused A u - f and A^T r, one pass over A)",
                         "algorithmic_bytes_per_launch": alg_bytes,
                         "launch_us": prod_us, "peak_source": peak_src},
            "stage_us": stage_us,
            "e2e": {"value": e2e_iters / e2e_s, "unit": "iter/s",
                    "h2d_bytes_per_step": 4 * P.m / ITERS_PER_RECON,
                    "d2h_bytes_per_step": 4 * P.N / ITERS_PER_RECON,
                    "note": "tvcs_solve with pinned host f and u, %d reconstructions of %d iterations"
                            % (args.e2e_solves, ITERS_PER_RECON)},
            "gpu_launches": 2 * loop_launch_iters(args.steps) + 2,
            "clocks": clocks,
            "tau": tau,
            "relative_error_vs_phantom": rel_err_ubar,
        }
        if ws == 1 and not args.no_cpu_baseline:
            cb = oracle_sample(P, tau, want_u=True, algo=1 if args.algo == "ftvcs" else 0)
            out["cpu_baseline"] = {"value": cb["value"], "unit": "iter/s", "cores": cb["cores"],
                                   "kind": "oracle",
                                   "sample": "%d IADM iterations of the same workload (FP64 C "
                                             "oracle, OpenMP), %.1f s" % (cb["iters"], cb["seconds"])}
            if cb["iters"] == ITERS_PER_RECON:
                ref = cb["u"].ravel()
                err = float(np.linalg.norm(u_gpu - ref) / np.linalg.norm(ref))
                out["parity_vs_oracle"] = {"rel_image_err": err, "iters": ITERS_PER_RECON,
                                           "ok": err <= 1e-4}
            # the same oracle on one core (a bounded sample of the same workload)
            import oracle
            nthr = oracle.num_threads()
            oracle.set_num_threads(1)
            try:
                cb1 = oracle_sample(P, tau, budget_s=8.0, algo=1 if args.algo == "ftvcs" else 0)
            finally:
                oracle.set_num_threads(nthr)
            out["cpu_baseline"]["one_thread"] = {
                "value": cb1["value"], "unit": "iter/s", "cores": 1,
                "sample": "%d iterations of the same workload, %.1f s" % (cb1["iters"], cb1["seconds"])}
        if ws == 1 and args.workload == "n128" and not args.no_sub_records:
            out["sub_records"] = sub_records(tv, args, stream, out)
    tv.tvcs_destroy(h)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    if out is not None:
        print(json.dumps(out), flush=True)


def ctypes_stream(stream) -> int:
    return int(stream.cuda_stream)


# ----------------------------------------------------------------------------- sub-records

def n256_segment(tv, precision, steps, stream):
    """The 256 x 256 single-image workload (m = 13107, A generated on the device
    from its seed and stored per `precision`): the product kernel's time against
    its algorithmic bytes, and `steps` iterations of the loop."""
    import torch
    import synth
    sp = workload_spec("n256", 0)
    P = synth.make_problem(sp["n"], sp["ratio"], sp["seed"], sp["n_ellipses"], sp["mu"], sp["beta"],
                           0.0, steps, sp["noise_c"], materialise=False)
    opt = tv.tvcs_default_options()
    opt.precision = precision
    opt.max_iter = steps
    opt.stream = ctypes_stream(stream)
    h = tv.tvcs_create(None, P.seed, P.m, P.n, P.mu, P.beta, 0.0, opt)
    with torch.cuda.stream(stream):
        f = torch.from_numpy(P.f).cuda()
        u = torch.empty(P.N, dtype=torch.float32, device="cuda")
    stream.synchronize()
    tv.tvcs_solve(h, f, u)                       # state, loop graphs
    tv.tvcs_iterate(h, 3)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    tv.tvcs_iterate(h, steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    reps = 20
    prod_us = tv.tvcs_time_stage(h, 2, reps) * 1e3 / reps
    tv.tvcs_destroy(h)
    peak, peak_src = hbm_peak()
    A_bytes = P.m * P.N * STORAGE[precision][1] + (4 * P.m if precision == 2 else 0)
    alg = A_bytes + 4 * (P.N + 2 * P.m)
    achieved = alg / (prod_us * 1e-6) / 1e9
    return {"workload": "n256_m13107_%s_single_image" % STORAGE[precision][0],
            "value": steps / (ms / 1e3), "unit": "iter/s", "steps": steps,
            "recons_per_s": steps / (ms / 1e3) / ITERS_PER_RECON,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "kernel": "k_products_q<%d>" % precision,
                         "algorithmic_bytes_per_launch": alg, "launch_us": prod_us,
                         "peak_source": peak_src}}


def batch_segment(tv, steps, warmup, stream, want_parity=True, images=256, gemm_shape=None):
    """`images` (256 by default) images of 128 x 128 sharing one 4915 x 16384 A (bf16
    hi/lo): `steps` batched iterations; the GEMM pair's time against the bf16 peak;
    image 0 against the FP64 oracle after the same iterations."""
    import numpy as np
    import torch
    import synth
    B = images
    A, ubars, F, mus, _ = synth.workload_shared_batch(count=B, n=128, ratio=0.3, seed=1)
    m, N = A.shape
    opt = tv.tvcs_default_options()
    opt.precision = tv.TVCS_PREC_BF16X2
    opt.stream = ctypes_stream(stream)
    opt.max_iter = max(warmup, 3)
    with torch.cuda.stream(stream):
        A_dev = torch.from_numpy(A).cuda()
        F_dev = torch.from_numpy(F).cuda()
        U_dev = torch.empty((B, N), dtype=torch.float32, device="cuda")
    stream.synchronize()
    h = tv.tvcs_create(A_dev, 0, m, 128, 1e3, 10.0, 0.0, opt)
    del A_dev
    if gemm_shape:
        g, p = (int(v) for v in gemm_shape.split(","))
        tv.tvcs_test_gemm_shape(h, g, p, g, p)
    tau = tv.tvcs_get_tau(h)
    fl = [F_dev[b] for b in range(B)]
    ul = [U_dev[b] for b in range(B)]
    tv.tvcs_solve_batched([h] * B, fl, ul, mus)      # warm-up: A^T, plans, loop graph
    tv.tvcs_destroy(h)
    opt.max_iter = steps
    opt.tau = tau
    with torch.cuda.stream(stream):
        A_dev = torch.from_numpy(A).cuda()
    stream.synchronize()
    h = tv.tvcs_create(A_dev, 0, m, 128, 1e3, 10.0, 0.0, opt)
    del A_dev
    if gemm_shape:
        tv.tvcs_test_gemm_shape(h, g, p, g, p)
    tv.tvcs_solve_batched([h] * B, fl, ul, mus)      # state and the loop graph of this count
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.2)
    ev0.record(stream)
    res = tv.tvcs_solve_batched([h] * B, fl, ul, mus)
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    assert all(r.iters == steps for r in res)
    loop_ms = res[0].ms
    reps = 20
    gemm_us = tv.tvcs_time_stage(h, 3, reps) * 1e3 / reps
    fix_us = tv.tvcs_time_stage(h, 4, reps) * 1e3 / reps
    us_us = tv.tvcs_time_stage(h, 5, reps) * 1e3 / reps
    U0 = U_dev[0].cpu().numpy()
    # end to end with pinned host buffers (f in, images out inside the timed call)
    F_host = torch.from_numpy(F).pin_memory()
    U_host = torch.empty((B, N), dtype=torch.float32).pin_memory()
    t0 = time.perf_counter()
    tv.tvcs_solve_batched([h] * B, [F_host[b] for b in range(B)], [U_host[b] for b in range(B)], mus)
    e2e_s = time.perf_counter() - t0
    tv.tvcs_destroy(h)
    # more than 512 images run in groups of nearly equal size, the smaller ones last:
    # the stage timings above are of the last group
    groups = -(-B // 512)
    last = B // groups
    flops = 2 * 3 * 2.0 * m * N * last               # two GEMMs, three bf16 terms each
    peak = bf16_peak()
    tf = flops / (gemm_us * 1e-6) / 1e12
    value = B * steps / (ms / 1e3)
    out = {"workload": "batch%d_n128_m4915_bf16x2_shared_A" % B, "value": value,
           "unit": "image-iter/s", "steps": steps, "recons_per_s": value / ITERS_PER_RECON,
           "ms_per_step": ms / steps,
           "roofline": {"bound": "tensor", "achieved": tf, "peak": peak[0], "unit": "TFLOP/s",
                        "frac": tf / peak[0], "kernel": "the two batched GEMMs, R = A U and G = A^T R (k_gemm_bf16x3_pair on CTA pairs or k_gemm_bf16x3, the shape the tuner picks)",
                        "flops_per_iteration": flops, "launch_pair_us": gemm_us,
                        "peak_source": peak[1],
                        # dram bytes of one launch pair (both GEMMs), from the committed capture
                        # at 256 images
                        "traffic": (traffic_from_profile(GEMM_SUMMARY, "dram_bytes_per_launch_pair")
                                    if B == 256 else None)},
           "stage_us": {"gemm_pair": gemm_us, "fixups": fix_us, "usolve_batched": us_us,
                        "loop_per_iteration": loop_ms * 1e3 / steps},
           "e2e": {"value": B * steps / e2e_s, "unit": "image-iter/s",
                   "h2d_bytes_per_step": 4 * m * B / steps, "d2h_bytes_per_step": 4 * N * B / steps},
           "gpu_launches": groups * batch_launches(steps), "clocks": clocks, "tau": tau,
           "groups": groups, "_A": A, "_F": F, "_mus": mus}
    if want_parity:
        import oracle
        ref = oracle.solve(A, F[0], 128, mus[0], 10.0, tau, max_iter=steps)
        err = float(np.linalg.norm(U0 - ref.u.ravel()) / np.linalg.norm(ref.u))
        out["parity_vs_oracle"] = {"rel_image_err": err, "image": 0, "iters": steps,
                                   "ok": err <= 1e-4}
    return out


# ----------------------------------------------------------------------------- batched arm

def run_batched(args):
    """256 images of 128 x 128 sharing one 4915 x 16384 A stored as bf16 hi/lo; a
    step is one iteration of all 256 images (u-steps as one batched launch, the
    products as two tcgen05 BF16x3 GEMMs)."""
    import torch

    import synth
    import __graft_entry__
    __graft_entry__.build()
    import paper_1001_1774_gb300 as tv
    stream = torch.cuda.Stream()
    b = batch_segment(tv, args.steps, args.warmup, stream,
                      want_parity=not args.no_cpu_baseline and args.steps <= ITERS_PER_RECON,
                      images=args.images, gemm_shape=args.gemm_shape)
    A, F, mus = b.pop("_A"), b.pop("_F"), b.pop("_mus")
    m, N = A.shape
    out = {"metric": METRIC, "value": b["value"], "unit": "image-iter/s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": b["ms_per_step"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3->f32",
           "data": "synthetic (seeded phantoms, Philox Gaussian A)",
           "recons_per_s": b["recons_per_s"],
           "config": {"workload": b["workload"], "images": args.images, "n": 128,
                      "m": m, "mu": "cycling 2e2, 5e2, 1e3, 2e3", "iters_per_recon": ITERS_PER_RECON,
                      "l2": "inputs larger than L2 (A and A^T bf16 hi/lo = 644 MB); no flush"}}
    for k in ("roofline", "stage_us", "e2e", "gpu_launches", "clocks", "tau", "parity_vs_oracle"):
        if k in b:
            out[k] = b[k]
    if not args.no_cpu_baseline:
        P = synth.Problem("batch_img0", 128, m, 1, mus[0], 10.0, 0.0, args.steps, 0.0, None, A,
                          F[0])
        cb = oracle_sample(P, b["tau"], budget_s=20.0)
        out["cpu_baseline"] = {"value": cb["value"], "unit": "image-iter/s", "cores": cb["cores"],
                               "kind": "oracle",
                               "sample": "%d IADM iterations of image 0 (FP64 C oracle, OpenMP), "
                                         "%.1f s" % (cb["iters"], cb["seconds"])}
    print(json.dumps(out), flush=True)


# ----------------------------------------------------------------------------- uneven arm

# Algorithmic operations per regenerated entry of A: 32-bit integer or binary32
# operations as the generator recipe writes them (a 32x32->64 multiply is 2, a
# three-way xor 2, a fused multiply-add 1), plus the products' 3 operations.
# Philox4x32-10: 10 rounds x (4 + 4 + 2 key additions) per 4 entries = 25 per
# entry; Box-Muller per pair: uniform 4 + ln 24 + sqrt 2 + cos/sin 26 + 2
# products = 58, i.e. 29 per entry; scale, dot and update 3.  Total 57.
ALU_OPS_PER_ENTRY = 57.0


def alu_peak():
    """Entries/s at the FP32/INT32 lane rate: 152 SMs x 128 lanes x max SM clock,
    divided by the algorithmic operations per entry."""
    mhz = 2070.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            mhz = float(json.load(fh).get("sm_max_mhz", mhz))
    except Exception:
        pass
    return 152 * 128 * mhz * 1e6 / ALU_OPS_PER_ENTRY / 1e9, (
        "derived: 152 SMs x 128 lanes x %.0f MHz / %.1f ops per entry" % (mhz, ALU_OPS_PER_ENTRY))


def run_uneven(args):
    """64 independent problems (n in {64, 96, 128, 192}, m/n^2 in {0.1, 0.2, 0.3,
    0.5}), every A regenerated in the product kernel, solved together to tol 1e-4
    (<= 500 iterations) by one loop graph; compared with the same 64 solves one
    at a time on the binary32 path with A stored in HBM."""
    import numpy as np
    import torch

    import synth
    import __graft_entry__
    __graft_entry__.build()
    import paper_1001_1774_gb300 as tv
    t0 = time.perf_counter()
    probs = synth.workload_uneven(64, materialise=False)
    t_gen = time.perf_counter() - t0
    stream = torch.cuda.Stream()
    opt = tv.tvcs_default_options()
    opt.a_mode = tv.TVCS_A_REGENERATE
    opt.stream = ctypes_stream(stream)
    hs, taus = [], []
    t0 = time.perf_counter()
    for P in probs:
        opt.max_iter = P.max_iter
        h = tv.tvcs_create(None, P.seed, P.m, P.n, P.mu, P.beta, P.tol, opt)
        hs.append(h)
        taus.append(tv.tvcs_get_tau(h))
    t_create = time.perf_counter() - t0
    with torch.cuda.stream(stream):
        fs = [torch.from_numpy(P.f).cuda() for P in probs]
        us = [torch.empty(P.N, dtype=torch.float32, device="cuda") for P in probs]
    stream.synchronize()
    t0 = time.perf_counter()
    tv.tvcs_solve_batched(hs, fs, us)      # warm-up: batch state, tile tuning, loop graph, a full solve
    t_warm = time.perf_counter() - t0
    sampler = ClockSampler(0)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.2)
    ev0.record(stream)
    res = tv.tvcs_solve_batched(hs, fs, us)
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    iters = [r.iters for r in res]
    loops = max(iters)
    U_gpu = [u.cpu().numpy() for u in us]
    reps = 3
    torch.cuda.nvtx.range_push("stage6")
    prod_ms = tv.tvcs_time_stage(hs[0], 6, reps) / reps
    torch.cuda.nvtx.range_pop()
    usolve_ms = tv.tvcs_time_stage(hs[0], 7, reps) / reps
    entries = sum(P.m * P.N for P in probs)
    entries_solve = sum(P.m * P.N * it for P, it in zip(probs, iters))
    # end to end: pinned host f in, host images out, inside the timed call
    F_host = [torch.from_numpy(P.f).pin_memory() for P in probs]
    U_host = [torch.empty(P.N, dtype=torch.float32).pin_memory() for P in probs]
    t0 = time.perf_counter()
    res_e = tv.tvcs_solve_batched(hs, F_host, U_host)
    e2e_s = time.perf_counter() - t0
    for h in hs:
        tv.tvcs_destroy(h)
    # the same 64 solves one at a time, binary32 with A stored in HBM (generated from the seed)
    one_ms, agree = 0.0, 0.0
    for k, (P, tau, ug) in enumerate(zip(probs, taus, U_gpu)):
        o2 = tv.tvcs_default_options()
        o2.stream = ctypes_stream(stream)
        o2.tau = tau
        o2.max_iter = P.max_iter
        h = tv.tvcs_create(None, P.seed, P.m, P.n, P.mu, P.beta, P.tol, o2)
        u = torch.empty(P.N, dtype=torch.float32, device="cuda")
        r = tv.tvcs_solve(h, fs[k], u)
        one_ms += r.ms
        ref = u.cpu().numpy()
        agree = max(agree, float(np.linalg.norm(ref - ug) / np.linalg.norm(ref)))
        tv.tvcs_destroy(h)
    peak = alu_peak()
    achieved = entries / (prod_ms * 1e-3) / 1e9
    value = sum(iters) / (ms / 1e3)
    out = {"metric": METRIC, "value": value, "unit": "problem-iter/s", "n_gpus": 1,
           "steps": loops, "warmup": loops, "ms_per_step": ms / loops,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic (seeded phantoms; every A regenerated from its Philox seed in the kernel)",
           "recons_per_s": len(probs) / (ms / 1e3),
           "config": {"workload": "uneven64_regenerated_A", "problems": len(probs),
                      "sides": sorted({P.n for P in probs}),
                      "ratios": sorted({round(P.m / P.N, 1) for P in probs}),
                      "entries_per_product_launch": entries, "mu": 1e3, "tol": 1e-4,
                      "max_iter": 500, "iterations": {"min": min(iters), "max": loops,
                                                      "sum": sum(iters)},
                      "l2": "A is never read from memory; x, r, g slices stay in shared memory"},
           "roofline": {"bound": "alu", "achieved": achieved, "peak": peak[0], "unit": "Gentries/s",
                        "frac": achieved / peak[0], "traffic": None,
                        "kernel": "k_regen_products (+ k_regen_reduce), all 64 problems per launch",
                        "launch_ms": prod_ms, "peak_source": peak[1]},
           "stage_ms": {"regen_products_all": prod_ms, "usolves_all": usolve_ms,
                        "loop_per_iteration": res[0].ms / loops},
           "entries_per_s_over_solve": entries_solve / (ms / 1e3),
           "vs_one_at_a_time_fp32_stored": {"recons_per_s": len(probs) / (one_ms / 1e3),
                                            "seconds": one_ms / 1e3,
                                            "speedup": one_ms / ms,
                                            "max_rel_image_diff": agree},
           "e2e": {"value": sum(r.iters for r in res_e) / e2e_s, "unit": "problem-iter/s",
                   "h2d_bytes_per_step": 4 * sum(P.m for P in probs) / loops,
                   "d2h_bytes_per_step": 4 * sum(P.N for P in probs) / loops},
           "gpu_launches": (len({P.n for P in probs}) + 3) * loops + 6,
           "setup_seconds": {"inputs": t_gen, "create_64_handles": t_create, "warmup_solve": t_warm},
           "clocks": clocks}
    if not args.no_cpu_baseline:
        import oracle
        # parity on the problems the oracle finishes in seconds, at the GPU's iteration counts
        checks = []
        for P, tau, ug, it in zip(probs, taus, U_gpu, iters):
            if P.n == 64 and P.m <= 1229 and len(checks) < 3:
                A = synth.gaussian_matrix(P.seed, P.m, P.N)
                ref = oracle.solve(A, P.f, P.n, P.mu, P.beta, tau, max_iter=it)
                checks.append(float(np.linalg.norm(ug - ref.u.ravel()) / np.linalg.norm(ref.u)))
        out["parity_vs_oracle"] = {"problems": len(checks), "max_rel_image_err": max(checks),
                                   "ok": max(checks) <= 1e-4}
        # oracle speed on one n = 128 problem, scaled to the batch's mean entries per iteration
        ks = next(k for k, P in enumerate(probs) if P.n == 128)
        Ps = probs[ks]
        Ps.A = synth.gaussian_matrix(Ps.seed, Ps.m, Ps.N)
        cb = oracle_sample(Ps, taus[ks], budget_s=20.0)
        mean_entries = entries / len(probs)
        out["cpu_baseline"] = {"value": cb["value"] * Ps.m * Ps.N / mean_entries,
                               "unit": "problem-iter/s", "cores": cb["cores"], "kind": "oracle",
                               "sample": "%d IADM iterations of one n=128, m=%d problem (FP64 C "
                                         "oracle, OpenMP), %.1f s, scaled by entries of A per "
                                         "iteration to the batch mean" % (cb["iters"], Ps.m,
                                                                          cb["seconds"])}
    print(json.dumps(out), flush=True)


# ----------------------------------------------------------------------------- partial-DCT arm

def run_dct(args):
    """Sec. 3.2's partial-DCT workload: 128 x 128, 30% of the DCT coefficients,
    sigma 0.001, mu = 500, beta = 2^6, tau = 1.9, reconstructions to tol 5e-5.
    A step is one IADM iteration; each timed reconstruction runs to the
    tolerance (the same iteration count every time)."""
    import numpy as np
    import torch

    import synth
    import __graft_entry__
    __graft_entry__.build()
    import paper_1001_1774_gb300 as tv
    P = synth.workload_dct128()
    rows = P.extra["rows"]
    stream = torch.cuda.Stream()
    opt = tv.tvcs_default_options()
    opt.tau = 1.9
    opt.max_iter = P.max_iter
    opt.stream = ctypes_stream(stream)
    opt.algo = 1 if args.algo == "ftvcs" else 0
    h = tv.tvcs_create_partial_dct(rows, P.n, P.mu, P.beta, P.tol, opt)
    with torch.cuda.stream(stream):
        f_dev = torch.from_numpy(P.f).cuda()
        u_dev = torch.empty(P.N, dtype=torch.float32, device="cuda")
    stream.synchronize()
    for _ in range(max(args.warmup // 1000, 1)):
        tv.tvcs_solve(h, f_dev, u_dev)           # warm-up reconstructions (build the graph)
    nrec = 3
    sampler = ClockSampler(0)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.2)
    ev0.record(stream)
    iters = 0
    for _ in range(nrec):
        res = tv.tvcs_solve(h, f_dev, u_dev)
        iters += res.iters
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    u_gpu = u_dev.cpu().numpy()
    reps = 400
    torch.cuda.nvtx.range_push("dct_products")
    prod_us = tv.tvcs_time_stage(h, 2, reps) * 1e3 / reps
    torch.cuda.nvtx.range_pop()
    torch.cuda.nvtx.range_push("usolve")
    us_us = tv.tvcs_time_stage(h, 1, reps) * 1e3 / reps
    torch.cuda.nvtx.range_pop()
    tv.tvcs_solve(h, f_dev, u_dev)               # a clean state after the stage timing
    f_host = torch.from_numpy(P.f).pin_memory()
    u_host = torch.empty(P.N, dtype=torch.float32).pin_memory()
    t0 = time.perf_counter()
    r_e = tv.tvcs_solve(h, f_host, u_host)
    e2e_s = time.perf_counter() - t0
    tv.tvcs_destroy(h)
    n = P.n
    flops = 4 * 2.0 * n ** 3                     # four dense n x n transforms per product call
    fp32_peak = 152 * 128 * 2 * 2070e6 / 1e12    # FMA lanes x 2 FLOP x max clock, TFLOP/s
    value = iters / (ms / 1e3)
    ub = P.ubar.ravel().astype(np.float64)
    out = {"metric": METRIC, "value": value, "unit": "iter/s", "n_gpus": 1,
           "steps": iters, "warmup": max(args.warmup // 1000, 1) * res.iters,
           "ms_per_step": ms / iters, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32",
           "data": "synthetic (seeded 10-ellipse phantom, seeded DCT rows, noise 0.001)",
           "recons_per_s": nrec / (ms / 1e3),
           "config": {"workload": "dct128_m4915_partial_dct", "n": n, "m": P.m, "mu": P.mu,
                      "beta": P.beta, "tau": 1.9, "tol": P.tol, "algo": args.algo.upper(),
                      "iters_per_recon": res.iters, "reconstructions": nrec,
                      "l2": "no matrix: the encoder is four n x n transforms; everything is L2-resident"},
           "roofline": {"bound": "alu", "achieved": flops / (prod_us * 1e-6) / 1e12,
                        "peak": fp32_peak, "unit": "TFLOP/s",
                        "frac": flops / (prod_us * 1e-6) / 1e12 / fp32_peak, "traffic": None,
                        "kernel": "k_dct_products (one 16-block cluster)",
                        "note": "latency-bound: 16.8 MFLOP per launch on one 16-SM cluster "
                                "(the peak is the whole GPU's; the cluster's 16 SMs have 8.5 TFLOP/s)",
                        "launch_us": prod_us,
                        "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 FLOP x 2070 MHz"},
           "stage_us": {"dct_products": prod_us, "usolve_cluster": us_us},
           "e2e": {"value": r_e.iters / e2e_s, "unit": "iter/s",
                   "h2d_bytes_per_step": 4 * P.m / r_e.iters, "d2h_bytes_per_step": 4 * P.N / r_e.iters},
           "gpu_launches": nrec * (2 * loop_launch_iters(res.iters, P.max_iter) + 2),
           "relative_error_vs_phantom": float(np.linalg.norm(u_gpu - ub) / np.linalg.norm(ub)),
           "clocks": clocks}
    if not args.no_cpu_baseline:
        import oracle
        algo = 1 if args.algo == "ftvcs" else 0
        t0 = time.perf_counter()
        ref = oracle.solve_dct(rows, P.f, n, P.mu, P.beta, 1.9, max_iter=res.iters, algo=algo)
        el = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": res.iters / el, "unit": "iter/s", "cores": oracle.num_threads(),
                               "kind": "oracle",
                               "sample": "one reconstruction of %d iterations (FP64 C oracle, "
                                         "dense DCT matrices, OpenMP), %.1f s" % (res.iters, el)}
        err = float(np.linalg.norm(u_gpu - ref.u.ravel()) / np.linalg.norm(ref.u))
        out["parity_vs_oracle"] = {"rel_image_err": err, "iters": res.iters, "ok": err <= 1e-4}
    print(json.dumps(out), flush=True)



def run_batched_tol(args):
    """The 256 images of the shared-A batch, each run to its own eq. (stop) at tol
    1e-4 (at most 3000 iterations).  With mu cycling over 2e2 .. 2e3 the images
    stop at different iterations; the batch compacts the running images into the
    GEMMs' leading columns.  The same solve without compaction is timed beside it."""
    import numpy as np
    import torch

    import synth
    import __graft_entry__
    __graft_entry__.build()
    import paper_1001_1774_gb300 as tv
    B = 256
    A, ubars, F, mus, _ = synth.workload_shared_batch(count=B, n=128, ratio=0.3, seed=1)
    m, N = A.shape
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        A_dev = torch.from_numpy(A).cuda()
        F_dev = torch.from_numpy(F).cuda()
        U_dev = torch.empty((B, N), dtype=torch.float32, device="cuda")
    stream.synchronize()
    fl = [F_dev[b] for b in range(B)]
    ul = [U_dev[b] for b in range(B)]
    timing = {}
    tau = None
    for compact in (1, 0):
        opt = tv.tvcs_default_options()
        opt.precision = tv.TVCS_PREC_BF16X2
        opt.stream = ctypes_stream(stream)
        opt.max_iter = 3000
        opt.batch_compact = compact
        if tau is not None:
            opt.tau = tau
        h = tv.tvcs_create(A_dev, 0, m, 128, 1e3, 10.0, 1e-4, opt)
        tau = tv.tvcs_get_tau(h)
        tv.tvcs_solve_batched([h] * B, fl, ul, mus)   # warm-up: A^T, plans, the loop graph
        sampler = ClockSampler(0)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        sampler.start()
        time.sleep(0.2)
        ev0.record(stream)
        res = tv.tvcs_solve_batched([h] * B, fl, ul, mus)
        ev1.record(stream)
        torch.cuda.synchronize()
        clocks = sampler.stop()
        its = [r.iters for r in res]
        n_tol = sum(r.stopped_by_tol for r in res)
        timing[compact] = (ev0.elapsed_time(ev1), its, clocks, U_dev.cpu().numpy(), n_tol)
        if compact:
            F_host = torch.from_numpy(F).pin_memory()
            U_host = torch.empty((B, N), dtype=torch.float32).pin_memory()
            t0 = time.perf_counter()
            tv.tvcs_solve_batched([h] * B, [F_host[b] for b in range(B)],
                                  [U_host[b] for b in range(B)], mus)
            e2e_s = time.perf_counter() - t0
        tv.tvcs_destroy(h)
    ms, its, clocks, U_c, n_tol = timing[1]
    ms_full, its_full, _, U_f, _ = timing[0]
    assert its == its_full and np.array_equal(U_c, U_f), "compaction changed a result"
    its_a = np.array(its)
    value = B / (ms / 1e3)
    mean_active = its_a.sum() / its_a.max()
    out = {"metric": METRIC, "value": value, "unit": "recons/s", "n_gpus": 1,
           "steps": int(its_a.max()), "warmup": 1, "ms_per_step": ms / its_a.max(),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3->f32",
           "data": "synthetic (seeded phantoms, Philox Gaussian A)",
           "image_iter_per_s": float(its_a.sum()) / (ms / 1e3),
           "config": {"workload": "batch256tol_n128_m4915_bf16x2_shared_A", "images": B, "n": 128,
                      "m": m, "mu": "cycling 2e2, 5e2, 1e3, 2e3", "tol": 1e-4, "max_iter": 3000,
                      "iters_min_median_max": [int(its_a.min()), int(np.median(its_a)), int(its_a.max())],
                      "stopped_by_tol": int(n_tol),
                      "iters_by_mu": {str(mu): int(np.max(its_a[np.array(mus) == mu])) for mu in sorted(set(mus))},
                      "mean_active_images": mean_active,
                      "l2": "inputs larger than L2 (A and A^T bf16 hi/lo = 644 MB); no flush"},
           "compaction": {"ms": ms, "ms_without": ms_full, "speedup": ms_full / ms,
                          "results_identical": True},
           "roofline": {"bound": "tensor", "achieved": None, "peak": bf16_peak()[0], "unit": "TFLOP/s",
                        "frac": None, "traffic": None,
                        "kernel": "k_gemm_bf16x3 (columns = running images); see --workload batch256"},
           "e2e": {"value": B / e2e_s, "unit": "recons/s", "h2d_bytes_per_step": 4 * m * B / its_a.max(),
                   "d2h_bytes_per_step": 4 * N * B / its_a.max()},
           "gpu_launches": batch_launches(int(its_a.max())), "clocks": clocks, "tau": tau}
    print(json.dumps(out), flush=True)

def bf16_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["bf16_tflops"]), "measured burst (MEASURED_PEAKS.json bf16_tflops)"
    except Exception:
        return 1900.0, "fallback 1.9 PFLOP/s"


# ----------------------------------------------------------------------------- reference arm

def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    import synth
    P = make_workload(args, 0)
    tau = oracle.default_tau(P.A, 20 if args.workload == "n256" else 100)
    budget = args.ref_budget
    # warm-up: W oracle iterations at most, bounded in time
    t0 = time.perf_counter()
    oracle.solve(P.A, P.f, P.n, P.mu, P.beta, tau, max_iter=min(args.warmup, 3))
    warm = time.perf_counter() - t0
    # one step = one iteration, as in our arm; K steps when they fit the time budget
    cb = oracle_sample(P, tau, budget_s=budget, algo=1 if args.algo == "ftvcs" else 0,
                       max_iters=args.steps)
    A_bytes = P.m * P.N * 4
    value = cb["value"]
    sample = ("%d of %d requested %s iterations in one run (FP64 C oracle, OpenMP), %.1f s"
              % (cb["iters"], args.steps, args.algo.upper(), cb["seconds"]))
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "iter/s",
           "n_gpus": ws, "steps": cb["iters"], "requested_steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 / value, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded phantom, Philox Gaussian A)",
           "config": workload_config(P, A_bytes, 0, args.algo),
           "cpu_baseline": {"value": value, "unit": "iter/s", "cores": cb["cores"],
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": "iter/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0},
           "warmup_seconds": warm}
    print(json.dumps(out), flush=True)


def run_products(args):
    """The product kernel alone (rows a6-a7): A (m x n^2) generated on the device from
    seed 7 and stored per --precision, u and f set, then --steps back-to-back product
    launches timed with CUDA events.  The two launches that setting u and f makes
    come first (profiler captures skip them)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1001_1774_gb300 as tv
    n, m, prec = args.n, args.m, args.precision
    N = n * n
    opt = tv.tvcs_default_options()
    opt.precision = prec
    opt.tau = 0.1
    opt.host_loop = 1
    h = tv.tvcs_create(None, 7, m, n, 500.0, 10.0, 0.0, opt)
    g = torch.Generator(device="cuda").manual_seed(0)
    u = torch.rand(N, device="cuda", generator=g)
    f = torch.randn(m, device="cuda", generator=g)
    tv.tvcs_set_state(h, tv.TVCS_STATE_F, f)
    tv.tvcs_set_state(h, tv.TVCS_STATE_U, u)
    ms = tv.tvcs_time_stage(h, 2, args.steps)
    tv.tvcs_destroy(h)
    bpe = STORAGE[prec][1]
    alg = m * N * bpe + (4 * m if prec == 2 else 0) + 4 * (N + 2 * m)
    us = ms * 1e3 / args.steps
    peak, src = hbm_peak()
    print(json.dumps({"workload": "products_n%d_m%d_%s" % (n, m, STORAGE[prec][0]), "launches": args.steps,
                      "us_per_launch": us, "algorithmic_bytes": alg, "GB_s": alg / us / 1e3,
                      "frac_of_hbm": alg / us / 1e3 / peak, "peak_source": src}), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch256":
        run_batched(args)
    elif args.workload == "uneven64":
        run_uneven(args)
    elif args.workload == "dct128":
        run_dct(args)
    elif args.workload == "batch256tol":
        run_batched_tol(args)
    elif args.workload == "products":
        run_products(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
