#!/usr/bin/env python3
"""Throughput of the dense tableau simplex on GB300: pivots/s and tableau GB/s.

Workload (one step): four seeded synthetic dense LPs shaped like the paper's
Sec. 4 problems, all FP64 and solved to optimality --
  2048 x 2048 primal form (max c'x, Ax <= b),
  2048 x 2048 dual form (min b'y, A'y >= c, by the dual simplex),
  512 x 4096 and 4096 x 512 primal form (more variables than constraints and
  the reverse).
A entries uniform integers in [1, 1000], b in [1000, 100000], c in [1, 100].

`value` is pivots per second over the whole job, device-timed with CUDA
events on the library's stream, inputs resident in HBM before the timed
region (lp_load copies them device to device and builds the tableau inside
it).  L2 is flushed (256 MiB write) between steps, outside the step's events.
`e2e` is the same metric through the C ABI from pinned host buffers:
lp_load from host memory, lp_solve, lp_result into host memory, wall clock.
"""
import argparse
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD_NAME = ("dense LP set: 2048x2048 primal + 2048x2048 dual form + 512x4096 + 4096x512, "
                 "FP64, Dantzig pricing")
# the same shapes from the paper's own random family (Sec. 4): density 0.9,
# real-valued data, about 25 times the pivots of the integer family
PAPER_WORKLOAD_NAME = ("paper-family LP set: 2048x2048 primal + 2048x2048 dual form + 512x4096 + "
                       "4096x512, density 0.9, FP64, Dantzig pricing")
FP64_DFMA_PER_CLK_SM = 2          # GB300 FP64 rate: 1.25 TFLOP/s nominal = 2 DFMA/clk/SM
SMS, SM_MAX_MHZ = 152, 2070.0
HBM_NOMINAL_GBS = 7900.0          # GB300 HBM3e nominal
ALU_PEAK_TFLOPS = 2 * FP64_DFMA_PER_CLK_SM * SMS * SM_MAX_MHZ * 1e6 / 1e12
MAX_LE, MIN_GE = 0, 1
KERNEL_SRC = os.path.join(ROOT, "paper_1804_04737_gb300", "csrc", "gbs_pipe.cu")


def workload(seed, family="dense"):
    from paper_1804_04737_gb300 import lpgen
    gen = lpgen.dense_lp if family == "dense" else lpgen.paper_lp
    out = []
    A, b, c = gen(2048, 2048, seed)
    out.append(("2048x2048 primal", A, b, c, MAX_LE))
    out.append(("2048x2048 dual form", *lpgen.dual_of(A, b, c), MIN_GE))
    out.append(("512x4096 primal", *gen(512, 4096, seed), MAX_LE))
    out.append(("4096x512 primal", *gen(4096, 512, seed), MAX_LE))
    return out


def tableau_bytes(m, n, w=8):
    """Algorithmic bytes of one pivot: the rank-1 update reads and writes the
    whole (m+1) x (n+m+1) tableau once (Sec. 2 Step 5)."""
    return 2 * (m + 1) * (n + m + 1) * w


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# The kernel each LP of the set runs on (default options): primal LPs below
# 2^19 tableau elements on the pipelined primal kernel in place, larger ones
# on the two-pivots-per-pass kernel (double-buffered), the dual form on the
# two-pivots-per-pass dual simplex kernel (double-buffered).
INPLACE_KERNEL = "pivot_pipe_kernel<double> (in place)"
BLOCK_KERNEL = "pivot_block_kernel<double> (two pivots per pass)"
DUAL_KERNEL = "pivot_block_dual_kernel<double> (dual simplex, two pivots per pass)"
# (the in-place kernel runs no LP of the default set, so it has no record)
TRAFFIC_FILES = {
    BLOCK_KERNEL: os.path.join(ROOT, "profiles", "pivot_block_kernel_fp64_traffic.txt"),
    DUAL_KERNEL: os.path.join(ROOT, "profiles", "pivot_block_dual_kernel_fp64_traffic.txt"),
}


def kernel_of(m, n, sense):
    if sense != MAX_LE:
        return DUAL_KERNEL
    pitch = (n + m + 1 + 31) // 32 * 32
    return INPLACE_KERNEL if (m + 1) * pitch < 2 ** 19 else BLOCK_KERNEL


def kernel_traffic(name):
    """Mean DRAM bytes per launch of one kernel in one bench step, from the
    committed ncu summary, or None when there is none or the kernel source
    changed since that capture."""
    import hashlib
    try:
        rec = {}
        with open(TRAFFIC_FILES[name]) as f:
            for line in f:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    rec[k.strip()] = v.strip()
        sha = hashlib.sha256(open(KERNEL_SRC, "rb").read()).hexdigest()[:16]
        if rec.get("kernel_source_sha256_16") != sha:
            return None
        return float(rec["dram_bytes_per_launch"])
    except Exception:
        return None


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons while timing."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", "gbs_clocks_%d_%d.csv" % (os.getpid(), index))

    def __enter__(self):
        self.skip = 0
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            # nvidia-smi takes a while to start: wait for its first sample, so
            # that the samples kept (those after it) fall inside the timed region
            t0 = time.time()
            while time.time() - t0 < 5.0 and self.proc.poll() is None:
                with open(self.path) as g:
                    self.skip = sum(1 for _ in g)
                if self.skip:
                    break
                time.sleep(0.01)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc:
            return {"error": "nvidia-smi unavailable"}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if len(rows) > self.skip:
            rows = rows[self.skip:]  # the samples taken while the region ran
        if not rows:
            return {"error": "no samples"}
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None,
                "sm_max_mhz": float(rows[0][2]) if rows[0][2].replace(".", "").isdigit() else None,
                "samples": len(rows), "reasons": reasons}


def reduce_over_ranks(dist, maxes, sums, device="cpu"):
    """Max of `maxes` and sum of `sums` over the ranks of the default process
    group (identity without one).  Replicas: every rank runs its own solves,
    so whole-job throughput is the units of all ranks over the slowest rank's
    time."""
    if dist is None:
        return list(maxes), list(sums)
    import torch
    a = torch.tensor(list(maxes), dtype=torch.float64, device=device)
    b = torch.tensor(list(sums), dtype=torch.float64, device=device)
    dist.all_reduce(a, op=dist.ReduceOp.MAX)
    dist.all_reduce(b, op=dist.ReduceOp.SUM)
    return a.tolist(), b.tolist()


def cpu_oracle_run(lps, threads, cap=None):
    """Pivots and seconds of the oracle on the whole workload, each LP stopped
    after `cap` pivots when given."""
    import oracle
    oracle.set_threads(threads)
    pivots = 0
    t0 = time.perf_counter()
    for _, A, b, c, sense in lps:
        r = oracle.solve(A, b, c, sense=sense, max_iters=cap if cap else 10 ** 12)
        assert r.status == (oracle.ITER_LIMIT if cap and r.iters == cap else oracle.OPTIMAL)
        pivots += r.iters
    return pivots, time.perf_counter() - t0


def run_reference(args, rank, world):
    """The FP64 oracle (the paper's method as plain C, OpenMP over the rows of
    Step 5) on the host cores, same workload, metric and units."""
    if rank != 0:
        return
    cores = len(os.sched_getaffinity(0))
    lps = workload(0)
    for _ in range(args.warmup):
        cpu_oracle_run(lps, cores)
    piv = 0
    sec = 0.0
    for _ in range(args.steps):
        p, t = cpu_oracle_run(lps, cores)
        piv += p
        sec += t
    v = piv / sec
    line = {"impl": "reference", "metric": "pivots/s", "value": v, "unit": "pivots/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sec / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME, "seed": 0},
            "cpu_baseline": {"value": v, "unit": "pivots/s", "cores": cores, "kind": "oracle",
                             "sample": "the whole workload (4 LPs) per step"},
            "e2e": {"value": v, "unit": "pivots/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_lp8192(args, capi, torch):
    """8192 x 8192 dense LP: FP64 against the FP32 tableau with FP64
    reinversion every k in {50, 200} pivots.  The FP64 path is bit-identical
    to the FP64 oracle at this size (tests/test_gpu_parity.py), so FP32
    objective errors are measured against it."""
    from paper_1804_04737_gb300 import lpgen
    A, b, c = lpgen.dense_lp(8192, 8192, 0)
    dA, db, dc = (torch.from_numpy(v).cuda() for v in (A, b, c))
    torch.cuda.synchronize()
    out = []
    ref = None
    for prec, k in ((capi.LP_FP64, 0), (capi.LP_FP32_REINV, 50), (capi.LP_FP32_REINV, 200)):
        h = capi.lp_create(capi.lp_options_default(precision=prec, reinv_k=max(k, 1)))
        best = None
        for rep in range(1 + max(1, args.steps // 5)):
            t0 = time.perf_counter()
            capi.lp_load(h, dA, db, dc)
            capi.lp_solve(h)
            obj, st, it = capi.lp_result(h)
            wall = time.perf_counter() - t0
            kms, launches = capi.lp_kernel_time(h)
            if rep and (best is None or wall < best[0]):
                best = (wall, kms, launches, obj, st, it)
        capi.lp_destroy(h)
        wall, kms, launches, obj, st, it = best
        w = 8 if prec == capi.LP_FP64 else 4
        if ref is None:
            ref = obj
        out.append({"mode": "fp64" if prec == capi.LP_FP64 else "fp32+reinv k=%d" % k,
                    "status": capi.STATUS_NAMES[st], "pivots": it,
                    "solve_ms": round(1e3 * wall, 2), "pivot_kernel_ms": round(kms, 2),
                    "pivot_kernel_launches": launches,
                    "pivots_per_s": round(it / wall, 1),
                    "tableau_gbs_kernel": round(it * tableau_bytes(8192, 8192, w) / kms / 1e6, 1),
                    # two pivots per pass over the tableau at this size: the
                    # tableau traffic is half the algorithmic bytes, and FP64 is
                    # bound by the FMA rate (one FMA per element and pivot)
                    "tflops_kernel": round(it * 2 * 8193 * 16385 / kms / 1e9, 4),
                    "fp64_alu_frac": (round(it * 2 * 8193 * 16385 / kms / 1e9 / ALU_PEAK_TFLOPS, 4)
                                      if prec == capi.LP_FP64 else None),
                    "obj": obj, "obj_rel_err_vs_fp64": abs(obj - ref) / abs(ref)})
    print(json.dumps({"workload": "dense LP 8192x8192, FP64 vs FP32 tableau + FP64 reinversion",
                      "results": out, "hbm_peak_gbs": peaks()[0]}), flush=True)


def run_batch(args, capi, torch):
    """1024 dense LPs, m and n log-uniform in [32, 1024], one batched launch
    (autotuned launch shape) against one LP per launch."""
    import numpy as np
    from paper_1804_04737_gb300 import lpgen
    lps = [(torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda(), torch.from_numpy(c).cuda(),
            capi.LP_MAX_LE) for A, b, c in lpgen.batch_lps(1024, 32, 1024, seed=0)]
    torch.cuda.synchronize()
    best = capi.lp_batch_autotune(lps, cache_path="/tmp/gbs_batch_tune.txt")
    for _ in range(args.warmup):
        capi.lp_solve_batch(lps, best)
    walls, kms = [], []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        obj, st, it = capi.lp_solve_batch(lps, best)
        walls.append(time.perf_counter() - t0)
        kms.append(capi.lp_batch_stats()[0])
    pivots = int(np.sum(it))
    alg = sum(int(it[k]) * tableau_bytes(int(L[0].shape[0]), int(L[0].shape[1]))
              for k, L in enumerate(lps))
    h = capi.lp_create()
    t0 = time.perf_counter()
    for A, b, c, s in lps[:128]:
        capi.lp_load(h, A, b, c, s)
        capi.lp_solve(h)
        capi.lp_result(h)
    single = 128 / (time.perf_counter() - t0)
    capi.lp_destroy(h)
    wall = float(np.median(walls))
    print(json.dumps({"workload": "batch of 1024 dense LPs, m,n log-uniform [32,1024], FP64",
                      "lps_per_s": round(1024 / wall, 1), "wall_ms": round(1e3 * wall, 2),
                      "kernel_ms": round(float(np.median(kms)), 2), "pivots": pivots,
                      "pivots_per_s": round(pivots / wall, 1),
                      "tableau_gbs_kernel": round(alg / float(np.median(kms)) / 1e6, 1),
                      "all_optimal": bool(np.all(st == capi.LP_OPTIMAL)),
                      "launch_shape": {"group_elems": best.group_elems, "threads": best.threads},
                      "one_lp_per_launch_lps_per_s": round(single, 1)}), flush=True)
    # FP32 tableaus with FP64 reinversion every k pivots, the same batch; the
    # FP64 batch (bit-identical to the FP64 oracle) is the reference objective
    for k in (50, 200):
        opt = capi.lp_options_default(precision=capi.LP_FP32_REINV, reinv_k=k)
        capi.lp_solve_batch(lps, opt)
        t0 = time.perf_counter()
        o32, s32, i32 = capi.lp_solve_batch(lps, opt)
        w32 = time.perf_counter() - t0
        k32 = capi.lp_batch_stats()[0]
        err = float(np.max(np.abs(o32 - obj) / np.maximum(1.0, np.abs(obj))))
        print(json.dumps({"workload": "batch of 1024 dense LPs, m,n log-uniform [32,1024], "
                                      "FP32 tableau + FP64 reinversion k=%d" % k,
                          "lps_per_s": round(1024 / w32, 1), "wall_ms": round(1e3 * w32, 2),
                          "pivot_kernel_ms": round(k32, 2), "pivots": int(np.sum(i32)),
                          "all_optimal": bool(np.all(s32 == capi.LP_OPTIMAL)),
                          "max_obj_rel_err_vs_fp64": err}), flush=True)


def run_serve(args, capi, torch):
    """Poisson stream of dense LPs (m, n log-uniform in [64, 4096]; a pool of
    distinct LPs reused round robin) into a server with a 60 GB HBM budget;
    arrival rate swept up by 1.5x until throughput stops rising.  FP64, then
    FP32 tableaus with FP64 reinversion every 50 pivots."""
    import numpy as np
    from paper_1804_04737_gb300 import lpgen
    pool = [lpgen.dense_lp(m, n, seed=k) for k, (m, n) in
            enumerate(lpgen.log_uniform_shapes(96, 64, 4096, seed=0))]
    per_point = max(200, 40 * args.steps)

    def sweep(opt):
        rng = np.random.default_rng(0)
        srv = capi.lp_server_create(opt, hbm_budget_bytes=60 << 30, max_slots=512)
        points = []
        rate = 50.0
        try:
            for _ in range(10):
                arrivals = np.cumsum(rng.exponential(1.0 / rate, size=per_point))
                tickets = []
                t0 = time.perf_counter()
                for k, ta in enumerate(arrivals):
                    d = t0 + ta - time.perf_counter()
                    if d > 0:
                        time.sleep(d)
                    A, b, c = pool[k % len(pool)]
                    tickets.append((capi.lp_server_submit(srv, A, b, c), A.shape))
                lat, objs = [], []
                for t, (m, n) in tickets:
                    r = capi.lp_server_wait(srv, t, m, n, timeout_s=600)
                    lat.append(r[5])
                    objs.append(r[0])
                span = time.perf_counter() - t0
                thr = per_point / span
                points.append({"offered_per_s": round(rate, 1), "lps_per_s": round(thr, 1),
                               "p50_ms": round(float(np.percentile(lat, 50)), 2),
                               "p99_ms": round(float(np.percentile(lat, 99)), 2)})
                if len(points) > 1 and thr < 1.05 * points[-2]["lps_per_s"]:
                    break
                rate *= 1.5
        finally:
            capi.lp_server_destroy(srv)
        return points, objs

    # one LP per launch on the same requests (lp_load + lp_solve + lp_result,
    # FP64, one handle), for the served rates to be compared with; the pass
    # is timed after one untimed pass, in which the handle's buffers grow
    h = capi.lp_create(capi.lp_options_default())
    try:
        for timed in (False, True):
            t0 = time.perf_counter()
            for A, b, c in pool:
                capi.lp_load(h, A, b, c)
                capi.lp_solve(h)
                capi.lp_result(h)
        one = len(pool) / (time.perf_counter() - t0)
    finally:
        capi.lp_destroy(h)
    fp64, obj64 = sweep(capi.lp_options_default())
    fp32, obj32 = sweep(capi.lp_options_default(precision=capi.LP_FP32_REINV, reinv_k=50))
    # the last point's requests are the same LPs in the same order in both
    # sweeps (same seed and pool): the FP32 objectives against the FP64 ones
    n = min(len(obj64), len(obj32))
    err = max(abs(a - b) / max(1.0, abs(b)) for a, b in zip(obj32[:n], obj64[:n]))
    print(json.dumps({"workload": "serving: Poisson stream of dense LPs, m,n log-uniform "
                      "[64,4096], 60 GB HBM budget", "requests_per_point": per_point,
                      "alone_from_tableau_elems": 1 << 24,  # lp_options.solo_elems default
                      "one_lp_per_launch_fp64_lps_per_s": round(one, 1),
                      "fp64": {"saturation": max(fp64, key=lambda p: p["lps_per_s"]), "sweep": fp64},
                      "fp32_reinv_k50": {"saturation": max(fp32, key=lambda p: p["lps_per_s"]),
                                         "sweep": fp32,
                                         "max_obj_rel_err_vs_fp64_server": err}}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gbsimplex", choices=["gbsimplex", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="lp2048set",
                    choices=["lp2048set", "paperset", "lp8192", "batch1024", "serve"],
                    help="lp2048set is the headline line; the others report their own figures")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1804_04737_gb300 import capi

    torch.cuda.set_device(local)
    family = "paper" if args.workload == "paperset" else "dense"
    wname = PAPER_WORKLOAD_NAME if family == "paper" else WORKLOAD_NAME
    if args.workload not in ("lp2048set", "paperset"):
        return {"lp8192": run_lp8192, "batch1024": run_batch,
                "serve": run_serve}[args.workload](args, capi, torch)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.Stream()
    lps = workload(rank, family)
    dev_in = [(name, *(torch.from_numpy(v).cuda() for v in (A, b, c)), sense)
              for name, A, b, c, sense in lps]
    handles = [capi.lp_create(capi.lp_options_default(cuda_stream=stream, device=local))
               for _ in lps]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()

    def device_step():
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            for h, (_, A, b, c, sense) in zip(handles, dev_in):
                capi.lp_load(h, A, b, c, sense)
                capi.lp_solve_async(h)
            ev1.record(stream)
        stats = []
        for h in handles:
            obj, st, it = capi.lp_result(h)
            if st != capi.LP_OPTIMAL:
                raise RuntimeError("solve ended with status %s" % capi.STATUS_NAMES[st])
            kms, _ = capi.lp_kernel_time(h)
            stats.append((it, kms, obj))
        ev1.synchronize()
        return ev0.elapsed_time(ev1), stats

    for _ in range(args.warmup):
        device_step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    step_ms, pivots, kernel_ms, alg_bytes = [], 0, 0.0, 0.0
    per_kernel = {}  # name -> [launches, ms, algorithmic bytes, pivots]
    with Clocks(local) as clk:
        for _ in range(args.steps):
            ms, stats = device_step()
            step_ms.append(ms)
            for (it, kms, _), (_, A, _b, _c, sense) in zip(stats, lps):
                pivots += it
                kernel_ms += kms
                by = it * tableau_bytes(A.shape[0], A.shape[1])
                alg_bytes += by
                rec = per_kernel.setdefault(kernel_of(A.shape[0], A.shape[1], sense),
                                            [0, 0.0, 0.0, 0])
                rec[0] += 1
                rec[1] += kms
                rec[2] += by
                rec[3] += it
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    (total_ms,), (all_pivots,) = reduce_over_ranks(dist, [sum(step_ms)], [pivots], "cuda")
    all_pivots = int(all_pivots)

    # end to end from pinned host buffers through the C ABI
    host_in = []
    for _, A, b, c, sense in lps:
        pin = [torch.from_numpy(v).pin_memory() for v in (A, b, c)]
        m, n = A.shape
        host_in.append((pin, torch.empty(n, dtype=torch.float64).pin_memory(),
                        torch.empty(m, dtype=torch.float64).pin_memory(), sense))
    h2d = sum(8 * (A.size + b.size + c.size) for _, A, b, c, _ in lps)
    d2h = sum(8 * (A.shape[0] + A.shape[1] + 1) for _, A, _, _, _ in lps)

    def e2e_step():
        piv = 0
        for h, (pin, x, y, sense) in zip(handles, host_in):
            capi.lp_load(h, pin[0].numpy(), pin[1].numpy(), pin[2].numpy(), sense)
            capi.lp_solve(h)
            _, st, it = capi.lp_result(h, x.numpy(), y.numpy())
            piv += it
        return piv

    e2e_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_piv = 0
    for _ in range(args.steps):
        e2e_piv += e2e_step()
    torch.cuda.synchronize()
    e2e_sec = time.perf_counter() - t0
    (e2e_sec_max,), (e2e_piv_all,) = reduce_over_ranks(dist, [e2e_sec], [e2e_piv], "cuda")
    e2e_val = e2e_piv_all / e2e_sec_max

    for h in handles:
        capi.lp_destroy(h)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    hbm_peak, peak_kind = peaks()
    gbs = alg_bytes / (kernel_ms * 1e-3) / 1e9

    def roofline_of(name):
        """HBM and FP64-ALU rooflines of one kernel: algorithmic bytes (or
        flops) per launch over its mean CUDA-event launch duration."""
        launches, ms, by, piv = per_kernel[name]
        sec = ms * 1e-3
        flops = by / 16 * 2  # one FMA (2 flops) per 16 bytes of FP64 read + write
        hbm = {"bound": "hbm", "achieved": round(by / sec / 1e9, 1), "peak": hbm_peak,
               "unit": "GB/s", "frac": round(by / sec / 1e9 / hbm_peak, 4),
               "peak_kind": peak_kind,
               "frac_of_nominal": round(by / sec / 1e9 / HBM_NOMINAL_GBS, 4)}
        alu = {"bound": "alu", "achieved": round(flops / sec / 1e12, 4),
               "peak": round(ALU_PEAK_TFLOPS, 4), "unit": "TFLOP/s",
               "frac": round(flops / sec / 1e12 / ALU_PEAK_TFLOPS, 4),
               "peak_kind": "derived: 2 FP64 FMA/clk/SM x 152 SMs x 2070 MHz"}
        r = dict(max((hbm, alu), key=lambda x: x["frac"]))
        r["secondary"] = alu if r["bound"] == "hbm" else hbm
        r["kernel"] = name
        r["launches_per_step"] = launches // args.steps
        r["mean_launch_ms"] = round(ms / launches, 4)
        r["algorithmic_bytes_per_launch"] = round(by / launches)
        r["share_of_pivot_kernel_time"] = round(ms / kernel_ms, 4)
        return r

    dominant = max(per_kernel, key=lambda k: per_kernel[k][1])
    roof = roofline_of(dominant)
    # (the DRAM records are of the integer family's step)
    roof["traffic"] = kernel_traffic(dominant) if family == "dense" else None
    others = []
    for k in per_kernel:
        if k != dominant:
            r = roofline_of(k)
            r["traffic"] = kernel_traffic(k) if family == "dense" else None
            others.append(r)
    roof["others"] = others
    line = {
        "metric": "pivots/s", "value": all_pivots / (total_ms * 1e-3), "unit": "pivots/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wname, "seed": "rank", "lps": [n for n, *_ in lps],
                   "pivots_per_step": pivots // args.steps,
                   "l2": "flushed between steps (256 MiB write), outside the step events",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "tableau_gbs": round(gbs, 1),
        "e2e": {"value": e2e_val, "unit": "pivots/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "roofline": roof,
        "gpu_launches": 5 * len(lps) * args.steps,
        "clocks": clk.summary(),
    }
    if world == 1 and not args.no_cpu_baseline:
        # the whole workload, repeated until about 10 s of oracle time
        cores = len(os.sched_getaffinity(0))
        # the paper family's LPs take thousands of pivots: the sample stops
        # each LP after a fixed number of them
        cap, cap1 = (200, 20) if family == "paper" else (None, None)
        p, t, reps = 0, 0.0, 0
        while t < 10.0 and reps < 1000:
            dp, dt = cpu_oracle_run(lps, cores, cap)
            p, t, reps = p + dp, t + dt, reps + 1
        p1, t1 = cpu_oracle_run(lps, 1, cap1)
        what = "the whole workload (4 LPs)" if cap is None else "the first %d pivots of each LP" % cap
        what1 = "the whole workload" if cap1 is None else "the first %d pivots of each LP" % cap1
        line["cpu_baseline"] = {"value": p / t, "unit": "pivots/s", "cores": cores,
                                "kind": "oracle",
                                "sample": "%s %d times, %.1f s" % (what, reps, t),
                                "single_thread": {"value": p1 / t1, "unit": "pivots/s",
                                                  "sample": "%s once, %.1f s" % (what1, t1)}}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
