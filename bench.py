#!/usr/bin/env python3
"""Throughput of the dense tableau simplex on GB300: pivots/s and tableau GB/s.

Default workload (one step): the 8192 x 8192 dense LP (tableau 8193 x 16385,
1.07 GB in FP64), primal form max c'x s.t. Ax <= b, x >= 0, solved to
optimality in FP64 (Sec. 2 Steps 1-5, Dantzig pricing): lp_load from device
buffers (the tableau is built inside the timed region) and lp_solve.  A
entries uniform integers in [1, 1000], b in [1000, 100000], c in [1, 100],
seed 0.  Beside it, on the same LP: the FP32 tableau with FP64 reinversion
every k in {50, 200} pivots, with its objective error against the FP64
oracle.

`value` is pivots per second over the whole job, device-timed with CUDA
events on the library's stream, inputs resident in HBM.  The tableau (1.07 GB,
two buffers) is larger than L2, so nothing survives in L2 from one step to
the next.  `e2e` is the same metric through the C ABI with host buffers:
lp_load from pinned host memory, lp_solve, lp_result into pinned host memory,
wall clock.  `roofline` is that of the pivot kernel (one launch per solve):
the FP64 FMA rate of the fmas it executes (one per updated tableau element
and pivot; the two-pivot primal kernel leaves in place the column vectors
whose entries in both pivot rows of a pass are zero, and counts what it
updates) and the DRAM bytes it moves (from an ncu record of the same
launch), the larger fraction leading; pivot-equivalent GB/s (2 x tableau
bytes per pivot) is reported beside them, not as a bound: two pivots share
one pass over the tableau, and vectors left in place are not moved.

Other workloads (--workload): lp2048set (2048^2 primal and dual form,
512 x 4096, 4096 x 512), paperset (the same shapes from the paper's random
family), batch1024, serve, servespill (servers that spill idle LPs to host
memory, off and on), product (the emulated-FP64 product alone).
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

MAX_LE, MIN_GE = 0, 1
HBM_NOMINAL_GBS = 7900.0          # GB300 HBM3e nominal
FP64_DFMA_PER_CLK_SM = 2          # GB300 FP64: 1.25 TFLOP/s nominal = 2 DFMA per clock per SM
KERNEL_SRC = os.path.join(ROOT, "paper_1804_04737_gb300", "csrc", "gbs_pipe.cu")

WORKLOADS = {
    "lp8192": ("dense LP 8192x8192 (tableau 8193x16385, 1.07 GB FP64), primal form, FP64, Dantzig "
               "pricing; FP32 tableau + FP64 reinversion every 50 and 200 pivots beside it"),
    "lp2048set": ("dense LP set: 2048x2048 primal + 2048x2048 dual form + 512x4096 + 4096x512, "
                  "FP64, Dantzig pricing"),
    # the same shapes from the paper's own random family (Sec. 4): density 0.9,
    # real-valued data, about 25 times the pivots of the integer family
    "paperset": ("paper-family LP set: 2048x2048 primal + 2048x2048 dual form + 512x4096 + "
                 "4096x512, density 0.9, FP64, Dantzig pricing"),
}
# what the reference arm times per step: the oracle's first REF_PIVOTS pivots
# of each LP (8192^2: a full solve is several seconds of host time)
REF_PIVOTS = {"lp8192": 20, "lp2048set": None, "paperset": 200}


def workload(name, seed=0):
    from paper_1804_04737_gb300 import lpgen
    if name == "lp8192":
        return [("8192x8192 primal", *lpgen.dense_lp(8192, 8192, seed), MAX_LE)]
    gen = lpgen.dense_lp if name == "lp2048set" else lpgen.paper_lp
    out = []
    A, b, c = gen(2048, 2048, seed)
    out.append(("2048x2048 primal", A, b, c, MAX_LE))
    out.append(("2048x2048 dual form", *lpgen.dual_of(A, b, c), MIN_GE))
    out.append(("512x4096 primal", *gen(512, 4096, seed), MAX_LE))
    out.append(("4096x512 primal", *gen(4096, 512, seed), MAX_LE))
    return out


def bench_config(name, world):
    """The `config` of both arms' lines (identical, so the driver can pair them)."""
    cfg = {"workload": WORKLOADS[name], "seed": 0,
           "parallelism": "replicas" if world > 1 else "single GPU"}
    if name == "lp8192":
        cfg.update({"m": 8192, "n": 8192, "l2": "inputs larger than L2 (1.07 GB tableau, "
                                                 "two buffers)"})
    else:
        cfg["l2"] = "flushed between steps (256 MiB write), outside the step events"
    return cfg


def tableau_bytes(m, n, w=8):
    """Algorithmic bytes of one pivot: the rank-1 update reads and writes the
    whole (m+1) x (n+m+1) tableau once (Sec. 2 Step 5)."""
    return 2 * (m + 1) * (n + m + 1) * w


def tableau_flops(m, n):
    """One fma (2 flops) per tableau element and pivot (Sec. 2 Step 5)."""
    return 2 * (m + 1) * (n + m + 1)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def bf16_peak():
    """(TFLOP/s, how): the measured dense bf16 rate (burst), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"


def device_fp64_peak(index):
    """(TFLOP/s, how): 2 FP64 FMA per clock per SM x the device's SM count x its
    maximum SM clock (nvidia-smi), the derived FP64 FMA peak."""
    import torch
    sms = torch.cuda.get_device_properties(index).multi_processor_count
    mhz = None
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(index), "--query-gpu=clocks.max.sm",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True,
                             timeout=30).stdout.strip()
        mhz = float(out.splitlines()[0])
    except Exception:
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
                mhz = float(json.load(f)["sm_max_mhz"])
        except Exception:
            mhz = 2070.0
    tf = 2 * FP64_DFMA_PER_CLK_SM * sms * mhz * 1e6 / 1e12
    return tf, "derived: %d FP64 FMA/clk/SM x %d SMs x %.0f MHz" % (FP64_DFMA_PER_CLK_SM, sms, mhz)


# The kernel each LP runs on (default options): primal LPs below 2^19 tableau
# elements on the pipelined primal kernel in place, larger ones on the
# two-pivots-per-pass kernel (double-buffered), the dual form on the
# two-pivots-per-pass dual simplex kernel (double-buffered).
INPLACE_KERNEL = "pivot_pipe_kernel<double> (in place)"
BLOCK_KERNEL = "pivot_block_kernel<double> (two pivots per pass)"
DUAL_KERNEL = "pivot_block_dual_kernel<double> (dual simplex, two pivots per pass)"
# DRAM records (ncu) per kernel and workload; the in-place kernel runs no LP of
# these sets, so it has none
TRAFFIC_FILES = {
    ("lp8192", BLOCK_KERNEL): "pivot_block_kernel_fp64_8192_traffic.txt",
    ("lp2048set", BLOCK_KERNEL): "pivot_block_kernel_fp64_traffic.txt",
    ("lp2048set", DUAL_KERNEL): "pivot_block_dual_kernel_fp64_traffic.txt",
}


def kernel_of(m, n, sense):
    if sense != MAX_LE:
        return DUAL_KERNEL
    pitch = (n + m + 1 + 31) // 32 * 32
    return INPLACE_KERNEL if (m + 1) * pitch < 2 ** 19 else BLOCK_KERNEL


def kernel_traffic(wname, kernel):
    """Mean DRAM bytes (read + write) per launch of one kernel in one step of
    the workload, from the committed ncu record, or None when there is none
    or the kernel source changed since that capture."""
    import hashlib
    try:
        rec = {}
        with open(os.path.join(ROOT, "profiles", TRAFFIC_FILES[(wname, kernel)])) as f:
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
    # one LP per launch on one handle: an untimed pass first (the handle's
    # buffers grow to the largest of the 128), then the timed one
    h = capi.lp_create()
    for A, b, c, s in lps[:128]:
        capi.lp_load(h, A, b, c, s)
        capi.lp_solve(h)
        capi.lp_result(h)
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
    """Serving (the workload's fifth configuration): a Poisson stream of dense
    LPs, m and n log-uniform in [64, 4096], into a server with a 60 GB HBM
    budget.  First a sweep: 400 requests per point (200 at --steps 5 or
    fewer), arrival rate raised 1.5x until the served rate stops rising, for
    the FP64 server and for FP32 tableaus with FP64 reinversion every 50
    pivots.  Then the stated stream: 20000 requests at each server's
    saturating rate, and one LP per launch (lp_load + lp_solve + lp_result,
    FP64, one handle) over the same 20000 requests.  The FP64 server runs
    twice: with its persistent kernel (lanes 0) and with three lanes.  The requests cycle
    through a pool of 512 distinct seeded LPs (20000 distinct ones would take
    about 150 GB of host memory and more generator time than the stream)."""
    import numpy as np
    from paper_1804_04737_gb300 import lpgen
    pool = [lpgen.dense_lp(m, n, seed=k) for k, (m, n) in
            enumerate(lpgen.log_uniform_shapes(512, 64, 4096, seed=0))]
    per_point = max(200, 40 * args.steps) if args.steps <= 10 else 400
    stream_len = 20000

    def run_stream(srv, rate, count, rng):
        arrivals = np.cumsum(rng.exponential(1.0 / rate, size=count))
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
        return {"offered_per_s": round(rate, 1), "requests": count,
                "lps_per_s": round(count / span, 1),
                "p50_ms": round(float(np.percentile(lat, 50)), 2),
                "p99_ms": round(float(np.percentile(lat, 99)), 2)}, objs

    def sweep(opt):
        rng = np.random.default_rng(0)
        srv = capi.lp_server_create(opt, hbm_budget_bytes=60 << 30, max_slots=512)
        points = []
        rate = 50.0
        try:
            for _ in range(12):
                pt, _ = run_stream(srv, rate, per_point, rng)
                points.append(pt)
                if len(points) > 1 and pt["lps_per_s"] < 1.05 * points[-2]["lps_per_s"]:
                    break
                rate *= 1.5
            best = max(points, key=lambda p: p["lps_per_s"])
            # the stated stream, at the rate that saturated the server
            stream, objs = run_stream(srv, best["offered_per_s"], stream_len,
                                      np.random.default_rng(1))
        finally:
            capi.lp_server_destroy(srv)
        return points, best, stream, objs

    def one_per_launch():
        # one LP per launch on the same 20000 requests (after one untimed pass
        # over the pool, in which the handle's buffers grow)
        h = capi.lp_create(capi.lp_options_default())
        try:
            for A, b, c in pool:
                capi.lp_load(h, A, b, c)
                capi.lp_solve(h)
                capi.lp_result(h)
            t0 = time.perf_counter()
            for k in range(stream_len):
                A, b, c = pool[k % len(pool)]
                capi.lp_load(h, A, b, c)
                capi.lp_solve(h)
                capi.lp_result(h)
            return stream_len / (time.perf_counter() - t0)
        finally:
            capi.lp_destroy(h)

    one = one_per_launch()
    fp64_pts, fp64_best, fp64_stream, obj64 = sweep(capi.lp_options_default(lanes=0))
    lane_pts, lane_best, lane_stream, objl = sweep(capi.lp_options_default(lanes=3))
    fp32_pts, fp32_best, fp32_stream, obj32 = sweep(
        capi.lp_options_default(precision=capi.LP_FP32_REINV, reinv_k=50))
    one_after = one_per_launch()
    # the two streams hold the same LPs in the same order: FP32 against FP64
    err = max(abs(a - b) / max(1.0, abs(b)) for a, b in zip(obj32, obj64))
    print(json.dumps({"workload": "serving: Poisson stream of dense LPs, m,n log-uniform "
                      "[64,4096], 60 GB HBM budget", "pool": len(pool),
                      "sweep_requests_per_point": per_point,
                      "alone_from_tableau_elems": 1 << 24,  # lp_options.solo_elems default
                      "stream_requests": stream_len,
                      "one_lp_per_launch_fp64_lps_per_s": round(one, 1),
                      "one_lp_per_launch_again_after_the_servers": round(one_after, 1),
                      "fp64": {"stream_at_saturation": fp64_stream, "sweep": fp64_pts},
                      "fp64_3_lanes": {"stream_at_saturation": lane_stream, "sweep": lane_pts,
                                       "same_objectives_as_server_kernel": objl == obj64},
                      "fp32_reinv_k50": {"stream_at_saturation": fp32_stream, "sweep": fp32_pts,
                                         "max_obj_rel_err_vs_fp64_server": err}}), flush=True)

def run_serve_spill(args, capi, torch):
    """Spilling idle LPs to host memory (lp_options.spill_pivots), with it off
    and on, on two streams where some LPs hold the device for long:
    - FP64: a Poisson stream (100 requests/s) of small dense LPs (m, n
      log-uniform in [64, 512]) with one LP of the paper's family at 2048^2
      (seeds 1 and 2 in turn; seed 1 takes 24734 pivots, 0.55 s alone) in
      every 100 requests; LPs of at least 2^22 tableau elements run alone,
      and with spilling on they run 400 pivots at a time and are spilled
      while others wait;
    - FP32 + FP64 reinversion every 50 pivots: a Poisson stream (100/s) of
      LPs of the paper's family, m and n log-uniform in [256, 1024] (tens to
      thousands of pivots), under a 64 MB budget (a few LPs at a time); with
      spilling on, LPs that made 100 pivots since their admission are spilled
      between rounds when the queue head does not fit.
    Latency percentiles of the small and of the large LPs (FP64) or of all of
    them (FP32), served rate, spills; the results are the same bits with
    spilling off and on (checked)."""
    import numpy as np
    from paper_1804_04737_gb300 import lpgen
    count = 250 if args.steps <= 5 else 500

    def stream(opt, budget, lps, rate, seed):
        srv = capi.lp_server_create(opt, hbm_budget_bytes=budget, max_slots=256)
        try:
            arrivals = np.cumsum(np.random.default_rng(seed).exponential(1.0 / rate, size=len(lps)))
            tickets = []
            t0 = time.perf_counter()
            for (A, b, c), ta in zip(lps, arrivals):
                d = t0 + ta - time.perf_counter()
                if d > 0:
                    time.sleep(d)
                tickets.append(capi.lp_server_submit(srv, A, b, c))
            res = [capi.lp_server_wait(srv, t, A.shape[0], A.shape[1], timeout_s=600)
                   for t, (A, _, _) in zip(tickets, lps)]
            span = time.perf_counter() - t0
            sp, rs, host = capi.lp_server_spill_stats(srv)
        finally:
            capi.lp_server_destroy(srv)
        return res, span, {"spills": sp, "restores": rs, "pinned_host_mb": round(host / 2 ** 20, 1)}

    def pct(v):
        return {"p50_ms": round(float(np.percentile(v, 50)), 2),
                "p99_ms": round(float(np.percentile(v, 99)), 2)}

    def same(ra, rb):
        return all(a[1] == b[1] and a[2] == b[2] and
                   np.array_equal(np.asarray(a[3]).view(np.uint64), np.asarray(b[3]).view(np.uint64))
                   for a, b in zip(ra, rb))

    out = {"workload": "serving with spilling of idle LPs to host memory", "requests": count}
    # FP64: small LPs and large ones that run alone
    smalls = [lpgen.dense_lp(m, n, seed=k) for k, (m, n) in
              enumerate(lpgen.log_uniform_shapes(96, 64, 512, seed=3))]
    bigs = [lpgen.paper_lp(2048, 2048, seed=s) for s in (1, 2)]
    lps, big = [], []
    for k in range(count):
        big.append(k % 100 == 12)
        lps.append(bigs[(k // 100) % 2] if big[-1] else smalls[k % len(smalls)])
    fp64 = {}
    runs = {}
    for spill in (0, 400):
        opt = capi.lp_options_default(solo_elems=1 << 22, spill_pivots=spill)
        res, span, st = stream(opt, 8 << 30, lps, 100.0, 5)
        lat = np.array([r[5] for r in res])
        isbig = np.array(big)
        fp64["spill_pivots_%d" % spill] = {
            "lps_per_s": round(len(lps) / span, 1), "small": pct(lat[~isbig]),
            "large": pct(lat[isbig]), **st}
        runs[spill] = res
    fp64["same_results"] = same(runs[0], runs[400])
    out["fp64_small_lps_and_2048sq_alone_100_per_s"] = fp64
    # FP32 rounds under a small budget
    lps32 = [lpgen.paper_lp(m, n, seed=100 + k) for k, (m, n) in
             enumerate(lpgen.log_uniform_shapes(count // 2, 256, 1024, seed=4))]
    fp32 = {}
    runs = {}
    for spill in (0, 100):
        opt = capi.lp_options_default(precision=capi.LP_FP32_REINV, reinv_k=50, spill_pivots=spill)
        res, span, st = stream(opt, 64 << 20, lps32, 100.0, 6)
        lat = np.array([r[5] for r in res])
        fp32["spill_pivots_%d" % spill] = {"lps_per_s": round(len(lps32) / span, 1), **pct(lat), **st}
        runs[spill] = res
    fp32["same_results"] = same(runs[0], runs[100])
    out["fp32_reinv_k50_paper_family_256_1024_budget_64mb_100_per_s"] = fp32
    print(json.dumps(out), flush=True)


def cpu_oracle_run(lps, threads, cap=None):
    """Pivots and seconds of the oracle's pivoting on the workload (the Step 1
    build excluded), each LP stopped after `cap` pivots when given."""
    import oracle
    oracle.set_threads(threads)
    pivots, sec = 0, 0.0
    for _, A, b, c, sense in lps:
        t = oracle.OracleTableau(A, b, c, sense)
        t0 = time.perf_counter()
        st = t.run(cap if cap else 10 ** 12)
        sec += time.perf_counter() - t0
        assert st == (oracle.ITER_LIMIT if cap and t.iters.value == cap else oracle.OPTIMAL)
        pivots += t.iters.value
    return pivots, sec


def run_reference(args, rank, world):
    """The FP64 oracle (the paper's method as plain C, OpenMP over the rows of
    Step 5) on the host cores: same workload, config, metric and units; each
    step a bounded sample of the workload."""
    if rank != 0:
        return
    if args.workload not in WORKLOADS:
        print(json.dumps({"impl": "reference", "unavailable":
                          "the reference arm covers the single-LP workloads only"}), flush=True)
        return
    cores = len(os.sched_getaffinity(0))
    lps = workload(args.workload, 0)
    cap = REF_PIVOTS[args.workload]
    for _ in range(args.warmup):
        cpu_oracle_run(lps, cores, cap)
    piv, sec = 0, 0.0
    for _ in range(args.steps):
        p, t = cpu_oracle_run(lps, cores, cap)
        piv += p
        sec += t
    v = piv / sec
    what = ("the first %d pivots of each LP" % cap if cap else "the whole workload") + \
        " per step, Step 1 build excluded"
    line = {"impl": "reference", "metric": "pivots/s", "value": v, "unit": "pivots/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sec / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(args.workload, world),
            "cpu_baseline": {"value": v, "unit": "pivots/s", "cores": cores, "kind": "oracle",
                             "sample": what},
            "e2e": {"value": v, "unit": "pivots/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def lp8192_extras(args, capi, torch, lps, dev_in, g_obj, g_iters, local):
    """Beside the FP64 line of the 8192^2 LP: the oracle's first 200 pivots on
    all host cores and its first 10 on one (cpu_baseline), the rest of its
    solve (parity of the FP64 pivots and objective), and the FP32 tableau with
    FP64 reinversion every 50 and 200 pivots, with objective errors against
    the oracle."""
    import numpy as np
    import oracle
    _, A, b, c, sense = lps[0]
    _, dA, db, dc, _ = dev_in[0]
    out = {}
    ores = None
    if not args.no_cpu_baseline:
        cores = len(os.sched_getaffinity(0))
        oracle.set_threads(cores)
        t = oracle.OracleTableau(A, b, c, sense)
        t0 = time.perf_counter()
        t.run(200)
        t200, p200 = time.perf_counter() - t0, t.iters.value
        t.run()  # on to the optimum, untimed
        ores = t.result()
        del t
        oracle.set_threads(1)
        t1 = oracle.OracleTableau(A, b, c, sense)
        t0 = time.perf_counter()
        t1.run(10)
        ts, ps = time.perf_counter() - t0, t1.iters.value
        del t1
        oracle.set_threads(cores)
        out["cpu_baseline"] = {
            "value": p200 / t200, "unit": "pivots/s", "cores": cores, "kind": "oracle",
            "sample": "the first %d pivots of the 8192x8192 LP, Step 1 build excluded, %.1f s"
                      % (p200, t200),
            "single_thread": {"value": ps / ts, "unit": "pivots/s",
                              "sample": "the first %d pivots, %.1f s" % (ps, ts)}}
        out["parity"] = {"oracle_status": oracle.STATUS_NAMES[ores.status],
                         "oracle_pivots": ores.iters,
                         "fp64_pivots_equal": g_iters == ores.iters,
                         "fp64_obj_bitwise_equal": bool(np.float64(g_obj).view(np.uint64) ==
                                                        np.float64(ores.obj).view(np.uint64))}
    fp32 = []
    for k in (50, 200):
        h = capi.lp_create(capi.lp_options_default(precision=capi.LP_FP32_REINV, reinv_k=k,
                                                   device=local))
        runs = []
        try:
            for rep in range(1 + max(2, args.steps // 5)):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                capi.lp_load(h, dA, db, dc, sense)
                capi.lp_solve(h)
                obj, st, it = capi.lp_result(h)
                wall = time.perf_counter() - t0
                kms, launches = capi.lp_kernel_time(h)
                nre, rms, bms = capi.lp_fp32_stats(h)
                if rep:
                    runs.append((wall, kms, launches, obj, st, it, nre, rms, bms))
        finally:
            capi.lp_destroy(h)
        runs.sort()
        wall, kms, launches, obj, st, it, nre, rms, bms = runs[len(runs) // 2]
        fp32.append({"reinv_k": k, "status": capi.STATUS_NAMES[st], "pivots": it,
                     "pivots_per_s": round(it / wall, 1), "solve_ms": round(1e3 * wall, 2),
                     "pivot_kernel_ms": round(kms, 2), "pivot_kernel_launches": launches,
                     "reinversions": nre, "reinversion_ms": round(rms, 2),
                     "body_refresh_ms": round(bms, 2),
                     "pivot_equivalent_gbs_kernel":
                         round(it * tableau_bytes(8192, 8192, 4) / (kms * 1e-3) / 1e9, 1),
                     "obj": obj,
                     "obj_rel_err_vs_oracle": (abs(obj - ores.obj) / abs(ores.obj)
                                               if ores is not None else None),
                     "timing": "wall clock of lp_load + lp_solve + lp_result, inputs in HBM, "
                               "median of %d" % len(runs)})
    out["fp32_reinv"] = fp32
    out["emulated_fp64_product"] = product_bench(capi, torch, local)
    return out


def product_bench(capi, torch, local, m=8192, n=8192, s=334):
    """The body refresh's big product at the 8192^2 LP's final basis: the
    (m - s) x s rows of A times the s x (n + m + 1) block, emulated FP64 on the
    tensor cores (lp_dgemm_emulated), timed with CUDA events on its stream
    (digit split, product and epilogue): the 2 M N K FP64 flops it stands
    for per second, against the FP64 pipe's derived peak.  (How many of the 28
    bf16 digit products run depends on the data: digit planes that are zero
    for a whole row or column block are skipped; the tensor-pipe share is in
    the ncu record under profiles/.)"""
    import numpy as np
    M, N, K = m - s, n + m + 1, s
    rng = np.random.default_rng(0)
    A = torch.from_numpy(rng.integers(1, 1001, size=(M, K)).astype(np.float64)).cuda()
    B = torch.from_numpy(rng.standard_normal((K, N))).cuda()
    C = torch.empty((M, N), dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream()
    opt = capi.lp_options_default(cuda_stream=stream, device=local)
    capi.lp_dgemm_emulated(A, B, C, opt)  # grows the workspace
    times = []
    for _ in range(5):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        capi.lp_dgemm_emulated(A, B, C, opt)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = float(np.median(times))
    # the bf16 digit products the tensor cores ran (128 x 64 x 16 per MMA)
    tensor_flops = capi.lp_dgemm_stats() * 2.0 * 128 * 64 * 16
    bf16, bf16_how = bf16_peak()
    ref = (A.cpu().numpy() @ B[:, :256].cpu().numpy())
    err = float(np.max(np.abs(C[:, :256].cpu().numpy() - ref) / np.maximum(1.0, np.abs(ref))))
    fp64_peak, how = device_fp64_peak(local)
    flops = 2.0 * M * N * K
    return {"shape": {"M": M, "N": N, "K": K},
            "data": "A integers in [1, 1000] (the LP's own data), B standard normal", "ms": round(ms, 3),
            "fp64_equivalent_tflops": round(flops / ms / 1e9, 2),
            "vs_fp64_pipe_peak": round(flops / ms / 1e9 / fp64_peak, 2), "fp64_peak_kind": how,
            "fp64_pipe_ms_for_the_same_product": round(flops / (fp64_peak * 1e12) * 1e3, 1),
            "tensor": {"bf16_tflops_executed": round(tensor_flops / ms / 1e9, 1),
                       "bf16_flops_per_fp64_flop": round(tensor_flops / flops, 2),
                       "peak": bf16, "peak_kind": bf16_how,
                       "frac": round(tensor_flops / ms / 1e9 / bf16, 4),
                       "note": "digit products run (of 28 pairs, K padded to 64): the whole call, digit split, products and epilogue"},
            "max_rel_err_vs_numpy_fp64_first_256_columns": err}


def run_product(args, capi, torch):
    """The emulated-FP64 product alone, at the body refresh's largest size
    (one workspace-growing call, then five timed)."""
    print(json.dumps({"workload": "emulated-FP64 product of the 8192^2 LP's body refresh "
                                  "(tcgen05, bf16 digit planes)",
                      **product_bench(capi, torch, 0)}), flush=True)


def run_lpset(args, capi, torch, rank, world, local, dist):
    """Single-LP workloads: each step loads and solves every LP of the set
    once on the device, device-timed; then the same through host buffers."""
    import numpy as np
    wname = args.workload
    stream = torch.cuda.Stream()
    lps = workload(wname, 0)
    dev_in = [(name, *(torch.from_numpy(v).cuda() for v in (A, b, c)), sense)
              for name, A, b, c, sense in lps]
    handles = [capi.lp_create(capi.lp_options_default(cuda_stream=stream, device=local))
               for _ in lps]
    # the 8192^2 tableau is larger than L2; the smaller sets flush it
    flush = None if wname == "lp8192" else torch.empty(64 * 1024 * 1024, dtype=torch.float32,
                                                       device="cuda")
    torch.cuda.synchronize()

    def device_step():
        with torch.cuda.stream(stream):
            if flush is not None:
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
            stats.append((it, kms, obj, capi.lp_update_counts(h)))
        ev1.synchronize()
        return ev0.elapsed_time(ev1), stats

    for _ in range(args.warmup):
        device_step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    step_ms, pivots, kernel_ms, alg_bytes = [], 0, 0.0, 0.0
    # name -> [launches, ms, algorithmic bytes, pivots, flops, executed flops,
    #          constraint-row entries updated, left in place]
    per_kernel = {}
    last = None
    with Clocks(local) as clk:
        for _ in range(args.steps):
            ms, stats = device_step()
            step_ms.append(ms)
            last = stats
            for (it, kms, _, (upd, kept)), (_, A, _b, _c, sense) in zip(stats, lps):
                m, n = A.shape
                pivots += it
                kernel_ms += kms
                by = it * tableau_bytes(m, n)
                alg_bytes += by
                rec = per_kernel.setdefault(kernel_of(m, n, sense),
                                            [0, 0.0, 0.0, 0, 0.0, 0.0, 0, 0])
                rec[0] += 1
                rec[1] += kms
                rec[2] += by
                rec[3] += it
                rec[4] += it * tableau_flops(m, n)
                # the fmas executed: the updated constraint-row entries (the
                # two-pivot primal kernel counts them) and the objective row
                pitch = (n + m + 1 + 31) // 32 * 32
                rec[5] += 2 * (upd + it * pitch) if upd + kept else it * tableau_flops(m, n)
                rec[6] += upd
                rec[7] += kept
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
        return

    hbm_peak, peak_kind = peaks()
    fp64_peak, fp64_how = device_fp64_peak(local)

    def roofline_of(name):
        """The pivot kernel's two real rooflines, per launch over its mean
        CUDA-event duration: FP64 FMA (the fmas it executes: one per updated
        element and pivot) and the DRAM bytes it moves (ncu record); the
        larger fraction leads.  Pivot-equivalent GB/s (2 x tableau bytes per
        pivot) is reported too; it is not a bound, since two pivots share one
        pass over the tableau and vectors left in place are not moved."""
        launches, ms, by, piv, flops, xflops, upd, kept = per_kernel[name]
        sec = ms * 1e-3
        traffic = kernel_traffic(wname, name)
        fma = {"achieved": round(xflops / sec / 1e12, 4), "peak": round(fp64_peak, 4),
               "unit": "TFLOP/s", "frac": round(xflops / sec / 1e12 / fp64_peak, 4),
               "peak_kind": fp64_how}
        hbm = None
        if traffic:
            gbs = traffic * launches / sec / 1e9
            hbm = {"achieved": round(gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                   "frac": round(gbs / hbm_peak, 4), "peak_kind": peak_kind,
                   "frac_of_nominal": round(gbs / HBM_NOMINAL_GBS, 4)}
        lead = hbm if hbm is not None and hbm["frac"] > fma["frac"] else fma
        return {"bound": "hbm" if lead is hbm else "alu", "achieved": lead["achieved"],
                "peak": lead["peak"], "unit": lead["unit"], "frac": lead["frac"],
                "traffic": traffic, "kernel": name,
                "launches_per_step": launches // args.steps,
                "mean_launch_ms": round(ms / launches, 4),
                "algorithmic_bytes_per_launch": round(by / launches),
                "flops_per_launch": round(flops / launches),
                "executed_flops_per_launch": round(xflops / launches),
                "updated_fraction": round(upd / (upd + kept), 4) if upd + kept else 1.0,
                "fp64_fma": fma, "hbm_moved": hbm,
                "pivot_equivalent_gbs": round(by / sec / 1e9, 1),
                "share_of_pivot_kernel_time": round(ms / kernel_ms, 4)}

    dominant = max(per_kernel, key=lambda k: per_kernel[k][1])
    roof = roofline_of(dominant)
    roof["others"] = [roofline_of(k) for k in per_kernel if k != dominant]
    line = {
        "metric": "pivots/s", "value": all_pivots / (total_ms * 1e-3), "unit": "pivots/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(wname, world),
        "lps": [n for n, *_ in lps], "pivots_per_step": pivots // args.steps,
        "tableau_gbs": round(alg_bytes / (kernel_ms * 1e-3) / 1e9, 1),
        "e2e": {"value": e2e_val, "unit": "pivots/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "roofline": roof,
        "gpu_launches": 5 * len(lps) * args.steps,
        "clocks": clk.summary(),
    }
    if wname == "lp8192":
        line.update(lp8192_extras(args, capi, torch, lps, dev_in, last[0][2], last[0][0], local))
    elif world == 1 and not args.no_cpu_baseline:
        # the whole workload, repeated until about 10 s of oracle time; the
        # paper family's LPs take thousands of pivots, so there the sample
        # stops each LP after a fixed number of them
        cores = len(os.sched_getaffinity(0))
        cap, cap1 = (200, 20) if wname == "paperset" else (None, None)
        p, t, reps = 0, 0.0, 0
        while t < 10.0 and reps < 1000:
            dp, dt = cpu_oracle_run(lps, cores, cap)
            p, t, reps = p + dp, t + dt, reps + 1
        p1, t1 = cpu_oracle_run(lps, 1, cap1)
        what = "the whole workload (4 LPs)" if cap is None else "the first %d pivots of each LP" % cap
        what1 = "the whole workload" if cap1 is None else "the first %d pivots of each LP" % cap1
        line["cpu_baseline"] = {"value": p / t, "unit": "pivots/s", "cores": cores,
                                "kind": "oracle",
                                "sample": "%s %d times, Step 1 build excluded, %.1f s"
                                          % (what, reps, t),
                                "single_thread": {"value": p1 / t1, "unit": "pivots/s",
                                                  "sample": "%s once, %.1f s" % (what1, t1)}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=15)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gbsimplex", choices=["gbsimplex", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="lp8192",
                    choices=["lp8192", "lp2048set", "paperset", "batch1024", "serve", "servespill",
                             "product"],
                    help="lp8192 is the headline line; the others report their own figures")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1804_04737_gb300 import capi

    torch.cuda.set_device(local)
    if args.workload in ("batch1024", "serve", "servespill", "product"):
        return {"batch1024": run_batch, "serve": run_serve, "servespill": run_serve_spill,
                "product": run_product}[args.workload](args, capi, torch)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    try:
        run_lpset(args, capi, torch, rank, world, local, dist)
    finally:
        if dist:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
