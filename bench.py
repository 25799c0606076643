#!/usr/bin/env python
"""Benchmark of exact echelon form + transformation over GF(p) (arXiv 1806.04211).

One step = gfe_echelon (Steps 1-3 of the Chief, with transformation) of every
matrix of the workload, inputs resident in HBM.  Metric: m*n*r / time in
GF(p) multiply-adds per second (bit multiply-adds for GF(2)), the paper's
cost model (Section 5: an alpha x beta block of rank r costs alpha*beta*r).

Default workload: the largest single-GPU configuration, bit-packed GF(2) at
n = 100000, i.e. one uniform Bernoulli(1/2) matrix and its rank-deficient
twin (product of n x 0.75n and 0.75n x n factors), seeded (synth.py).  The
plain CUDA-core comparator runs on the n = 32768 member of the same family
(at n = 100000 it would take minutes per matrix), beside the tensor-core
path on the same inputs.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--n N]

Prints ONE JSON line (rank 0).  Under torchrun every rank echelonises its own
matrices (different seeds; no data-path collective): weak scaling.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GF(p) mul-adds/s for echelon+transform vs plain GPU path; serving p50/p99"
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=100000)
    ap.add_argument("--plain-n", type=int, default=32768, help="side of the tensor-vs-plain comparison")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain CUDA-core comparator")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle cpu_baseline")
    ap.add_argument("--no-forms", action="store_true", help="skip the batched (C4) and served (C5) legs")
    ap.add_argument("--c4", type=int, default=4096, help="matrices of the batched leg")
    ap.add_argument("--c5", type=int, default=2000, help="measured requests of the serving leg")
    ap.add_argument("--c5-warmup", type=int, default=200, help="warm-up requests of the serving leg")
    ap.add_argument("--gf2-mad", action="store_true",
                    help="run only the GF(2) multiply-add comparison: bit-packed M4RM kernel vs the e4m3 tensor-core "
                         "kernel per shape, with the measured LOP3 and shared-memory load peaks")
    ap.add_argument("--single", type=int, default=0,
                    help="profiling run: one matrix of N rows (GF(2) unless --p; uniform, or --twin), one untimed and one "
                         "counted call; prints the library's launch counts and algorithmic work")
    ap.add_argument("--twin", action="store_true", help="with --single: the rank-0.75n twin")
    ap.add_argument("--p", type=int, default=2, help="with --single: the field (uint8 storage for p > 2)")
    ap.add_argument("--cols", type=int, default=0, help="with --single: columns (0: square)")
    ap.add_argument("--block", type=int, default=0, help="with --single: top-level block side (0: the table)")
    ap.add_argument("--side-tiles", type=int, default=-1,
                    help="with --single: tiles per CTA of the planner's side-stream multiply-adds (-1: default)")
    ap.add_argument("--trace", action="store_true", help="with --single: time every launch (events; the "
                                                          "multiply-add stamps itself) and group by kind and shape")
    ap.add_argument("--mad-shapes", action="store_true",
                    help="profiling run: the tensor-core multiply-add alone on the planner's GF(2) shape classes")
    ap.add_argument("--cpu-omp-worker", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--no-c3", action="store_true", help="skip the C3 tensor-vs-plain leg")
    ap.add_argument("--no-f2", action="store_true", help="skip the paper-scale 100000^2 GF(193) leg")
    return ap.parse_args()


def workload(n):
    # (p, m, n, rank-of-twin or None)
    return [(2, n, n, None), (2, n, n, (3 * n) // 4)]


def workload_name(n):
    return "C2 GF(2) bit-packed n=%d: uniform + rank-%d twin" % (n, (3 * n) // 4)


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if os.environ.get("GFE_BENCH_BACKEND", "nccl") == "nccl" else "gloo"
        if backend == "nccl":
            # each rank on its own GPU before NCCL starts: a barrier issued
            # before any device is chosen (the reference arm's) would put
            # every rank on GPU 0
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(ws, x, device):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allsum(ws, x, device):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


class Clocks:
    """nvidia-smi sampler (200 ms) running during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
            "fallback"


def union_ms(recs):
    """Length of the union of the launches' [start, end) intervals (ms)."""
    iv = sorted((r["start_ms"], r["start_ms"] + r["ms"]) for r in recs)
    tot, cs, ce = 0.0, None, None
    for s0, e0 in iv:
        if ce is None or s0 > ce:
            if ce is not None:
                tot += ce - cs
            cs, ce = s0, e0
        else:
            ce = max(ce, e0)
    return tot + (ce - cs if ce is not None else 0.0)


# DRAM bytes (read + write) of the tensor-core multiply-add per algorithmic
# byte (A, B, W read, C written), from one ncu capture of every k_mad_tc
# launch of one GF(2) 24576^2 matrix with the 6144-wide blocks of the
# n = 100000 policy (dram__bytes_read.sum + dram__bytes_write.sum over 5816
# launches: 38.64 GB; the library's algorithmic bytes for the same launches:
# 40.47 GB), with the current kernel (banded tile order, GF(2) epilogue).
# The full-size step is too large to capture; its launches are scaled by
# their algorithmic bytes.
MAD_TRAFFIC_PER_ALG_BYTE = 0.955


def roofline(prof, codec_bytes, trace):
    """Roofline of the dominant kernel kind of the timed region.  The
    planner runs multiply-adds on several streams at once, so per-launch
    times overlap; the rate is the launches' algorithmic flops over the time
    at least one of them ran (the union of their intervals, which the
    tensor-core multiply-add stamps itself with %globaltimer)."""
    pk, src = peaks()
    kinds = ["mad_tensor", "mad_plain"]
    k = max(kinds, key=lambda x: prof["ms"][x])
    ms, madds, launches = prof["ms"][k], prof["madds"][k], prof["timed"][k]
    if ms <= 0 or launches == 0:
        return None
    recs = [r for r in trace if r["kind"] == k]
    um = union_ms(recs) if recs and len(recs) == launches else None
    if k == "mad_tensor":
        # fp8 (e4m3) MMA: 2x the measured dense bf16 rate (nominal 4.5 / 2.25
        # PFLOP/s); bf16 storage runs at the bf16 rate.  Sustained figure:
        # the kernel is timed inside a long step.
        ratio = 2.0 if codec_bytes == 1 else 1.0
        peak = pk["bf16_tflops_sustained"] * ratio
        achieved = 2.0 * madds / ((um if um else ms) * 1e-3) / 1e12
        alg_bytes = prof["bytes"][k] / max(prof["launches"][k], 1)
        return {"kernel": "k_mad_tc<%s> (tcgen05)" % ("e4m3" if codec_bytes == 1 else "bf16"), "bound": "tensor",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": MAD_TRAFFIC_PER_ALG_BYTE * alg_bytes,
                "traffic_source": "bytes per launch: %.3f x the algorithmic bytes per launch, the ratio from an ncu "
                                  "capture of every multiply-add of one 24576^2 matrix with the same 6144 blocks"
                                  % MAD_TRAFFIC_PER_ALG_BYTE,
                "peak_source": "%s bf16 sustained x %.0f" % (src, ratio),
                "denominator": ("union of the launches' intervals (%s clock)" % recs[0].get("clock", "event"))
                if um else "sum of launch times",
                "union_ms": um, "sum_of_launch_ms": ms,
                "launches": launches, "avg_launch_ms": ms / launches,
                "achieved_per_launch_avg": 2.0 * madds / (ms * 1e-3) / 1e12,
                "frac_per_launch_avg": 2.0 * madds / (ms * 1e-3) / 1e12 / peak,
                "algorithmic_flops_per_launch": 2.0 * madds / launches,
                "algorithmic_bytes_per_launch": prof["bytes"][k] / max(prof["launches"][k], 1)}
    # CUDA-core multiply-add: 2 integer ops (one IMAD) per multiply-add; peak =
    # 152 SMs x 128 INT32 lanes x the maximum SM clock x 2 ops per IMAD
    peak = 152 * 128 * pk.get("sm_max_mhz", 2070.0) * 1e6 * 2 / 1e12
    achieved = 2.0 * madds / (ms * 1e-3) / 1e12
    return {"kernel": "k_mad_plain (CUDA-core int32)", "bound": "alu", "achieved": achieved, "peak": peak,
            "unit": "TOP/s", "frac": achieved / peak, "traffic": None,
            "peak_source": "derived: 152 SM x 128 INT32 lanes x %s MHz x 2" % pk.get("sm_max_mhz", 2070.0),
            "launches": launches, "avg_launch_ms": ms / launches}


def host_info():
    """The timing host: logical CPUs and CPU model (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for ln in f:
                    if ln.lower().startswith(("model name", "cpu part")):
                        model = ln.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    import platform
    return {"nproc": os.cpu_count(), "cpu_model": model or platform.processor() or "unknown",
            "machine": platform.machine()}


CPU_SAMPLE = 8192


def cpu_omp_worker(ns):
    """Runs in a child process (OMP_WAIT_POLICY=active, all cores): the
    OpenMP variant of the oracle's GF(2) elimination on the sample; prints
    one JSON line."""
    from oracle import oracle as O
    from paper_1806_04211_gb300 import synth
    A = synth.matrix(2, ns, ns, seed=1).numpy()
    O.echelon_gf2_omp(A[:256], 256, ns)  # thread pool up
    t = time.perf_counter()
    r = O.echelon_gf2_omp(A, ns, ns)
    dt = time.perf_counter() - t
    print(json.dumps({"seconds": dt, "rank": r["rank"], "threads": O.omp_threads()}), flush=True)


def cpu_baseline(n):
    """The oracle, as it stands, on a bounded sample: a uniform GF(2) matrix
    of side n_s = min(n, 8192) drawn like the workload's, single-threaded
    (about 5 s), and the OpenMP variant of the same elimination on all host
    cores (a child process) on the same sample."""
    from oracle import oracle as O
    from paper_1806_04211_gb300 import synth
    ns = min(n, CPU_SAMPLE)
    A = synth.matrix(2, ns, ns, seed=1).numpy()
    t = time.perf_counter()
    r = O.echelon_gf2(A, ns, ns, want_E=False, want_T=False)
    dt = time.perf_counter() - t
    out = {"value": ns * ns * r["rank"] / dt, "unit": "mul-adds/s", "cores": 1, "kind": "oracle",
           "sample": "one uniform GF(2) %dx%d matrix of the workload's distribution (bit-packed oracle, "
                     "echelon + transformation), %.1f s" % (ns, ns, dt),
           "host": host_info()}
    try:
        env = dict(os.environ, OMP_WAIT_POLICY="active")
        proc = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-omp-worker", str(ns)],
                              capture_output=True, text=True, timeout=600, env=env, cwd=ROOT)
        d = json.loads(proc.stdout.strip().splitlines()[-1])
        assert d["rank"] == r["rank"]
        out["openmp"] = {"value": ns * ns * d["rank"] / d["seconds"], "unit": "mul-adds/s",
                         "cores": d["threads"], "kind": "oracle algorithm, OpenMP (rows in parallel per pivot)",
                         "seconds": d["seconds"], "sample": "the same matrix"}
    except Exception as e:  # the single-threaded figure stands on its own
        out["openmp"] = {"unavailable": repr(e)[:200]}
    return out


def c4_matrices(count, seed=1):
    from paper_1806_04211_gb300 import synth
    return synth.c4_specs(count, seed)


def c5_requests(count, seed=1):
    from paper_1806_04211_gb300 import synth
    return synth.c5_specs(count, seed)


C4_WORKERS = 16  # planner workers for the matrices above the one-launch kernels' work cut-off


def bench_batched(dev, count, plain_count=512, clock_index=None):
    """C4: gfe_batch_echelon over `count` matrices of the seeded draw (median
    of three calls after one untimed call) vs the plain per-matrix path on the
    first `plain_count`.  The library sends a matrix of side <= 2048 and work
    m n min(m,n) <= 4e9 (GF(2): a 16th of it) to its one-launch kernels (one
    thread block per matrix) and the rest to its blocked planner."""
    import torch
    from paper_1806_04211_gb300 import gfe, synth
    specs = c4_matrices(count)
    mats = [(synth.matrix(p, m, n, seed=5000 + i, rank=rk, device=dev), p, n) for i, (p, m, n, rk) in enumerate(specs)]
    units = float(sum(m * n * min(m, n) for p, m, n, rk in specs))
    one_launch = sum(1 for p, m, n, rk in specs
                     if m * n * min(m, n) / (16 if p == 2 else (2.5 if p <= 13 else 1)) <= 4e9)
    gfe.batch_echelon(mats, workers=C4_WORKERS)
    torch.cuda.synchronize()
    times = []
    clocks = Clocks(clock_index) if clock_index is not None else None
    if clocks:
        clocks.start()
    for _ in range(3):
        t = time.perf_counter()
        res = gfe.batch_echelon(mats, workers=C4_WORKERS)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t)
    clk = clocks.stop() if clocks else None
    tb = sorted(times)[1]
    madds = float(sum(m * n * d["rank"] for (p, m, n, rk), d in zip(specs, res)))
    pc = min(plain_count, count)
    t = time.perf_counter()
    for A, p, n in mats[:pc]:
        gfe.echelon(A, p, n=n, impl="plain")
    torch.cuda.synchronize()
    tp = time.perf_counter() - t
    return {"matrices": count, "of": 4096, "batched_matrices_per_s": count / tb, "plain_matrices_per_s": pc / tp,
            "speedup": (tp / pc) / (tb / count), "batched_madds_per_s": madds / tb, "wall_ms": tb * 1e3,
            "wall_ms_runs": [x * 1e3 for x in times], "clocks": clk, "workers": C4_WORKERS,
            "one_launch_matrices": one_launch,
            "planner_matrices": count - one_launch, "plain_sample": pc,
            "sample": "seeded C4 draw, %d matrices (sum m*n*min(m,n) = %.3g), median of 3 calls; plain path "
                      "timed on the first %d" % (count, units, pc)}


C5_WORKERS = 12


def bench_serving(dev, warm, count, cap=120 << 30):
    """C5: Poisson arrivals at 0.5x and 0.8x the saturated rate; latency =
    submit to result ready (host clock).  Baseline: the same trace served one
    request at a time by the plain path (service times measured, queue replayed)."""
    import numpy as np
    import torch
    from paper_1806_04211_gb300 import gfe, synth
    reqs = c5_requests(warm + count)
    mats = [(synth.matrix(p, n, n, seed=7000 + i, rank=rk, device=dev), p, n) for i, (p, n, rk) in enumerate(reqs)]
    torch.cuda.synchronize()

    def serve(rate, order):
        rng = np.random.RandomState(3)
        lat, t0 = [], time.perf_counter()
        with gfe.Server(cap, workers=C5_WORKERS) as srv:
            tickets, nxt = [], t0
            for i in order:
                A, p, n = mats[i]
                now = time.perf_counter()
                if rate and nxt > now:
                    time.sleep(nxt - now)
                tickets.append(srv.submit(A, p, n if p == 2 else None))
                nxt += rng.exponential(1.0 / rate) if rate else 0.0
            for t in tickets:
                lat.append(srv.wait(t)["latency_us"] / 1e3)
        return lat, time.perf_counter() - t0

    serve(0, range(warm))                                    # warm-up requests
    meas = list(range(warm, warm + count))
    _, tsat = serve(0, meas)                                 # saturated: all at once
    sat = count / tsat
    out = {"requests": count, "warmup_requests": warm, "saturated_matrices_per_s": sat, "hbm_cap_gb": cap >> 30,
           "workers": C5_WORKERS}
    for frac in (0.5, 0.8):
        lat, tt = serve(frac * sat, meas)
        out["at_%.1fx" % frac] = {"rate": frac * sat, "matrices_per_s": count / tt,
                                  "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99))}
    # serial plain baseline: service times, then the same arrival trace replayed
    svc = []
    for i in meas:
        A, p, n = mats[i]
        torch.cuda.synchronize()
        t = time.perf_counter()
        gfe.echelon(A, p, n=n if p == 2 else None, impl="plain")
        torch.cuda.synchronize()
        svc.append(time.perf_counter() - t)
    for frac in (0.5, 0.8):
        rng = np.random.RandomState(3)
        rate = frac * sat
        arr, tcur, lat = 0.0, 0.0, []
        for k, sv in enumerate(svc):
            start = max(arr, tcur)
            tcur = start + sv
            lat.append((tcur - arr) * 1e3)
            arr += rng.exponential(1.0 / rate)
        out["plain_serial_at_%.1fx" % frac] = {"p50_ms": float(np.percentile(lat, 50)),
                                               "p99_ms": float(np.percentile(lat, 99)),
                                               "matrices_per_s": count / max(tcur, arr)}
    out["plain_serial_saturated_matrices_per_s"] = count / sum(svc)
    return out


def bench_c3(dev):
    """C3: the exact tensor-core form vs the CUDA-core modular form on the same
    inputs -- 32768^2 over GF(7) and 20000 x 50000 over GF(251), each uniform
    and a rank-0.6*min twin (one seed each)."""
    import torch
    from paper_1806_04211_gb300 import gfe, synth
    out = {}
    for p, m, n in [(7, 32768, 32768), (251, 20000, 50000)]:
        for rk in (None, int(0.6 * min(m, n))):
            A = synth.matrix(p, m, n, seed=11, rank=rk, device=dev)
            row = {}
            for impl in ("tensor", "plain"):
                gfe.echelon(A, p, impl=impl) if impl == "tensor" else None
                torch.cuda.synchronize()
                t = time.perf_counter()
                d = gfe.echelon(A, p, impl=impl)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t
                row[impl] = {"seconds": dt, "madds_per_s": m * n * d["rank"] / dt}
            key = "GF(%d) %dx%d %s" % (p, m, n, "uniform" if rk is None else "rank-%d twin" % rk)
            row["speedup"] = row["plain"]["seconds"] / row["tensor"]["seconds"]
            out[key] = row
            del A
    return out


GF2_SHAPES = [  # (m, n, k): planner shapes (leaf-level, UpdateRow, ClearDown) and large squares
    (1024, 2816, 256), (3072, 3072, 3072), (3072, 30720, 3072), (6144, 6144, 6144), (6144, 92160, 6144),
    (8192, 16384, 2048), (16384, 16384, 16384)]


def bench_gf2_mad(dev, reps=5):
    """GF(2) job MAD on one shape at a time: the bit-packed kernel
    (gfe_mad_gf2, CUDA events around the launch) against the tensor-core
    kernel on e4m3 operands (the planner's representation; device-stamped
    duration of k_mad_tc alone, without gfe_mad's conversions).  Median of
    `reps` after one warm-up; inputs larger than L2 for all but the smallest."""
    import torch
    from paper_1806_04211_gb300 import gfe, synth
    pk = gfe.gf2_peaks()
    out = {"peaks": pk, "shapes": []}
    for m, n, k in GF2_SHAPES:
        Aw = synth.bernoulli_gf2(m, k, 3, 1, device=dev)
        Bw = synth.bernoulli_gf2(k, n, 3, 2, device=dev)
        C = torch.empty((m, synth.gf2_words_per_row(n)), dtype=torch.int64, device=dev)
        gfe.mad_gf2(None, Aw, Bw, n, k, out=C)
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            gfe.mad_gf2(None, Aw, Bw, n, k, out=C)
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        t_bits = statistics.median(ts)
        ref_bits = C
        A8 = synth.unpack_gf2(Aw, k)
        B8 = synth.unpack_gf2(Bw, n)
        del Aw, Bw
        C8 = gfe.mad(None, A8, B8, 2)
        ts = []
        for _ in range(reps):
            gfe.profile_enable(True, kinds=["mad_tensor"])
            gfe.profile_read(True)
            gfe.trace_enable(1 << 12)
            gfe.mad(None, A8, B8, 2, out=C8)
            torch.cuda.synchronize()
            prof = gfe.profile_read(True)
            gfe.trace_enable(0)
            gfe.profile_enable(False)
            ts.append(prof["ms"]["mad_tensor"])
        t_tc = statistics.median(ts)
        same = bool(torch.equal(synth.pack_gf2(C8), ref_bits))
        madds = float(m) * n * k
        nb = n / 8.0
        lookups = m * ((k + 7) // 8) * nb                      # one n-bit entry per row and slice
        builds = -(-m // 512) * ((k + 7) // 8) * 256 * nb      # 256 entries per slice and 512-row tile
        out["shapes"].append({
            "m": m, "n": n, "k": k, "equal": same,
            "bits_m4rm": {"ms": t_bits, "madds_per_s": madds / (t_bits * 1e-3),
                          "frac_of_alu_lop3": madds / (t_bits * 1e-3) / pk["gf2_madds_per_s_alu"],
                          "smem_bytes": lookups + builds,
                          "frac_of_lds": (lookups + builds) / (t_bits * 1e-3) / pk["lds_bytes_per_s"]},
            "e4m3_tensor": {"ms": t_tc, "madds_per_s": madds / (t_tc * 1e-3)},
            "faster": "bits_m4rm" if t_bits < t_tc else "e4m3_tensor"})
        del A8, B8, C8, C, ref_bits
        gfe.release_workspace()
        torch.cuda.empty_cache()
    return out


def bench_paper_scale(dev):
    """The paper's 200000^2 GF(193) experiment (Section 5) at the largest side
    that fits one GPU with the transformation: 100000^2, uniform; one
    untimed call, then one timed call (host clock around a synchronize)."""
    import torch
    from paper_1806_04211_gb300 import gfe, synth
    n = 100000
    A = synth.matrix(193, n, n, seed=1, device=dev)
    gfe.echelon(A, 193)
    torch.cuda.synchronize()
    t = time.perf_counter()
    d = gfe.echelon(A, 193)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t
    r = d["rank"]
    del d, A
    gfe.release_workspace()
    torch.cuda.empty_cache()
    return {"workload": "GF(193) %dx%d uniform, echelon + transformation" % (n, n), "seconds": dt, "rank": r,
            "madds_per_s": float(n) * n * r / dt,
            "paper": "200000^2 GF(193): 445 min on 64 cores (Section 5), about 3.0e11 mul-adds/s"}


def union_of(iv):
    iv = sorted(iv)
    tot, cs, ce = 0.0, None, None
    for s0, e0 in iv:
        if ce is None or s0 > ce:
            if ce is not None:
                tot += ce - cs
            cs, ce = s0, e0
        else:
            ce = max(ce, e0)
    return tot + (ce - cs if ce is not None else 0.0)


def run_single(args, dev):
    """One GF(2) matrix of the C2 family through the batched entry point (one
    worker): an untimed call, then a counted one (and with --trace a traced
    one: per-kind unions of launch intervals, multiply-add shape classes)."""
    import collections
    import torch
    from paper_1806_04211_gb300 import gfe, synth
    m, p = args.single, args.p
    n = args.cols or m
    if args.block:
        gfe.set_block_policy(args.block, args.block)
    if args.side_tiles >= 0:
        gfe._check(gfe.lib().gfe_set_side_tiles(args.side_tiles))
    A = synth.matrix(p, m, n, seed=1, rank=(3 * min(m, n)) // 4 if args.twin else None, device=dev)
    arg = (A, p, n) if p == 2 else (A, p)
    gfe.batch_echelon([arg], workers=1)
    torch.cuda.synchronize()
    gfe.profile_enable(True, kinds=["other"])  # counts only: no kind is timed
    gfe.profile_read(True)
    t = time.perf_counter()
    d = gfe.batch_echelon([arg], workers=1)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t
    pr = gfe.profile_read(True)
    gfe.profile_enable(False)
    out = {"p": p, "m": m, "n": n, "rank": d[0]["rank"], "block": args.block or gfe.lib().gfe_auto_block(p, m, n),
           "seconds": dt, "madds_per_s": float(m) * n * d[0]["rank"] / dt,
           "launches": pr["launches"], "madds": pr["madds"], "algorithmic_bytes": pr["bytes"],
           "host_syncs": pr["host_syncs"]}
    if args.trace:
        gfe.profile_enable(True)
        gfe.profile_read(True)
        gfe.trace_enable(1 << 21)
        gfe.batch_echelon([arg], workers=1)
        torch.cuda.synchronize()
        tr = gfe.trace_read(True)
        gfe.trace_enable(0)
        gfe.profile_enable(False)
        by = collections.defaultdict(list)
        for r in tr:
            by[r["kind"]].append((r["start_ms"], r["start_ms"] + r["ms"]))
        out["union_ms_by_kind"] = {k: union_of(v) for k, v in by.items()}
        out["union_ms_all"] = union_of([x for v in by.values() for x in v])

        def bucket(x):
            for lim in (64, 256, 1024, 2048, 4096, 6144, 12288):
                if x <= lim:
                    return str(lim)
            return "more"
        cls = collections.defaultdict(lambda: [0, 0.0, 0.0])
        for r in tr:
            if r["kind"] == "mad_tensor":
                c = cls["m<=%s n<=%s k<=%s" % (bucket(r["m"]), bucket(r["n"]), bucket(r["k"]))]
                c[0] += 1
                c[1] += r["ms"]
                c[2] += 2.0 * r["m"] * r["n"] * r["k"]
        out["mad_classes"] = sorted(({"shape": k, "launches": v[0], "ms": v[1],
                                      "tflops": v[2] / (v[1] * 1e-3) / 1e12 if v[1] else 0.0}
                                     for k, v in cls.items()), key=lambda x: -x["ms"])
    gfe.set_block_policy()
    gfe._check(gfe.lib().gfe_set_side_tiles(4))
    return out


MAD_SHAPES = [(1024, 256, 256), (1024, 1024, 256), (1024, 6144, 256), (256, 1024, 256), (6144, 6144, 64),
              (6144, 6144, 8), (6144, 6144, 6144), (6144, 92160, 6144), (1024, 92160, 256), (128, 256, 64)]


def run_mad_shapes(dev, reps=7):
    """The tensor-core multiply-add alone (GF(2) e4m3 codes, W given) on the
    planner's shape classes: median device-stamped duration of k_mad_tc."""
    import torch
    from paper_1806_04211_gb300 import gfe, synth
    out = []
    for m, n, k in MAD_SHAPES:
        A = synth.uniform_u8(m, k, 2, 1, 1, device=dev)
        B = synth.uniform_u8(k, n, 2, 1, 2, device=dev)
        W = synth.uniform_u8(m, n, 2, 1, 3, device=dev)
        C = torch.empty_like(W)
        gfe.mad(W, A, B, 2, out=C)
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            gfe.profile_enable(True, kinds=["mad_tensor"])
            gfe.profile_read(True)
            gfe.trace_enable(1 << 10)
            gfe.mad(W, A, B, 2, out=C)
            torch.cuda.synchronize()
            pr = gfe.profile_read(True)
            gfe.trace_enable(0)
            gfe.profile_enable(False)
            ts.append(pr["ms"]["mad_tensor"] * 1e3)
        t = statistics.median(ts)
        out.append({"m": m, "n": n, "k": k, "kernel_us": t, "tflops": 2.0 * m * n * k / (t * 1e-6) / 1e12})
        del A, B, W, C
    gfe.release_workspace()
    return out


def run_reference(args, ws, rank):
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_1806_04211_gb300 import synth
    ns = min(args.n, 4096)
    A = synth.matrix(2, ns, ns, seed=1).numpy()
    for _ in range(args.warmup):
        O.echelon_gf2(A, ns, ns)
    times, units = [], 0.0
    for _ in range(args.steps):
        t = time.perf_counter()
        r = O.echelon_gf2(A, ns, ns)
        times.append(time.perf_counter() - t)
        units += ns * ns * r["rank"]
    tot = sum(times)
    v = units / tot
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "mul-adds/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64 (bit-packed GF(2))",
            "data": "synthetic (seeded SplitMix64)",
            "config": {"workload": workload_name(args.n), "sample": "uniform %dx%d per step" % (ns, ns)},
            "cpu_baseline": {"value": v, "unit": "mul-adds/s", "cores": 1, "kind": "oracle",
                             "sample": "uniform GF(2) %dx%d, bit-packed oracle, 1 thread" % (ns, ns),
                             "host": host_info()},
            "e2e": {"value": v, "unit": "mul-adds/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.cpu_omp_worker:
        cpu_omp_worker(args.cpu_omp_worker)
        return
    ws, rank, local = dist_setup()
    if ws > 1:
        # the side legs (plain comparator, C4, C5, C3, paper scale) describe
        # one GPU and are reported by the single-GPU run; a multi-GPU run times
        # the headline alone, so the GPUs it holds are not kept waiting
        args.no_plain = args.no_forms = args.no_c3 = args.no_f2 = True
    if args.impl == "reference":
        run_reference(args, ws, rank)
        barrier(ws)
        return
    import torch
    from paper_1806_04211_gb300 import gfe, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    if args.gf2_mad or args.single or args.mad_shapes:
        if rank == 0:
            if args.gf2_mad:
                print(json.dumps({"gf2_mad": bench_gf2_mad(dev)}), flush=True)
            if args.single:
                print(json.dumps({"single": run_single(args, dev)}), flush=True)
            if args.mad_shapes:
                print(json.dumps({"mad_shapes": run_mad_shapes(dev)}), flush=True)
        barrier(ws)
        return

    def make_insts(n):
        out = []
        for idx, (p, m, nn, rk) in enumerate(workload(n)):
            A = synth.matrix(p, m, nn, seed=1 + 1000 * rank + idx, rank=rk, device=dev)
            out.append((p, m, nn, A))
        return out

    insts = make_insts(args.n)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    codec_bytes = 1  # GF(2) entries are stored as e4m3 centred residues inside the library

    def step(impl, insts):
        # the tensor-core path runs the workload's matrices through the
        # batched entry point (concurrent workers); the plain comparator is
        # the per-matrix path, one call after the other
        units = 0.0
        if impl == "plain":
            for p, m, n, A in insts:
                d = gfe.echelon(A, p, n=n, impl=impl)
                units += m * n * d["rank"]
            return units
        res = gfe.batch_echelon([(A, p, n) for p, m, n, A in insts], workers=len(insts))
        for (p, m, n, A), d in zip(insts, res):
            units += m * n * d["rank"]
        return units

    def timed(impl, insts, steps):
        per, units = [], 0.0
        barrier(ws)
        torch.cuda.synchronize()
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            units += step(impl, insts)
            e1.record(stream)
            e1.synchronize()
            per.append(e0.elapsed_time(e1))
        torch.cuda.synchronize()
        barrier(ws)
        return per, units

    for _ in range(args.warmup):
        step("tensor", insts)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    gfe.profile_enable(True, kinds=["mad_tensor", "mad_plain"])
    gfe.profile_read(True)
    gfe.trace_enable(1 << 21)
    per, units = timed("tensor", insts, args.steps)
    prof = gfe.profile_read(True)
    trace = gfe.trace_read(True)
    gfe.trace_enable(0)
    gfe.profile_enable(False)
    clk = clocks.stop()
    tot_ms = allmax(ws, sum(per), dev)
    all_units = allsum(ws, units, dev)
    value = all_units / (tot_ms * 1e-3)
    launches = sum(prof["launches"].values())

    # end to end through the public API with host buffers: every step copies
    # its inputs from pinned host memory, echelonises them and copies every
    # output (rank, pivots, R, M, K) back to pinned host memory.  As a
    # throughput user would, the copies run on a copy stream and overlap the
    # neighbouring steps' compute: step s+1's inputs go up (into the other
    # of two device input sets) and step s-1's outputs come down while step
    # s computes.  The timed region runs from the first copy to the last.
    host_in = [(p, m, n, A.cpu().pin_memory()) for p, m, n, A in insts]
    dev_in = [[torch.empty_like(A) for p, m, n, A in insts] for _ in range(2)]
    # pinned host buffers for every output (shapes from one untimed run)
    res0 = gfe.batch_echelon([(A, p, n) for p, m, n, A in insts], workers=len(insts))
    host_out = [[torch.empty(o.shape, dtype=o.dtype).pin_memory() for o in (d["ups"], d["rho"], d["R"], d["M"], d["K"])]
                for d in res0]
    del res0
    copy_st = torch.cuda.Stream()
    in_ready = [torch.cuda.Event(), torch.cuda.Event()]
    # with copies in flight beside the compute the workers sleep in their
    # waits (GFE_WAIT_BLOCK): polling workers made the concurrent copies about
    # three times slower and the steps 5-15% slower on GB300, while sleeping
    # costs about 1.3% when nothing else runs
    gfe.set_wait_policy("block")

    def upload(k):
        with torch.cuda.stream(copy_st):
            for buf, (p, m, n, Ah) in zip(dev_in[k], host_in):
                buf.copy_(Ah, non_blocking=True)
            in_ready[k].record(copy_st)

    e2e_units, h2d, d2h = 0.0, 0, 0
    barrier(ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    upload(0)
    for s_ in range(args.steps):
        cur = s_ % 2
        stream.wait_event(in_ready[cur])
        if s_ + 1 < args.steps:
            upload(1 - cur)  # the other input set: its step has returned, so it is free
        flush.zero_()
        res = gfe.batch_echelon([(buf, p, n) for buf, (p, m, n, Ah) in zip(dev_in[cur], host_in)],
                                workers=len(host_in))
        done = torch.cuda.Event()
        done.record(stream)
        with torch.cuda.stream(copy_st):
            copy_st.wait_event(done)
            for (p, m, n, Ah), d, hs in zip(host_in, res, host_out):
                outs = [d["ups"], d["rho"], d["R"], d["M"], d["K"]]
                for h, o in zip(hs, outs):
                    h.copy_(o, non_blocking=True)
                    o.record_stream(copy_st)  # its memory is not reused before the copy is done
                e2e_units += m * n * d["rank"]
                h2d += Ah.numel() * Ah.element_size()
                d2h += 8 + sum(o.numel() * o.element_size() for o in outs)
        del res
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t0) * 1e3
    gfe.set_wait_policy("auto")
    del dev_in
    e2e_ms = allmax(ws, e2e_ms, dev)
    e2e_units = allsum(ws, e2e_units, dev)
    del insts, host_in, host_out
    gfe.release_workspace()
    torch.cuda.empty_cache()
    print("main leg: %.4g mul-adds/s, %.1f ms per step; e2e %.4g" % (value, tot_ms / args.steps,
                                                                     e2e_units / (e2e_ms * 1e-3)),
          file=sys.stderr, flush=True)

    # the plain CUDA-core path (the comparator the metric names) beside the
    # tensor-core path, on the same inputs of a smaller member of the family
    plain = None
    if not args.no_plain:
        pinsts = make_insts(args.plain_n)
        step("tensor", pinsts)
        tper, tunits = timed("tensor", pinsts, 1)
        pper, punits = timed("plain", pinsts, 1)
        tt, pt = allmax(ws, sum(tper), dev), allmax(ws, sum(pper), dev)
        plain = {"workload": workload_name(args.plain_n), "value": allsum(ws, punits, dev) / (pt * 1e-3),
                 "unit": "mul-adds/s", "ms_per_step": pt,
                 "tensor_same_inputs": {"value": allsum(ws, tunits, dev) / (tt * 1e-3), "ms_per_step": tt},
                 "speedup": pt / tt}
        del pinsts
        gfe.release_workspace()
        torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_baseline(args.n)
    batched = served = c3 = None
    if rank == 0 and not args.no_forms:  # the CUDA-core forms first, before the long tensor-core C3 leg
        batched = bench_batched(dev, args.c4, clock_index=local)
        gfe.release_workspace()
        torch.cuda.empty_cache()
        served = bench_serving(dev, args.c5_warmup, args.c5)
        gfe.release_workspace()
        torch.cuda.empty_cache()
    if rank == 0 and not args.no_c3:
        c3 = bench_c3(dev)
    f2 = None
    if rank == 0 and not args.no_f2:
        gfe.release_workspace()
        torch.cuda.empty_cache()
        try:
            f2 = bench_paper_scale(dev)
        except Exception as e:  # reported, not fatal: the headline above stands
            f2 = {"error": repr(e)[:300]}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "mul-adds/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "e4m3 operands, fp32 exact-integer accumulation",
                "data": "synthetic (seeded SplitMix64; uniform + low-rank twin)",
                "config": {"workload": workload_name(args.n), "p": 2, "n": args.n, "matrices_per_gpu": len(workload(args.n)),
                           "l2": "flushed between steps (256 MiB write)", "parallelism": "independent matrices per GPU"},
                "roofline": roofline(prof, codec_bytes, trace),
                "plain_gpu_path": plain,
                "cpu_baseline": cpu,
                "e2e": {"value": e2e_units / (e2e_ms * 1e-3), "unit": "mul-adds/s",
                        "h2d_bytes_per_step": h2d // max(args.steps, 1), "d2h_bytes_per_step": d2h // max(args.steps, 1),
                        "copies": "pinned host buffers; a copy stream overlaps each step's uploads and downloads "
                                  "with the neighbouring steps' compute; timed from the first upload to the last "
                                  "download",
                        "wait_policy": "block (gfe_set_wait_policy: the workers sleep in their waits while copies "
                                       "run beside them)"},
                "tensor_vs_plain_C3": c3,
                "batched_C4": batched,
                "served_C5": served,
                "paper_scale_f2": f2,
                "clocks": clk,
                "gpu_launches": launches,
                "gpu_launches_per_step": launches / max(args.steps, 1),
                "profile": {"ms": prof["ms"], "launches": prof["launches"], "host_syncs": prof["host_syncs"],
                            "host_syncs_per_step": prof["host_syncs"] / max(args.steps, 1)}}
        print(json.dumps(line), flush=True)
    barrier(ws)


if __name__ == "__main__":
    main()
