#!/usr/bin/env python3
"""Benchmark of the hard-leaf sieve (S2_hard) and pi(x) on GB300.

One step = one S2_hard(x, y, c) evaluation through the C ABI, x = 10^18,
y = 20 * iroot3(x) = 2*10^7, c = 5: the whole hard-leaf path (segment
schedule, sieve + leaf resolution, carry scan, int128 combine).  The metric
is sieved integers per second, z / t with z = x / y the span of the sieve.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 runs one replica per GPU (torchrun), each doing the full workload; the
hard-leaf sieve has no exchange step, so ranks never talk except for the
final max-over-ranks timing.  --impl reference times the CPU oracle
(single-threaded C) on a bounded sample of the same workload instead.
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
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pi(x) wall time at 1e16/1e18 + sieved ints/s and batched queries/s vs plain, bit-exact"
UNIT = "sieved ints/s"
X = 10 ** 18
ALPHA = 20
C = 5
PI_1E16 = 279238341033925      # Table 1
PI_1E18 = 24739954287740860    # Table 1
# oracle sample: the same hard-leaf sieve of [1, z] at a size the CPU finishes
ORACLE_X = 10 ** 12


def iroot3(n):
    r = int(round(n ** (1.0 / 3)))
    while r ** 3 > n:
        r -= 1
    while (r + 1) ** 3 <= n:
        r += 1
    return r


def workload():
    y = ALPHA * iroot3(X)
    return {"x": X, "y": y, "c": C, "z": X // y}


def config(seg_bytes, parallelism="replicas"):
    w = workload()
    return {"workload": "S2_hard hard-leaf sieve x=%.0e y=%d*iroot3(x)=%d c=%d (one evaluation per step)"
                        % (w["x"], ALPHA, w["y"], C),
            "x": w["x"], "y": w["y"], "z": w["z"], "c": C, "seg_bytes": seg_bytes,
            "l2": "flushed between timed steps (256 MiB write)", "parallelism": parallelism}


def dist_env():
    return int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), \
        int(os.environ.get("LOCAL_RANK", "0"))


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [t.strip() for t in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def profile_traffic():
    """DRAM bytes per launch of the sieve kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    try:
        with open(os.path.join(ROOT, "profiles", "hard_sieve_traffic.json")) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    h = hashlib.sha256()
    for name in ("pc_hard.cu", "pc_sieve.cuh", "pc_common.cuh"):
        with open(os.path.join(ROOT, "paper_1503_01839_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    if rec.get("source_sha256") != h.hexdigest() or rec.get("x") != X or rec.get("y") != workload()["y"]:
        return None
    return rec.get("dram_bytes_per_launch")


# Algorithmic unit costs of the roofline models (stated in the design notes).  The
# hard-leaf sieve: per crossing one 32-bit shared-memory read-modify-write and about 4
# integer operations; per (segment, prime) step one 64-bit reduction (about 16 integer
# operations); per hard leaf one 64-by-32 division (about 16) and a count of the set
# bits below u: the block prefix plus on average half of a 1024-bit block (16 words:
# 16 bank accesses and about 32 integer operations) -> 17 accesses and 48 operations.
HARD_SMEM = {"crossing": 1.0, "leaf": 17.0}
HARD_INT = {"crossing": 4.0, "step": 16.0, "leaf": 48.0}
# Easy leaves: per leaf resolved alone one division by a 32-bit reciprocal (two 32x32-bit
# products, a shift and a remainder test: 8), the odd-number pi record's index and bit (3),
# its popcount and sum (3) and the leaf's term (2); per run of clustered leaves, taken by its
# pi value l, the same: one division by p_l, one lookup, and the run's term from the
# neighbouring l's lookup (16).  P2: one shared-memory atomic per crossing.
EASY_INT = {"leaf": 16.0, "run": 16.0}
P2_SMEM = {"crossing": 1.0}


def roofline_term(work, ms, peak_per_s, unit):
    achieved = work / (ms / 1000.0)
    return {"work": work, "achieved": achieved / 1e9, "peak": peak_per_s / 1e9, "unit": unit,
            "frac": achieved / peak_per_s}


def ncu_summary(name, sources):
    """The committed ncu counters of a kernel (profiles/<name>_ncu.json), if they were
    taken on the current source of the files that define it."""
    try:
        with open(os.path.join(ROOT, "profiles", name + "_ncu.json")) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    h = hashlib.sha256()
    for src in sources:
        with open(os.path.join(ROOT, "paper_1503_01839_gb300", "csrc", src), "rb") as f:
            h.update(f.read())
    if rec.get("source_sha256") != h.hexdigest():
        return None
    return rec


def hard_roofline(st, sieve_ms, n_sm, f_mhz, traffic):
    """Both terms of the shared-memory / INT32 model of the hard-leaf sieve:
    t_roof = max(bank accesses / (32 N_SM f), integer ops / (128 N_SM f))."""
    clears, leaves, steps = float(st["clears"]), float(st["hard_leaves"]), float(st["steps"])
    f = f_mhz * 1e6
    smem = roofline_term(HARD_SMEM["crossing"] * clears + HARD_SMEM["leaf"] * leaves, sieve_ms, 32.0 * n_sm * f,
                         "G smem-bank-accesses/s")
    smem["per_unit"] = "1 per crossing, 17 per hard leaf"
    ints = roofline_term(HARD_INT["crossing"] * clears + HARD_INT["step"] * steps + HARD_INT["leaf"] * leaves,
                         sieve_ms, 128.0 * n_sm * f, "G int32-ops/s")
    ints["per_unit"] = "4 per crossing, 16 per (segment, prime) step, 48 per hard leaf"
    top = smem if smem["frac"] >= ints["frac"] else ints
    out = {"bound": "smem" if top is smem else "alu", "achieved": top["achieved"], "peak": top["peak"],
           "unit": top["unit"], "frac": top["frac"], "traffic": traffic, "kernel": "hard_sieve_kernel",
           "kernel_ms": sieve_ms, "terms": {"smem": smem, "int32": ints},
           "peak_basis": "32 banks / 128 INT32 lanes x %d SMs x %.0f MHz (max SM clock, MEASURED_PEAKS.json)"
                         % (n_sm, f_mhz)}
    nc = ncu_summary("hard_sieve_kernel", ("pc_hard.cu", "pc_sieve.cuh", "pc_common.cuh"))
    if nc:
        out["ncu"] = {k: nc[k] for k in ("workload", "alu_pipe", "issue_active", "shared_pipe", "warps_active")
                      if k in nc}
    return out


def other_rooflines(sp, n_sm, f_mhz):
    """Rooflines of the easy-leaf kernel (INT32) and the P2 sieve (shared-memory
    atomics) from one pi(x) call's counters and CUDA-event kernel times."""
    f = f_mhz * 1e6
    out = {}
    if sp.get("ms_easy_kernel", 0) > 0:
        work = EASY_INT["leaf"] * sp["easy_leaves"] + EASY_INT["run"] * sp["easy_runs"]
        t = roofline_term(work, sp["ms_easy_kernel"], 128.0 * n_sm * f, "G int32-ops/s")
        t.update({"bound": "alu", "kernel_ms": sp["ms_easy_kernel"], "easy_leaves": sp["easy_leaves"],
                  "easy_runs": sp["easy_runs"], "easy_run_leaves": sp["easy_run_leaves"],
                  "per_unit": "16 per leaf resolved alone, 16 per run of clustered leaves"})
        nc = ncu_summary("easy_kernel", ("pc_leaves.cu", "pc_common.cuh"))
        if nc:
            t["ncu"] = {k: nc[k] for k in ("workload", "alu_pipe", "issue_active", "l2_hit", "dram_gbs") if k in nc}
        out["easy_kernel"] = t
    if sp.get("ms_p2_kernel", 0) > 0:
        t = roofline_term(P2_SMEM["crossing"] * sp["p2_clears"], sp["ms_p2_kernel"], 32.0 * n_sm * f,
                          "G smem-bank-accesses/s")
        t.update({"bound": "smem", "kernel_ms": sp["ms_p2_kernel"], "crossings": sp["p2_clears"],
                  "per_unit": "1 shared-memory atomic per crossing"})
        nc = ncu_summary("p2_sieve_kernel", ("pc_p2.cu", "pc_sieve.cuh", "pc_common.cuh"))
        if nc:
            t["ncu"] = {k: nc[k] for k in ("workload", "bank_conflict_frac", "issue_active", "shared_pipe")
                        if k in nc}
        out["p2_sieve_kernel"] = t
    return out


def cpu_baseline(seconds_cap=30.0):
    """The oracle (single-threaded C, unchanged) on a bounded sample: the
    same per-leaf sieve of [1, z] at x = 10^12, y = iroot3(x)."""
    import oracle
    oracle.build()
    x = ORACLE_X
    y = iroot3(x)
    t0 = time.perf_counter()
    n = 0
    while True:
        oracle.leaf_sums(x, y, C)
        n += 1
        if time.perf_counter() - t0 > min(10.0, seconds_cap) or n >= 5:
            break
    dt = (time.perf_counter() - t0) / n
    return {"value": (x // y) / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "oracle per-leaf sieve of [1, z], x=1e12, y=iroot3(x)=10^4, z=1e8, c=5; %d run(s)" % n}


def host_cpu():
    """The host's core count and CPU model (the oracle runs there)."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k, _, v = line.partition(":")
                k = k.strip().lower()
                if k in ("model name", "cpu model", "hardware") and v.strip():
                    model = v.strip()
                    break
    except OSError:
        pass
    if model is None:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    return {"nproc": os.cpu_count(), "cpu_model": model or "unknown"}


def cpu_oracle_pi(xs=(10 ** 10, 10 ** 12)):
    """The Meissel-Lehmer oracle (plain phi recursion, one core) on this host:
    wall time of pi(x) for each x, checked against Table 1."""
    import oracle
    oracle.build()
    table1 = {10 ** 10: 455052511, 10 ** 12: 37607912018}
    out = {}
    for x in xs:
        t0 = time.perf_counter()
        v = oracle.pi_meissel(x)
        dt = time.perf_counter() - t0
        assert v == table1[x], (x, v)
        out["%.0e" % x] = {"s": dt, "pi": v, "cores": 1}
    return out


def cpu_oracle_batch(n=4096, seed=0, x_max=10 ** 11):
    """The benchmark batch's queries up to x_max on every host core (spawned
    workers, one oracle pi(x) each): queries/s, beside the GPU batch figure."""
    import concurrent.futures as cf
    import multiprocessing
    import oracle
    from paper_1503_01839_gb300 import inputs
    oracle.build()
    xs = [x for x in inputs.batch_queries(n, seed) if x <= x_max]
    cores = os.cpu_count() or 1
    with cf.ProcessPoolExecutor(cores, mp_context=multiprocessing.get_context("spawn")) as ex:
        list(ex.map(oracle.iroot3, [8] * cores))            # start the workers outside the timing
        t0 = time.perf_counter()
        vals = list(ex.map(oracle.pi_meissel, xs, chunksize=16))
        dt = time.perf_counter() - t0
    return {"queries": len(xs), "x": "the batch's queries with x <= %.0e" % x_max, "s": dt,
            "qps": len(xs) / dt, "cores": cores, "results": vals}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    x = ORACLE_X
    y = iroot3(x)
    z = x // y
    for _ in range(args.warmup):
        oracle.leaf_sums(x, y, C)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.leaf_sums(x, y, C)
        times.append(time.perf_counter() - t0)
    ms = 1000 * statistics.mean(times)
    value = z / (ms / 1000)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic", "impl": "reference",
            "config": config(0),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "oracle per-leaf sieve of [1, z], x=1e12, y=10^4, z=1e8, c=5, "
                                       "one run per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_pi_mode(args):
    """Whole pi(x) evaluations through the C ABI (all phases), one per step; with
    --mode p2, P2(x, pi(y)) alone, y = alpha * iroot3(x)."""
    import torch
    import paper_1503_01839_gb300 as pc
    from paper_1503_01839_gb300 import build as pcbuild
    pcbuild.build()
    ctx = pc.Context(0, seg_bytes=args.seg_bytes, p2_bucket=1 if args.p2_bucket else 0)
    if args.mode == "p2":
        y = min(ALPHA * iroot3(X), math.isqrt(X))
        call = lambda: ctx.p2(X, y)
    else:
        call = lambda: ctx.pi_count(X, ALPHA)
    for _ in range(max(1, args.warmup)):
        ref = call()
    ts = []
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        assert call() == ref
        ts.append(time.perf_counter() - t0)
    st = ctx.stats()
    print(json.dumps({"mode": args.mode, "x": X, "alpha": ALPHA, "value": ref,
                      "p2_bucket": bool(args.p2_bucket), "ms_per_step": 1000 * statistics.mean(ts),
                      "phases_ms": {k: round(st[k], 3) for k in ("ms_tables", "ms_s1", "ms_trivial", "ms_easy",
                                                                  "ms_hard", "ms_p2", "ms_p2_kernel")}}), flush=True)
    ctx.close()
    return 0


batch_xs_results = None   # (queries, results) of the last run_batch, for the oracle's check


def run_batch(local, n, streams, seed=0):
    """The batched workload: n pi(x) queries, log10 x ~ U(8, 15) (seed 0),
    as one pc_pi_count_batch call, against a host loop of plain pc_pi_count
    calls over the same x on the same (warm) tables.  Results must agree."""
    import paper_1503_01839_gb300 as pc
    from paper_1503_01839_gb300 import inputs
    xs = inputs.batch_queries(n, seed)
    sha = hashlib.sha256(b"".join(int(v).to_bytes(8, "little") for v in xs)).hexdigest()
    with pc.Context(local, streams=streams) as cx:
        t0 = time.perf_counter()
        cx.autotune(min(xs), max(xs))              # alpha and segment size per decade
        t_tune = time.perf_counter() - t0
        tuned = {"1e%d" % (d - 1): cx.tuned(3 * 10 ** (d - 1)) + (cx.tuned_ctas(3 * 10 ** (d - 1)),)
                 for d in range(len(str(min(xs))), len(str(max(xs))) + 1)}
        t0 = time.perf_counter()
        cx.autotune_batch(xs)                      # the schedule's sieve segment size and residency
        t_tune_b = time.perf_counter() - t0
        cx.pi_count_batch(xs)                      # builds and warms the shared tables
        t0 = time.perf_counter()
        got = cx.pi_count_batch(xs)
        tb = time.perf_counter() - t0
        bst = cx.stats()
        launches = bst["kernel_launches"]
        cx_tuned_batch = cx.tuned_batch()
        t0 = time.perf_counter()
        plain = [cx.pi_count(v) for v in xs]
        tl = time.perf_counter() - t0
    assert got == plain, "batched and plain results differ"
    global batch_xs_results
    batch_xs_results = (xs, got)
    return {"queries": n, "x": "floor(10^e), e ~ U(8, 15), numpy default_rng(%d)" % seed, "x_sha256": sha,
            "slots": streams, "batch_s": tb, "batch_qps": n / tb, "plain_loop_s": tl, "plain_qps": n / tl,
            "speedup": tl / tb, "bit_exact": True, "gpu_launches": launches,
            "graph_launches": bst["graph_launches"], "graph_nodes": bst["graph_nodes"],
            "autotune_s": t_tune, "tuned_alpha_seg_ctas_per_decade": tuned,
            "autotune_batch_s": t_tune_b, "tuned_batch_seg_ctas_builtin_alpha": cx_tuned_batch}


def run_serve(local, n, rate, streams, lo_exp=9.0, hi_exp=17.0, check=64, policy=0):
    """The served workload: a Poisson stream of pi(x) / phi(x, a) requests
    (20 % phi, a ~ U{5..5000}, log10 x ~ U(lo_exp, hi_exp)) fed to the
    server at their arrival times; latency = arrival to result."""
    import random
    import threading
    import paper_1503_01839_gb300 as pc
    from paper_1503_01839_gb300 import inputs
    tr = inputs.served_trace(n, rate_per_s=rate, seed=1, lo_exp=lo_exp, hi_exp=hi_exp)
    x_max = max(r["x"] for r in tr)
    res = []
    with pc.Context(local, streams=streams) as cx:
        srv = pc.Server(cx, x_max=x_max, a_max=5000, policy=policy)
        done = threading.Event()

        def collect():
            while len(res) < n:
                res.extend(srv.poll(512, timeout_ms=50))
            done.set()

        th = threading.Thread(target=collect, daemon=True)
        th.start()
        t0 = time.perf_counter()
        late = 0.0
        for i, r in enumerate(tr):
            dt = t0 + r["t_ms"] / 1000.0 - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            else:
                late = max(late, -dt)
            srv.submit(pc.PC_QUERY_PHI if r["kind"] == "phi" else pc.PC_QUERY_PI, r["x"], r["a"], tag=i)
        t_last_arrival = time.perf_counter() - t0
        done.wait()
        t_end = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        by = {r["tag"]: r for r in res}
        # every result is the same as the request run alone: check a sample here (all in the tests)
        rnd = random.Random(5)
        for i in rnd.sample(range(n), min(check, n)):
            q = tr[i]
            want = cx.phi(q["x"], q["a"]) if q["kind"] == "phi" else cx.pi_count(q["x"])
            assert by[i]["status"] == 0 and by[i]["value"] == want, (q, by[i])
    lat = sorted(r["t_done_ms"] - r["t_submit_ms"] for r in res)
    achieved = n / t_end
    return {"policy": ["fifo", "small_first"][policy], "requests": n, "offered_qps": rate,
            "achieved_qps": achieved, "slots": streams,
            "x": "floor(10^e), e ~ U(%g, %g); 20%% phi(x, a), a ~ U{5..5000}; seed 1" % (lo_exp, hi_exp),
            "p50_ms": lat[len(lat) // 2], "p99_ms": lat[min(len(lat) - 1, (99 * len(lat)) // 100)],
            "drain_s": t_end - t_last_arrival, "feeder_max_late_ms": 1000 * late,
            "saturated": achieved < 0.9 * rate, "max_running": st["max_running"],
            "failed": st["failed"], "checked_alone": min(check, n)}


def max_over_ranks(v, world):
    """The largest of every rank's v (the slowest replica sets the job's time)."""
    if world <= 1:
        return v
    import torch
    t = torch.tensor([float(v)], dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t[0])


def sum_over_ranks(v, world):
    """Exact sum of a Python int (any size, e.g. a 128-bit partial sum) over ranks."""
    if world <= 1:
        return v
    import torch
    parts = [None] * world
    torch.distributed.all_gather_object(parts, int(v))
    return sum(parts)


def job_throughput(units_per_rank, world, seconds):
    """Whole-job throughput of `world` replicas that each processed
    units_per_rank units, timed by the slowest one."""
    return world * units_per_rank / seconds


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--seg-bytes", type=int, default=0)
    ap.add_argument("--p2-bucket", action="store_true",
                    help="pi / p2 modes: P2 by the bucket sieve of Section 2.3 (pc_params.p2_bucket)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-pi", action="store_true", help="skip the pi(1e16)/pi(1e18) wall-time lines")
    ap.add_argument("--x", type=float, default=1e18, help="profiling only: a smaller x than the benchmark's")
    ap.add_argument("--alpha", type=int, default=20)
    ap.add_argument("--mode", default="s2_hard", choices=["s2_hard", "pi", "p2", "batch", "batch-graph", "serve"],
                    help="pi / batch / serve: time only that part; batch-graph: only the batched call, "
                         "twice, no tuning and no plain loop (profiling aids)")
    ap.add_argument("--batch", type=int, default=4096, help="queries of the batched workload (0: skip)")
    ap.add_argument("--serve", type=int, default=1000, help="requests of the served workload (0: skip)")
    ap.add_argument("--serve-rate", type=float, default=2000.0)
    ap.add_argument("--serve-low-rate", type=float, default=150.0,
                    help="a second, FIFO run offered below capacity, where latency is service time (0: skip)")
    ap.add_argument("--streams", type=int, default=8, help="query slots of the batched/served forms")
    ap.add_argument("--shard", action="store_true",
                    help="N > 1: split one S2_hard into N independent shards instead of N replicas")
    args = ap.parse_args()
    global X, ALPHA
    X, ALPHA = int(args.x), args.alpha
    if args.mode in ("pi", "p2"):
        return run_pi_mode(args)
    if args.mode == "batch":
        print(json.dumps(run_batch(0, args.batch, args.streams)), flush=True)
        return 0
    if args.mode == "batch-graph":
        import paper_1503_01839_gb300 as pc
        from paper_1503_01839_gb300 import inputs
        xs = inputs.batch_queries(args.batch, 0)
        with pc.Context(0, streams=args.streams) as cx:
            cx.pi_count_batch(xs)                  # builds the shared tables
            t0 = time.perf_counter()
            cx.pi_count_batch(xs)
            dt = time.perf_counter() - t0
            st = cx.stats()
        print(json.dumps({"mode": "batch-graph", "queries": len(xs), "batch_s": dt, "qps": len(xs) / dt,
                          "kernel_launches": st["kernel_launches"], "graph_launches": st["graph_launches"],
                          "graph_nodes": st["graph_nodes"]}), flush=True)
        return 0
    if args.mode == "serve":
        for pol in (0, 1):
            print(json.dumps(run_serve(0, args.serve, args.serve_rate, args.streams, policy=pol)), flush=True)
        if args.serve_low_rate > 0:
            print(json.dumps(run_serve(0, args.serve, args.serve_low_rate, args.streams, policy=0)), flush=True)
        return 0
    if args.impl == "reference":
        return run_reference(args)

    world, rank, local = dist_env()
    import torch
    import paper_1503_01839_gb300 as pc
    from paper_1503_01839_gb300 import build as pcbuild
    pcbuild.build()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")

    w = workload()
    x, y, c, z = w["x"], w["y"], w["c"], w["z"]
    ctx = pc.Context(local, seg_bytes=args.seg_bytes)
    stream = torch.cuda.current_stream()
    ctx.set_stream(stream.cuda_stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    # one step: the whole S2_hard on every rank (replicas), or with --shard
    # rank r's shard of it (Section 4 starting values, no exchange of counts)
    shard = args.shard and world > 1
    step = (lambda x_, y_, c_: ctx.s2_hard_shard(x_, y_, c_, rank, world)) if shard else ctx.s2_hard

    # warm-up (also builds the device tables for this x)
    ref = None
    for _ in range(max(1, args.warmup)):
        v = step(x, y, c)
        ref = v if ref is None else ref
        assert v == ref, "S2_hard changed between runs"
    torch.cuda.synchronize()

    # device-timed steps (inputs resident; L2 flushed between steps)
    if world > 1:
        torch.distributed.barrier()
    evs = []
    stats = []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        t_wall0 = time.perf_counter()
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            v = step(x, y, c)
            e1.record(stream)
            assert v == ref
            evs.append((e0, e1))
            stats.append(ctx.stats())
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall0
    step_ms = [a.elapsed_time(b) for a, b in evs]
    tot_ms = max_over_ranks(sum(step_ms), world)
    ms_per_step = tot_ms / args.steps
    # shards split one z among the ranks; replicas each sieve all of it
    value = job_throughput(z, 1 if shard else world, ms_per_step / 1000.0)

    # end to end through the C ABI: host scalars in, host int128 out
    e2e_times = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        v = step(x, y, c)
        e2e_times.append(time.perf_counter() - t0)
        assert v == ref
    e2e_s = max_over_ranks(statistics.mean(e2e_times), world)

    st = stats[-1]
    sieve_ms = statistics.mean(s["ms_hard_sieve"] for s in stats)
    launches = sum(int(s["kernel_launches"]) for s in stats)

    peaks = measured_peaks()
    sm_max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    traffic = profile_traffic()

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "strong" if shard else "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": config(int(st["seg_bytes"]), "shards (Section 4 starting values)" if shard else "replicas"),
            "e2e": {"value": job_throughput(z, 1 if shard else world, e2e_s), "unit": UNIT, "h2d_bytes_per_step": 24, "d2h_bytes_per_step": 16},
            "gpu_launches": launches,
            "roofline": hard_roofline(st, sieve_ms, n_sm, sm_max_mhz, traffic),
            "clocks": clk.summary(),
            "s2_hard": str(sum_over_ranks(ref, world) if shard else ref),
            "hard_leaves": int(st["hard_leaves"]), "clears": int(st["clears"]),
            "hard_leaves_per_s": float(st["hard_leaves"]) / (ms_per_step / 1000.0),
            "segments": int(st["segments"]), "steps_seg_prime": int(st["steps"]),
            "work_items": int(st["work_items"]), "item_steps": int(st["item_steps"]),
            "warp_steps": int(st["warp_steps"]), "leaf_warp_steps": int(st["leaf_warp_steps"]),
            "timed_wall_s": t_wall}

    if rank == 0 and not args.no_pi:
        pis = {}
        # pc_pi_count(x, 0): the library's own alpha (built-in table), as a user calls it
        for xx, want in ((10 ** 16, PI_1E16), (10 ** 18, PI_1E18)):
            al = 0
            ctx.pi_count(xx, al)
            ts = []
            for _ in range(5):
                flush.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                got = ctx.pi_count(xx, al)
                ts.append(time.perf_counter() - t0)
                assert got == want, (xx, got, want)
            sp = ctx.stats()
            pis["%.0e" % xx] = {"wall_s": min(ts), "wall_s_mean": statistics.mean(ts),
                                "wall_s_stdev": statistics.stdev(ts), "runs": len(ts),
                                "alpha": ctx.tuned(xx)[0], "pi": got, "table1": want, "y": sp["y"],
                                "timing": "host wall clock around pc_pi_count, 5 runs (best, mean, stdev), "
                                          "L2 flushed before each",
                                "ms": {k: round(sp[k], 3) for k in ("ms_tables", "ms_s1", "ms_trivial",
                                                                     "ms_easy", "ms_hard", "ms_p2",
                                                                     "ms_hard_sieve", "ms_easy_kernel",
                                                                     "ms_p2_kernel")},
                                "rooflines": other_rooflines(sp, n_sm, sm_max_mhz)}
        line["pi_wall"] = pis
    if rank == 0 and args.batch > 0:
        line["batch"] = run_batch(local, args.batch, args.streams)
    if rank == 0 and args.serve > 0:
        line["served"] = [run_serve(local, args.serve, args.serve_rate, args.streams, policy=pol) for pol in (0, 1)]
        if args.serve_low_rate > 0:
            line["served"].append(run_serve(local, args.serve, args.serve_low_rate, args.streams, policy=0))
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
        line["cpu_baseline"]["host"] = host_cpu()
        line["cpu_baseline"]["oracle_pi"] = cpu_oracle_pi()
        if args.batch > 0:
            ob = cpu_oracle_batch(args.batch)
            if batch_xs_results:
                gpu = [v for x, v in zip(*batch_xs_results) if x <= 10 ** 11]
                ob["bit_exact_with_gpu_batch"] = gpu == ob["results"]
            del ob["results"]
            line["cpu_baseline"]["oracle_batch"] = ob
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
