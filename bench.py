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


def config(seg_bytes):
    w = workload()
    return {"workload": "S2_hard hard-leaf sieve x=%.0e y=%d*iroot3(x)=%d c=%d (one evaluation per step)"
                        % (w["x"], ALPHA, w["y"], C),
            "x": w["x"], "y": w["y"], "z": w["z"], "c": C, "seg_bytes": seg_bytes,
            "l2": "flushed between timed steps (256 MiB write)", "parallelism": "replicas"}


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
    """Whole pi(x) evaluations through the C ABI (all phases), one per step."""
    import torch
    import paper_1503_01839_gb300 as pc
    from paper_1503_01839_gb300 import build as pcbuild
    pcbuild.build()
    ctx = pc.Context(0, seg_bytes=args.seg_bytes)
    for _ in range(max(1, args.warmup)):
        ref = ctx.pi_count(X, ALPHA)
    ts = []
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        assert ctx.pi_count(X, ALPHA) == ref
        ts.append(time.perf_counter() - t0)
    st = ctx.stats()
    print(json.dumps({"mode": "pi", "x": X, "alpha": ALPHA, "pi": ref, "ms_per_step": 1000 * statistics.mean(ts),
                      "phases_ms": {k: round(st[k], 3) for k in ("ms_tables", "ms_s1", "ms_trivial", "ms_easy",
                                                                  "ms_hard", "ms_p2")}}), flush=True)
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--seg-bytes", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-pi", action="store_true", help="skip the pi(1e16)/pi(1e18) wall-time lines")
    ap.add_argument("--x", type=float, default=1e18, help="profiling only: a smaller x than the benchmark's")
    ap.add_argument("--alpha", type=int, default=20)
    ap.add_argument("--mode", default="s2_hard", choices=["s2_hard", "pi"],
                    help="pi: time whole pi(x) evaluations instead (profiling aid)")
    args = ap.parse_args()
    global X, ALPHA
    X, ALPHA = int(args.x), args.alpha
    if args.mode == "pi":
        return run_pi_mode(args)
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

    # warm-up (also builds the device tables for this x)
    ref = None
    for _ in range(max(1, args.warmup)):
        v = ctx.s2_hard(x, y, c)
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
            v = ctx.s2_hard(x, y, c)
            e1.record(stream)
            assert v == ref
            evs.append((e0, e1))
            stats.append(ctx.stats())
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall0
    step_ms = [a.elapsed_time(b) for a, b in evs]
    tot_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([tot_ms], dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        tot_ms = float(t[0])
    ms_per_step = tot_ms / args.steps
    value = world * z / (ms_per_step / 1000.0)

    # end to end through the C ABI: host scalars in, host int128 out
    e2e_times = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        v = ctx.s2_hard(x, y, c)
        e2e_times.append(time.perf_counter() - t0)
        assert v == ref
    e2e_s = statistics.mean(e2e_times)
    if world > 1:
        t = torch.tensor([e2e_s], dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_s = float(t[0])

    st = stats[-1]
    sieve_ms = statistics.mean(s["ms_hard_sieve"] for s in stats)
    launches = sum(int(s["kernel_launches"]) for s in stats)

    # roofline of the sieve kernel: 32-bit shared-memory bank accesses.
    # per crossing-off: one atomic RMW (1); per hard leaf: the block-prefix
    # read (1) + on average half of a 1024-bit block of u64 words (16).
    peaks = measured_peaks()
    sm_max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    accesses = float(st["clears"]) + 17.0 * float(st["hard_leaves"])
    achieved = accesses / (sieve_ms / 1000.0) / 1e9
    peak = 32.0 * n_sm * sm_max_mhz * 1e6 / 1e9
    traffic = profile_traffic()

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": config(int(st["seg_bytes"])),
            "e2e": {"value": world * z / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 24, "d2h_bytes_per_step": 16},
            "gpu_launches": launches,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "G smem-bank-accesses/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": "hard_sieve_kernel", "kernel_ms": sieve_ms,
                         "peak_basis": "32 banks x %d SMs x %.0f MHz (max SM clock, MEASURED_PEAKS.json)"
                                       % (n_sm, sm_max_mhz)},
            "clocks": clk.summary(),
            "s2_hard": str(ref), "hard_leaves": int(st["hard_leaves"]), "clears": int(st["clears"]),
            "hard_leaves_per_s": float(st["hard_leaves"]) / (ms_per_step / 1000.0),
            "segments": int(st["segments"]), "steps_seg_prime": int(st["steps"]),
            "timed_wall_s": t_wall}

    if rank == 0 and not args.no_pi:
        pis = {}
        for xx, want, al in ((10 ** 16, PI_1E16, 20), (10 ** 18, PI_1E18, 20)):
            ctx.pi_count(xx, al)
            ts = []
            for _ in range(3):
                flush.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                got = ctx.pi_count(xx, al)
                ts.append(time.perf_counter() - t0)
                assert got == want, (xx, got, want)
            sp = ctx.stats()
            pis["%.0e" % xx] = {"wall_s": min(ts), "alpha": al, "pi": got, "table1": want,
                                "ms": {k: round(sp[k], 3) for k in ("ms_tables", "ms_s1", "ms_trivial",
                                                                     "ms_easy", "ms_hard", "ms_p2")}}
        line["pi_wall"] = pis
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
