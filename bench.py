"""Benchmark of the exact KNN self-join on B300 (one JSON line on stdout).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload unif|expo|batched|served] [--no-cpu-baseline] [--no-e2e]

A step is one pass of the whole join -- search-distance selection, grid
index, density queue, every scan pass and the output -- over each point set
of the workload:
  unif: Unif-2D, Unif-4D, Unif-6D, n = 2,000,000 each, K = 32 (three joins);
  expo: Expo-2D, Expo-4D, Expo-6D, n = 2,000,000 each, K = 64.
Points are synthetic (seeded uniform on the 2^-24 grid, or exponential with
rate 40, as in the paper's Sec. 5.1 classes) and resident in HBM before the
timed region.  L2 (126 MB) is flushed by a 256 MiB write before every timed
step; each step is timed with CUDA events on the library's stream and the
flush is outside the events.

value = query points per second over the whole job (all ranks); e2e is the
same metric through the C ABI with pinned host buffers (copies timed).
Roofline, per join: T_roof = max(T_fp32, T_bytes), T_fp32 = W_ref * (3d - 1)
flops at the FP32 peak (SMs x 128 lanes x 2 flops x max SM clock), T_bytes =
n*4d (points read) + n*K*12 (ids and FP64 distances written) bytes at the
measured HBM peak, with W_ref the candidate count of the reference grid
schedule counted by the oracle's grid join.  The FP32 term binds the step,
so the contract's roofline entry is for the scan kernel (the dominant
kernel) as ALU-bound: achieved = the step's W_ref * (3d - 1) flops / the
event-timed duration of its scan launches.

Before the warm-up each join's cell-width multiplier is autotuned through
knnjoin_autotune (untimed; --no-autotune keeps the default 1.25); the value
used is reported per join.

--impl reference times the CPU oracle (exact grid join, OpenMP on the host
cores) on a bounded sample of the same workload per step.

--workload batched: 256 independent joins (n log-uniform in [1k, 200k], d in
{2,3,4,6}, K in {4..64}, uniform or exponential(40)) through
knnjoin_self_join_batch (worker pool, concurrent) against a plain loop of
knnjoin_self_join calls on one stream; both timed per step, results equal.
--workload join: R x S through knnjoin_join, 2M uniform queries against 2M
uniform points for d = 2, 4, 6, K = 32 (sampled rows checked against the
oracle's brute force unless --no-cpu-baseline).
--workload served: a Poisson stream of joins (n log-uniform in [10k, 5M],
d 2..6, K 8..128, uniform / exponential(40) / clustered 2-D) submitted and
polled through knnjoin_submit/knnjoin_poll at rho x the measured capacity;
p50/p99 latency (submit -> done) against FIFO one-at-a-time serving.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import knn_inputs as gen  # noqa: E402

METRIC = "query points/s (K=32, 2M pts, 2-6D)"
UNIT = "query points/s"
WORKLOADS = {
    "unif": ["unif2d_2m", "unif4d_2m", "unif6d_2m"],
    "expo": ["expo2d_2m", "expo4d_2m", "expo6d_2m"],
}
WORKLOAD_TEXT = {
    "unif": "Unif-2D/4D/6D: n=2,000,000 each, coords i.i.d. uniform [0,1) float32 (2^-24 grid), "
            "K=32, seed 0; one step = the three joins",
    "expo": "Expo-2D/4D/6D: n=2,000,000 each, coords i.i.d. exponential(40) float32, K=64, seed 0; "
            "one step = the three joins",
}


def peaks():
    """(HBM GB/s, its kind, SM max MHz) from the driver-written measured peaks,
    else the fallback figures (6.4 TB/s, 2032 MHz)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured", float(j.get("sm_max_mhz") or 2032.0)
    except Exception:
        return 6400.0, "fallback", 2032.0


# FP32 lanes per SM on B300 (4 sub-partitions x 32); one FMA = 2 flops.
FP32_LANES_PER_SM = 128


def fp32_peak_tflops(sms: int, sm_mhz: float) -> float:
    """Nominal FP32 FMA peak from unit counts and clock: SMs x 128 lanes x 2
    flops x SM clock."""
    return sms * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


def csrc_digest() -> str:
    """sha256 prefix over the scan kernel's sources: its translation unit
    (csrc/scan2_launch.cu) and every header it includes (names and bytes)."""
    import hashlib
    sys.path.insert(0, os.path.join(ROOT, "paper_1810_04758_b300"))
    from paper_1810_04758_b300 import build as kbuild
    files = sorted(kbuild._includes(os.path.join(kbuild.CSRC, "scan2_launch.cu"), set()))
    h = hashlib.sha256()
    for f in files:
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(names, buffers=None):
    """DRAM bytes (read + write) per step of the scan launches of the named
    joins, from the committed ncu counters (profiles/k_scan2_traffic.json);
    None when a join has none, the scan kernel's sources changed since they
    were taken, or a join now runs with another candidate buffer size
    (buffers: join -> entries, as the joins ran)."""
    try:
        with open(os.path.join(ROOT, "profiles", "k_scan2_traffic.json")) as f:
            j = json.load(f)
    except (OSError, ValueError):
        return None
    if j.get("csrc_sha256_prefix") != csrc_digest():
        return None
    try:
        if buffers and any(j["joins"][nm].get("buffer_entries") != buffers.get(nm) for nm in names):
            return None
        return int(sum(j["joins"][nm]["scan_dram_bytes"] for nm in names))
    except (KeyError, TypeError):
        return None


def tune_cache_keys(path: str) -> set:
    """(d, K, floor(log2 n)) keys already in a knnjoin tune cache file."""
    if not path or not os.path.exists(path):
        return set()
    try:
        with open(path) as f:
            return {(e["d"], e["K"], e["nlog2"]) for e in json.load(f)["entries"]}
    except (OSError, ValueError, KeyError):
        return set()


def wref_table():
    try:
        with open(os.path.join(ROOT, "tests", "golden", "wref_2m.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(x: float, device, world: int) -> float:
    """Maximum of a per-rank value over all ranks (the job's time is the
    slowest rank's); identity on one rank."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def algorithmic_work(name: str, n: int, d: int, K: int, wref: dict) -> tuple[float, float, float]:
    """(compulsory bytes, FP32 flops, no-reuse candidate bytes) of one join.
    Compulsory bytes: the points read once (n*4d) and the ids and FP64
    distances written once (n*K*12).  Flops: W_ref candidate evaluations x
    (3d - 1) (d differences, d squares, d - 1 additions), W_ref counted by the
    oracle's grid schedule.  The candidate bytes W_ref*4d credit no on-chip
    reuse and are a diagnostic, not a bound."""
    w = wref.get(name, {}).get("candidates")
    if w is None:
        return float("nan"), float("nan"), float("nan")
    return float(n * 4 * d + n * K * 12), float(w) * (3 * d - 1), float(w) * 4 * d


# ---------------------------------------------------------------------------
# CPU oracle arm
# ---------------------------------------------------------------------------
def oracle_sample_step(points_by_name, rows: int, threads: int):
    """One bounded sample of the workload on the CPU oracle (exact grid join,
    OpenMP on `threads` host cores): for each point set, `rows` strided query
    rows answered against the whole set -- the search distance and the grid
    index over all n points are part of every call.  Returns (queries
    answered, seconds, per-set detail).  Nothing is extrapolated: the rate is
    queries answered / time spent."""
    import oracle
    total_q, total_t, detail = 0, 0.0, {}
    for name, (p, K) in points_by_name.items():
        n = len(p)
        r = min(rows, n)
        t0 = time.perf_counter()
        if r >= n:
            oracle.grid(p, K, threads=threads)
        else:
            oracle.grid_rows(p, K, np.linspace(0, n - 1, r).astype(np.int64), threads=threads)
        dt = time.perf_counter() - t0
        total_q += r
        total_t += dt
        detail[name] = {"rows": r, "s": round(dt, 3)}
    return total_q, total_t, detail


def oracle_full_join(name: str, threads: int):
    """Seconds of one whole oracle grid join of a named 2M-point set."""
    import oracle
    p, K = gen.config_points(name)
    t0 = time.perf_counter()
    oracle.grid(p, K, threads=threads)
    return time.perf_counter() - t0


def oracle_bf_small(threads: int) -> dict:
    """The brute-force oracle on the small uniform set (Unif-2D, n = 20,000,
    K = 8) with all host cores and with one: query points/s of each."""
    import oracle
    p, K = gen.config_points("unif2d_20k")
    out = {"set": "unif2d_20k (n=20000, d=2, K=8)", "what": "oracle_bf: every pair, canonical FP64"}
    for label, th in (("all_cores", threads), ("one_core", 1)):
        t0 = time.perf_counter()
        oracle.bf(p, K, threads=th)
        dt = time.perf_counter() - t0
        out[label] = {"threads": th, "s": round(dt, 3), "q_per_s": len(p) / dt}
    return out


def step_config(args, world: int) -> dict:
    """The `config` of the unif / expo step (both arms print the same)."""
    return {"workload": WORKLOAD_TEXT[args.workload], "n": 2_000_000, "d": [2, 4, 6],
            "K": 64 if args.workload == "expo" else 32,
            "l2": "flushed (256 MiB write) before every timed step",
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    names = WORKLOADS[args.workload]
    pts = {nm: gen.config_points(nm) for nm in names}
    cores = host_cores()
    rows = args.cpu_sample
    for _ in range(args.warmup):
        oracle_sample_step(pts, rows, cores)
    step_s = []
    detail = {}
    t0 = time.perf_counter()
    for _ in range(args.steps):
        q, sec, detail = oracle_sample_step(pts, rows, cores)
        step_s.append(sec)
    wall = time.perf_counter() - t0
    value = q / statistics.median(step_s)
    line = {
        "impl": "reference", "metric": METRIC if args.workload == "unif" else METRIC.replace("K=32", "K=64"),
        "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * statistics.median(step_s),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": step_config(args, world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"per step, {rows} strided query rows of each 2M-point set "
                                   f"answered by the exact CPU grid join against the whole set "
                                   f"(search distance and index over all n included); value = "
                                   f"queries answered / measured step time, median of "
                                   f"{args.steps} steps, nothing extrapolated",
                         "detail": detail},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": round(wall, 2),
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_ours(args, rank, world, local_rank):
    import torch
    import paper_1810_04758_b300 as kj
    from paper_1810_04758_b300 import build as kbuild

    kbuild.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    ctx = kj.Context(device=local_rank, stream=stream, policy=args.policy,
                     tune_cache_path=args.tune_cache or None)
    names = WORKLOADS[args.workload]
    if args.configs:
        names = [nm for nm in names if nm in args.configs.split(",")]
    hosts = {nm: gen.config_points(nm) for nm in names}
    dpts = {nm: torch.from_numpy(p).to(dev) for nm, (p, K) in hosts.items()}
    outs = {nm: (torch.empty((len(p), K), dtype=torch.int32, device=dev),
                 torch.empty((len(p), K), dtype=torch.float64, device=dev))
            for nm, (p, K) in hosts.items()}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    # cell-width autotuning (untimed, before the warm-up): the library times
    # the join at several multipliers and keeps the fastest per (d, K, log2 n)
    tuned = {}
    if not args.no_autotune and args.policy == 0:
        cached = tune_cache_keys(args.tune_cache)
        for nm in names:
            n_, d_ = hosts[nm][0].shape
            if (d_, hosts[nm][1], int(n_).bit_length() - 1) in cached:
                tuned[nm] = "cached"
            else:
                tuned[nm] = ctx.autotune(dpts[nm], hosts[nm][1])
        torch.cuda.synchronize()

    def one_step(collect):
        # the step's joins one blocking call after another (per-join stats)
        per = {}
        for nm in names:
            K = hosts[nm][1]
            ctx.self_join(dpts[nm], K, *outs[nm])
            if collect:
                per[nm] = ctx.stats()
        return per

    plist, klist, olist = [dpts[nm] for nm in names], [hosts[nm][1] for nm in names], [outs[nm] for nm in names]

    def batch_step():
        # the step's joins through knnjoin_self_join_batch: the worker pool
        # runs them on their own streams, so one join's index build and
        # small passes overlap another's scan
        ctx.self_join_batch(plist, klist, olist)

    for _ in range(max(args.warmup, 0)):
        one_step(False)
        batch_step()
    torch.cuda.synchronize()

    def timed_steps(fn, collect):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        pers = []
        for i in range(args.steps):
            flush.fill_(float(i))
            evs[i][0].record(stream)
            r = fn(collect) if collect else fn()
            evs[i][1].record(stream)
            pers.append(r)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in evs], pers

    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        wall0 = time.perf_counter()
        step_ms, _ = timed_steps(batch_step, False)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        seq_ms, pers = timed_steps(one_step, True)
    per_cfg = {nm: [p[nm] for p in pers] for nm in names}
    launches = sum(p[nm]["launches"] for p in pers for nm in names)
    scan_ms = sum(p[nm]["ms_scan"] for p in pers for nm in names)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    total_ms = max_over_ranks(sum(step_ms), dev, world)
    seq_ms_per_step = max_over_ranks(sum(seq_ms), dev, world) / args.steps
    nq_step = sum(len(hosts[nm][0]) for nm in names)
    ms_per_step = total_ms / args.steps
    value = world * nq_step / (ms_per_step / 1000.0)

    # roofline: per join T_roof = max(T_fp32, T_bytes) with T_fp32 = W_ref*(3d-1)
    # flops at the FP32 peak and T_bytes = compulsory bytes at the HBM peak
    hbm, peak_kind, sm_max_mhz = peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    p32 = fp32_peak_tflops(sms, sm_max_mhz)
    wref = wref_table()
    alg_flops, cand_bytes, roof_ms = 0.0, 0.0, 0.0
    per_summary = {}
    for nm in names:
        p, K = hosts[nm]
        n, d = p.shape
        b, f, cb = algorithmic_work(nm, n, d, K, wref)
        alg_flops += f
        cand_bytes += cb
        st = per_cfg[nm]
        ms_join = statistics.median(s["ms_total"] for s in st)
        ms_scan_j = statistics.median(s["ms_scan"] for s in st)
        t_fp32 = f / (p32 * 1e12) * 1e3
        t_bytes = b / (hbm * 1e9) * 1e3
        t_roof = max(t_fp32, t_bytes)
        roof_ms += t_roof
        w_ref = wref.get(nm, {}).get("candidates")
        per_summary[nm] = {
            "ms": round(ms_join, 4), "q_per_s": n / (ms_join / 1e3),
            "ms_scan": round(ms_scan_j, 4),
            "ms_index": round(statistics.median(s["ms_index"] for s in st), 4),
            "passes": st[-1]["passes"], "pass_queries": st[-1]["pass_queries"],
            "ms_pass": [round(x, 3) for x in st[-1]["ms_pass"]],
            "pass_candidates": st[-1]["pass_candidates"],
            "candidates": st[-1]["candidates"], "band_entries": st[-1]["band_entries"],
            "overflow_queries": st[-1]["overflow_queries"],
            "w_ref": w_ref, "w_over_wref": (st[-1]["candidates"] / w_ref) if w_ref else None,
            "t_fp32_ms": round(t_fp32, 4), "t_bytes_ms": round(t_bytes, 4), "t_roof_ms": round(t_roof, 4),
            "bound": "alu" if t_fp32 >= t_bytes else "hbm",
            "join_roofline_frac": t_roof / ms_join, "scan_roofline_frac": t_roof / ms_scan_j,
            "fixed_point": st[-1]["fixed_point"], "cell_width": st[-1]["cell_width"],
            "width_mult": st[-1]["width_mult"], "buffer_entries": st[-1].get("buffer_entries"),
            "autotuned": nm in tuned,
        }
    scan_ms_per_step = scan_ms / args.steps
    achieved = alg_flops / (scan_ms_per_step / 1e3) / 1e12 if scan_ms_per_step > 0 else float("nan")
    roofline = {"bound": "alu", "achieved": achieved, "peak": p32, "unit": "TFLOP/s",
                "frac": achieved / p32,
                "traffic": None if args.configs else profiled_traffic(
                    names, {nm: per_summary[nm]["buffer_entries"] for nm in names}),
                "kernel": "k_scan2",
                "peak_kind": f"derived: {sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flops x "
                             f"{sm_max_mhz:.0f} MHz (max SM clock)",
                "algorithmic_flops_per_step": alg_flops,
                "scan_ms_per_step": scan_ms_per_step,
                "step_frac": roof_ms / ms_per_step,
                "step_roof_ms": roof_ms,
                "hbm_peak_gbs": hbm, "hbm_peak_kind": peak_kind,
                "note": "achieved = W_ref*(3d-1) FP32 flops of the step's joins / the event-timed "
                        "duration of the step's scan launches (the FP32 term binds the step: "
                        "per-join bounds in per_config); step_frac = sum over joins of "
                        "max(T_fp32, T_bytes) / the whole step's device time, T_bytes = "
                        "(n*4d + n*K*12) bytes at the HBM peak; traffic = ncu DRAM bytes of "
                        "the step's scan launches",
                "diagnostic_candidate_bytes": {
                    "bytes_per_step": cand_bytes,
                    "GBps_over_scan": cand_bytes / (scan_ms_per_step / 1e3) / 1e9 if scan_ms_per_step > 0
                    else None,
                    "what": "W_ref*4d candidate coordinate bytes with no on-chip reuse credited; a "
                            "candidate row serves several queries of a work item and the 2M-point "
                            "set stays in L2, so this is not a bound"}}

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        hpts = {nm: torch.from_numpy(hosts[nm][0]).pin_memory() for nm in names}
        hout = {nm: (torch.empty((len(hosts[nm][0]), hosts[nm][1]), dtype=torch.int32).pin_memory(),
                     torch.empty((len(hosts[nm][0]), hosts[nm][1]), dtype=torch.float64).pin_memory())
                for nm in names}
        # steps through knnjoin_submit / knnjoin_poll, several steps in flight: the
        # worker pool runs each join on its own stream, so a step's result
        # copies overlap the next step's kernels (output buffers alternate)
        depth = max(1, args.e2e_depth)
        hout2 = [hout] + [{nm: (torch.empty_like(hout[nm][0]).pin_memory(),
                                torch.empty_like(hout[nm][1]).pin_memory()) for nm in names}
                          for _ in range(depth - 1)]

        def wait(jid):
            while True:
                rc = ctx.poll(jid)
                if rc != 4:  # KNN_ERR_NOT_READY
                    if rc != 0:
                        raise RuntimeError(f"served join failed: {rc} {ctx.last_error()}")
                    return
                time.sleep(0.0001)

        def run_pipelined(nsteps):
            inflight = []
            for st_i in range(nsteps):
                bufs = hout2[st_i % depth]
                while inflight and inflight[0][0] <= st_i - depth:
                    wait(inflight.pop(0)[1])
                for nm in names:
                    jid, _, _ = ctx.submit(hpts[nm], hosts[nm][1], *bufs[nm])
                    inflight.append((st_i, jid))
            for _, jid in inflight:
                wait(jid)

        # warm-up (untimed): enough steps that every worker pipeline of the
        # pool has run a join and holds its scratch (a first join on a
        # pipeline grows the memory pool)
        run_pipelined(max(2, -(-8 // len(names)) + depth))
        torch.cuda.synchronize()
        e2e_steps = max(4, min(args.steps, 8))
        t0 = time.perf_counter()
        run_pipelined(e2e_steps)
        torch.cuda.synchronize()
        e_ms = (time.perf_counter() - t0) * 1e3 / e2e_steps
        # the same joins one blocking call after another, for reference
        t0 = time.perf_counter()
        for nm in names:
            ctx.self_join(hpts[nm], hosts[nm][1], *hout[nm])
        torch.cuda.synchronize()
        seq_ms = (time.perf_counter() - t0) * 1e3
        h2d = sum(hosts[nm][0].nbytes for nm in names)
        d2h = sum(len(hosts[nm][0]) * hosts[nm][1] * 12 for nm in names)

        # the step's copies alone (pinned host <-> device, events on one stream)
        def copy_ms(fn):
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            fn()
            torch.cuda.synchronize()
            a.record(stream)
            fn()
            e.record(stream)
            torch.cuda.synchronize()
            return a.elapsed_time(e)

        def h2d_copy():
            for nm in names:
                dpts[nm].copy_(hpts[nm], non_blocking=True)

        def d2h_copy():
            for nm in names:
                hout[nm][0].copy_(outs[nm][0], non_blocking=True)
                hout[nm][1].copy_(outs[nm][1], non_blocking=True)

        h2d_ms, d2h_ms = copy_ms(h2d_copy), copy_ms(d2h_copy)
        e2e = {"value": world * nq_step / (e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": e_ms, "steps": e2e_steps,
               "api": f"knnjoin_submit/knnjoin_poll, pinned host points and outputs, {depth} steps in flight",
               "sequential_self_join_ms_per_step": round(seq_ms, 3),
               "h2d_ms_per_step": round(h2d_ms, 3), "d2h_ms_per_step": round(d2h_ms, 3),
               "copies": "the step's inputs and results copied alone (pinned host memory, CUDA events)"}

    # FP32-only id mismatch (untimed): how often ranking by the FP32 filter
    # distance alone would change the exact rows, on strided sampled rows
    fp32_only = None
    if rank == 0 and args.fp32_rows > 0:
        fp32_only = {}
        for nm in names:
            n_ = len(hosts[nm][0])
            m = min(args.fp32_rows, n_)
            res = ctx.fp32_mismatch(dpts[nm], outs[nm][0], range(0, n_, n_ // m)[:m])
            fp32_only[nm] = {k: res[k] for k in ("rows", "positions_differing", "ids_missing",
                                                  "id_mismatch_rate", "row_mismatch_rate")}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = host_cores()
        q, sec, detail = oracle_sample_step(hosts, args.cpu_sample, cores)
        full_name = names[0]
        full_s = oracle_full_join(full_name, cores)
        cpu = {"value": q / sec, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{args.cpu_sample} strided query rows of each 2M-point set answered by "
                         f"the exact CPU grid join (OpenMP) against the whole set, search distance "
                         f"and index over all n included; value = queries answered / measured "
                         f"time, nothing extrapolated",
               "detail": detail,
               "full_join": {"set": full_name, "rows": len(hosts[full_name][0]), "s": round(full_s, 3),
                             "q_per_s": len(hosts[full_name][0]) / full_s,
                             "what": "one whole oracle join of this set, all rows, measured"},
               "brute_force_small": oracle_bf_small(cores)}

    ctx.close()
    if rank != 0:
        return 0
    line = {
        "metric": METRIC if args.workload == "unif" else METRIC.replace("K=32", "K=64"),
        "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (scan) + exact canonical-f64 re-score (integer emulation)",
        "data": "synthetic",
        "config": step_config(args, world),
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "fp32_only_mismatch": fp32_only,
        "policy": "paper GPU-Only (global eps, re-index)" if args.policy == 1 else "certified rings",
        "sequential_ms_per_step": seq_ms_per_step,
        "step_api": "knnjoin_self_join_batch (the three joins on the worker pool); per-join stats, "
                    "roofline and sequential_ms_per_step from the same joins as blocking calls",
        "clocks": clk.summary(),
        "per_config": per_summary,
        "wall_s_timed": round(wall, 3),
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# Batched and served workloads
# ---------------------------------------------------------------------------
def run_batched(args, rank, world, local_rank):
    import torch
    import paper_1810_04758_b300 as kj
    from paper_1810_04758_b300 import build as kbuild

    kbuild.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    jobs = gen.batched_jobs(args.jobs or 256, seed=0)
    pts = [torch.from_numpy(gen.batched_points(j)).to(dev) for j in jobs]
    Ks = [j["K"] for j in jobs]
    nq = sum(len(p) for p in pts)
    outs_a = [(torch.empty((len(p), K), dtype=torch.int32, device=dev),
               torch.empty((len(p), K), dtype=torch.float64, device=dev)) for p, K in zip(pts, Ks)]
    outs_b = [(torch.empty_like(a), torch.empty_like(b)) for a, b in outs_a]
    outs_c = [(torch.empty_like(a), torch.empty_like(b)) for a, b in outs_a]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    import tempfile
    tune_path = args.tune_cache or os.path.join(tempfile.mkdtemp(), "tune_batched.json")
    ctx = kj.Context(device=local_rank, stream=stream, workers=args.workers, tune_cache_path=tune_path)
    # autotuning (untimed): one join of each (d, K, floor(log2 n)) class of
    # the batch, its cell width and buffer size shared by every join of the
    # class (and by the worker pool)
    tuned_classes = {}
    if not args.no_autotune:
        for p, K in zip(pts, Ks):
            key = (p.shape[1], K, int(len(p)).bit_length() - 1)
            if key not in tuned_classes:
                tuned_classes[key] = ctx.autotune(p, K)
        torch.cuda.synchronize()
    # the same batch with the joins' scans done together (one launch per
    # (d, buffer size) group and pass over the union of their work items)
    uctx = kj.Context(device=local_rank, stream=stream, batch_union=True, tune_cache_path=tune_path)

    def plain():
        for p, K, (i, d) in zip(pts, Ks, outs_a):
            ctx.self_join(p, K, i, d)

    def batched():
        jl = [kj.KnnjoinJob(p.data_ptr(), len(p), p.shape[1], K, i.data_ptr(), d.data_ptr())
              for p, K, (i, d) in zip(pts, Ks, outs_b)]
        kj.knnjoin_self_join_batch(ctx.ctx, jl)

    def union():
        jl = [kj.KnnjoinJob(p.data_ptr(), len(p), p.shape[1], K, i.data_ptr(), d.data_ptr())
              for p, K, (i, d) in zip(pts, Ks, outs_c)]
        kj.knnjoin_self_join_batch(uctx.ctx, jl)

    def timed(fn):
        ms = []
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.fill_(float(i))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return statistics.median(ms)

    with ClockSampler(local_rank) as clk:
        ms_plain = timed(plain)
        ms_batch = timed(batched)
        ms_union = timed(union)
    same = all(torch.equal(a[0], b[0]) and torch.equal(a[1], b[1]) for a, b in zip(outs_a, outs_b))
    same_u = all(torch.equal(a[0], c[0]) and torch.equal(a[1], c[1]) for a, c in zip(outs_a, outs_c))
    ctx.close()
    uctx.close()
    if rank != 0:
        return 0
    value = world * nq / (ms_batch / 1e3)
    line = {
        "metric": "batched query points/s (256 joins, n 1k-200k, d 2-6, K 4-64)",
        "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_batch, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (scan) + exact canonical-f64 re-score", "data": "synthetic",
        "config": {"workload": f"Batched: {len(jobs)} joins, {nq} points in all, n log-uniform "
                               f"[1k,200k], d in {{2,3,4,6}}, K in {{4,8,16,32,64}}, uniform or "
                               f"exponential(40), seed 0", "workers": args.workers or 8,
                   "l2": "flushed (256 MiB write) before every timed step",
                   "autotuned_classes": len(tuned_classes)},
        "plain_per_job": {"value": world * nq / (ms_plain / 1e3), "ms_per_step": ms_plain,
                          "how": "knnjoin_self_join per job, sequentially on one stream"},
        "speedup_vs_plain": ms_plain / ms_batch,
        "results_identical_to_plain": bool(same),
        "union_scan": {"value": world * nq / (ms_union / 1e3), "ms_per_step": ms_union,
                       "speedup_vs_plain": ms_plain / ms_union,
                       "results_identical_to_plain": bool(same_u),
                       "how": "knnjoin_self_join_batch with batch_union: every join's pass loop on "
                              "its own stream and thread, each pass scanned by one launch per "
                              "(d, buffer size) group over the union of the joins' work items, "
                              "dense first across joins"},
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


def run_join(args, rank, world, local_rank):
    """R x S: for each d in {2, 4, 6}, 2M uniform query points against 2M
    uniform data points (independent streams), K = 32, through knnjoin_join;
    sampled query rows checked against the oracle's brute force."""
    import torch
    import paper_1810_04758_b300 as kj
    from paper_1810_04758_b300 import build as kbuild

    kbuild.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    K, n = 32, 2_000_000
    sets = {}
    for d in (2, 4, 6):
        q = gen.make_points("uniform", n, d, seed=1, name=f"join_queries_{d}d")
        p = gen.make_points("uniform", n, d, seed=0, name=f"join_data_{d}d")
        sets[d] = (q, p, torch.from_numpy(q).to(dev), torch.from_numpy(p).to(dev),
                   torch.empty((n, K), dtype=torch.int32, device=dev),
                   torch.empty((n, K), dtype=torch.float64, device=dev))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    ctx = kj.Context(device=local_rank, stream=stream)

    def step():
        for d, (_, _, tq, tp, oi, od) in sets.items():
            ctx.join(tq, tp, K, oi, od)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms = []
    with ClockSampler(local_rank) as clk:
        for i in range(args.steps):
            flush.fill_(float(i))
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step()
            e.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(e))
    total = max_over_ranks(sum(ms), dev, world)
    # sampled rows against the brute-force oracle
    checked = 0
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        for d, (q, p, _, _, oi, od) in sets.items():
            rows = np.linspace(0, n - 1, 64).astype(np.int64)
            wi, wd = oracle.bf_rs(q[rows], p, K)
            assert np.array_equal(oi.cpu().numpy()[rows], wi) and np.array_equal(od.cpu().numpy()[rows], wd)
            checked += len(rows)
    ctx.close()
    if rank != 0:
        return 0
    ms_step = total / args.steps
    line = {
        "metric": "R x S query points/s (K=32, 2M queries x 2M points, 2-6D)",
        "value": world * 3 * n / (ms_step / 1e3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 (scan) + exact canonical-f64 re-score", "data": "synthetic",
        "config": {"workload": "R x S: d in {2,4,6}, 2M uniform queries (stream 1) against 2M uniform "
                               "points (stream 0), K=32, knnjoin_join",
                   "l2": "flushed (256 MiB write) before every timed step"},
        "rows_checked_against_oracle": checked,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


def run_sharded(args, rank, world, local_rank):
    """One join split over the ranks by query rows (--shard): each rank
    indexes all points and computes its row range of every join of the
    workload (shard_rows, knnjoin_self_join_rows); the total work is fixed,
    so this is strong scaling.  At N = 1 it is the step as blocking calls."""
    import torch
    import paper_1810_04758_b300 as kj
    from paper_1810_04758_b300 import build as kbuild

    kbuild.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    ctx = kj.Context(device=local_rank, stream=stream, tune_cache_path=args.tune_cache or None)
    names = WORKLOADS[args.workload]
    hosts = {nm: gen.config_points(nm) for nm in names}
    dpts = {nm: torch.from_numpy(p).to(dev) for nm, (p, K) in hosts.items()}
    ranges = {nm: kj.shard_rows(len(p), world, rank) for nm, (p, K) in hosts.items()}
    outs = {nm: (torch.empty((e - b, hosts[nm][1]), dtype=torch.int32, device=dev),
                 torch.empty((e - b, hosts[nm][1]), dtype=torch.float64, device=dev))
            for nm, (b, e) in ranges.items()}
    if not args.no_autotune:
        cached = tune_cache_keys(args.tune_cache)
        for nm in names:
            n_, d_ = hosts[nm][0].shape
            if (d_, hosts[nm][1], int(n_).bit_length() - 1) not in cached:
                ctx.autotune(dpts[nm], hosts[nm][1])
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        launches = 0
        for nm in names:
            ctx.self_join_rows(dpts[nm], hosts[nm][1], *ranges[nm], *outs[nm])
            launches += ctx.stats()["launches"]
        return launches

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms, launches = [], 0
    with ClockSampler(local_rank) as clk:
        for i in range(args.steps):
            flush.fill_(float(i))
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(stream)
            launches += step()
            e.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(e))
    if world > 1:
        torch.distributed.barrier()
    total = max_over_ranks(sum(ms), dev, world)
    ctx.close()
    if rank != 0:
        return 0
    ms_step = total / args.steps
    nq_step = sum(len(p) for p, _ in hosts.values())
    line = {
        "metric": METRIC if args.workload == "unif" else METRIC.replace("K=32", "K=64"),
        "value": nq_step / (ms_step / 1e3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "f32 (scan) + exact canonical-f64 re-score", "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT[args.workload], "n": 2_000_000, "d": [2, 4, 6],
                   "K": hosts[names[0]][1], "l2": "flushed (256 MiB write) before every timed step",
                   "parallelism": f"row shards x{world} (each rank: full index, its rows)"},
        "gpu_launches": launches,
        "step_api": "knnjoin_self_join_rows, one shard of each join per rank, blocking calls",
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


def run_index(args, rank, world, local_rank):
    """Resident index: for each d in {2, 4, 6}, 2M uniform points indexed once
    (knnjoin_index_create, untimed) and kept on the device; one step = one
    batch of uniform query points per d through knnjoin_index_query, K = 32.
    The same batches through knnjoin_join (index rebuilt per batch) are timed
    beside it; sampled rows are checked against the oracle's brute force."""
    import torch
    import paper_1810_04758_b300 as kj
    from paper_1810_04758_b300 import build as kbuild

    kbuild.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    K, n, B = 32, 2_000_000, args.batch
    nb = args.steps + args.warmup
    stream = torch.cuda.current_stream(dev)
    ctx = kj.Context(device=local_rank, stream=stream)
    sets = {}
    for d in (2, 4, 6):
        p = gen.make_points("uniform", n, d, seed=0, name=f"unif{d}d_2m")
        q = gen.make_points("uniform", nb * B, d, seed=2, name=f"index_queries_{d}d")
        tp = torch.from_numpy(p).to(dev)
        t0 = time.perf_counter()
        ix = ctx.index(tp, K)
        torch.cuda.synchronize()
        build_ms = ix.stats()["ms_total"]
        sets[d] = dict(p=p, q=q, tp=tp, tq=torch.from_numpy(q).to(dev), ix=ix, build_ms=build_ms,
                       build_wall_ms=(time.perf_counter() - t0) * 1e3,
                       oi=torch.empty((B, K), dtype=torch.int32, device=dev),
                       od=torch.empty((B, K), dtype=torch.float64, device=dev))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def batch(v, i):
        return v["tq"][i * B:(i + 1) * B]

    def timed(fn):
        for i in range(args.warmup):
            fn(i)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        ms = []
        for i in range(args.warmup, nb):
            flush.fill_(float(i))
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn(i)
            e.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(e))
        return ms

    def via_index(i):
        for v in sets.values():
            v["ix"].query(batch(v, i), K, v["oi"], v["od"])

    def via_join(i):
        for v in sets.values():
            ctx.join(batch(v, i), v["tp"], K, v["oi"], v["od"])

    with ClockSampler(local_rank) as clk:
        ms_ix = timed(via_index)
        ms_join = timed(via_join)
    total = max_over_ranks(sum(ms_ix), dev, world)
    total_join = max_over_ranks(sum(ms_join), dev, world)
    # the last batch: resident index against the oracle on sampled rows
    checked = 0
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        via_index(nb - 1)
        torch.cuda.synchronize()
        for d, v in sets.items():
            rows = np.linspace(0, B - 1, 64).astype(np.int64)
            q = v["q"][(nb - 1) * B:nb * B]
            wi, wd = oracle.bf_rs(q[rows], v["p"], K)
            assert np.array_equal(v["oi"].cpu().numpy()[rows], wi)
            assert np.array_equal(v["od"].cpu().numpy()[rows], wd)
            checked += len(rows)
    per_d = {f"{d}d": {"index_build_ms": round(v["build_ms"], 3)} for d, v in sets.items()}
    for v in sets.values():
        v["ix"].close()
    ctx.close()
    if rank != 0:
        return 0
    ms_step, ms_step_join = total / args.steps, total_join / args.steps
    line = {
        "metric": f"query points/s against a resident 2M-point index (K=32, batches of {B}, 2-6D)",
        "value": world * 3 * B / (ms_step / 1e3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 (scan) + exact canonical-f64 re-score", "data": "synthetic",
        "config": {"workload": f"resident index: d in {{2,4,6}}, 2M uniform points (seed 0) indexed once; "
                               f"one step = one batch of {B} uniform queries (stream 2) per d, K=32, "
                               f"knnjoin_index_query",
                   "l2": "flushed (256 MiB write) before every timed step"},
        "join_per_batch": {"value": world * 3 * B / (ms_step_join / 1e3), "ms_per_step": ms_step_join,
                           "api": "knnjoin_join on the same batches (index rebuilt per batch)"},
        "speedup_vs_join": ms_step_join / ms_step,
        "per_d": per_d,
        "rows_checked_against_oracle": checked,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


def run_served(args, rank, world, local_rank):
    import torch
    import paper_1810_04758_b300 as kj
    from paper_1810_04758_b300 import build as kbuild

    kbuild.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    jobs = gen.served_jobs(args.jobs or 500, seed=0)
    hosts = [gen.served_points(j) for j in jobs]
    pts = [torch.from_numpy(p).to(dev) for p in hosts]
    Ks = [j["K"] for j in jobs]
    nq = sum(len(p) for p in pts)
    torch.cuda.synchronize()
    # results of these jobs are kept and checked against the oracle on
    # sampled rows (the smallest, the largest and a spread between)
    by_size = sorted(range(len(jobs)), key=lambda k: len(hosts[k]))
    check_jobs = sorted(set(by_size[:: max(1, len(jobs) // 6)] + [by_size[-1]]))

    def serve(workers, rate, large_first=False, keep=()):
        """Submit job k at its Poisson arrival time (rate jobs/s; 0 = all at
        once), poll until done; returns (makespan s, latencies ms, kept
        outputs).  Outputs are allocated at submission and released when
        the job is done (as a server holds only the jobs in flight)."""
        ctx = kj.Context(device=local_rank, workers=workers, large_first=large_first)
        # warm the worker pipelines
        for k in range(min(len(jobs), workers)):
            ctx.self_join(pts[k][:2000].contiguous(), min(Ks[k], 1999))
        u = np.array([j["u_arrival"] for j in jobs])
        gaps = -np.log1p(-u) / rate if rate > 0 else np.zeros(len(jobs))
        arrivals = np.cumsum(gaps)
        pending, lat, live, kept = {}, {}, {}, {}
        t0 = time.perf_counter()
        k = 0
        while k < len(jobs) or pending:
            now = time.perf_counter() - t0
            # (all at once: at most 64 in flight, which saturates the pool
            # without holding every job's outputs at the same time)
            while k < len(jobs) and arrivals[k] <= now and (rate > 0 or len(pending) < 64):
                jid, oi, od = ctx.submit(pts[k], Ks[k])
                pending[jid] = k
                live[jid] = (oi, od)
                k += 1
            for jid in list(pending):
                # a finished job has its wall time set; read it, then retire
                # the job with the final poll
                stats = kj.KnnjoinStats()
                rc = kj.load_library().knnjoin_get_stats(ctx.ctx, jid, ctypes.byref(stats))
                if rc != 0 or stats.ms_wall <= 0:
                    continue
                st = ctx.poll(jid)
                if st != kj.KNN_OK:
                    raise RuntimeError(f"job failed: {ctx.last_error()}")
                kk = pending.pop(jid)
                lat[kk] = stats.ms_wall
                o = live.pop(jid)
                if kk in keep:
                    kept[kk] = o
            time.sleep(0.0002)
        span = time.perf_counter() - t0
        ctx.close()
        return span, lat, kept

    span_cap, _, kept = serve(args.workers or 8, 0.0, keep=check_jobs)
    capacity = len(jobs) / span_cap
    # sampled rows of served results against the oracle's brute force
    checked = 0
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        for kk in check_jobs:
            p = hosts[kk]
            rows = np.linspace(0, len(p) - 1, 24).astype(np.int64)
            wi, wd = oracle.bf_rows(p, Ks[kk], rows)
            gi, gd = kept[kk][0].cpu().numpy(), kept[kk][1].cpu().numpy()
            if not (np.array_equal(gi[rows], wi) and np.array_equal(gd[rows], wd)):
                raise RuntimeError(f"served job {kk}: sampled rows differ from the oracle")
            checked += len(rows)
    kept = None
    results = {}
    for rho in (0.5, 0.8, 0.95):
        rate = rho * capacity
        span, lat, _ = serve(args.workers or 8, rate)
        span1, lat1, _ = serve(1, rate)
        spanp, latp, _ = serve(args.workers or 8, rate, large_first=True)
        lv = sorted(v for v in lat.values() if v is not None)
        lv1 = sorted(v for v in lat1.values() if v is not None)
        lvp = sorted(v for v in latp.values() if v is not None)
        pct = lambda v, q: v[min(len(v) - 1, int(q * len(v)))] if v else None
        results[str(rho)] = {"arrival_jobs_per_s": rate,
                             "p50_ms": pct(lv, 0.5), "p99_ms": pct(lv, 0.99),
                             "q_per_s": nq / span,
                             "fifo_p50_ms": pct(lv1, 0.5), "fifo_p99_ms": pct(lv1, 0.99),
                             "fifo_q_per_s": nq / span1,
                             "large_first_p50_ms": pct(lvp, 0.5), "large_first_p99_ms": pct(lvp, 0.99),
                             "large_first_q_per_s": nq / spanp}
    if rank != 0:
        return 0
    top = results["0.95"]
    line = {
        "metric": "served query points/s at rho=0.95 with p50/p99 latency (Poisson join stream)",
        "value": world * top["q_per_s"], "unit": UNIT, "n_gpus": world, "steps": 1, "warmup": 1,
        "ms_per_step": span_cap * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 (scan) + exact canonical-f64 re-score", "data": "synthetic",
        "config": {"workload": f"Served: {len(jobs)} joins, {nq} points in all, n log-uniform "
                               f"[10k,5M], d 2..6, K log-uniform [8,128], 1/3 uniform, 1/3 "
                               f"exponential(40), 1/3 clustered 2-D; Poisson arrivals at rho x "
                               f"capacity", "workers": args.workers or 8},
        "capacity_jobs_per_s": capacity,
        "oracle_rows_checked": checked,
        "oracle_check": f"{checked} sampled rows of {len(check_jobs)} served joins (smallest to largest) "
                        f"equal to the oracle's brute force",
        "by_rho": results,
        "p50_ms": top["p50_ms"], "p99_ms": top["p99_ms"],
        "fifo_baseline": {"q_per_s": top["fifo_q_per_s"], "p50_ms": top["fifo_p50_ms"],
                          "p99_ms": top["fifo_p99_ms"], "how": "one worker: FIFO one job at a time"},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["batched", "served", "join", "index"],
                    default="unif")
    ap.add_argument("--jobs", type=int, default=0, help="batched/served: number of joins")
    ap.add_argument("--batch", type=int, default=16384, help="index: query points per batch")
    ap.add_argument("--shard", action="store_true",
                    help="unif/expo: split each join over the ranks by query rows (strong scaling) "
                         "instead of running replicas")
    ap.add_argument("--workers", type=int, default=0, help="batched/served: worker pipelines")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=50000,
                    help="CPU oracle: query rows per point set in one bounded sample")
    ap.add_argument("--fp32-rows", type=int, default=65536,
                    help="sampled rows per point set for the FP32-only mismatch rate (0: skip)")
    ap.add_argument("--policy", type=int, choices=[0, 1], default=0,
                    help="1: the paper's GPU-Only policy (global eps, re-index eps += eps_min/2)")
    ap.add_argument("--e2e-depth", type=int, default=2,
                    help="steps in flight in the end-to-end measurement (each holds its own pinned outputs)")
    ap.add_argument("--tune-cache", default="",
                    help="tune cache file (JSON): joins already in it are not re-tuned")
    ap.add_argument("--no-autotune", action="store_true",
                    help="use the default cell-width multiplier instead of autotuning it first")
    ap.add_argument("--configs", default="",
                    help="comma list restricting the workload's point sets (profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if args.workload not in WORKLOADS:
            print(json.dumps({"impl": "reference", "unavailable":
                              "the CPU oracle is timed on the unif/expo workloads only"}))
            return 0
        return run_reference(args, rank, world)
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    runner = {"batched": run_batched, "served": run_served, "join": run_join,
              "index": run_index}.get(args.workload, run_sharded if args.shard else run_ours)
    try:
        return runner(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
