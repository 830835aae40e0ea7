#!/usr/bin/env python3
"""Benchmark of the Fish School Behaviour per-step update on GB300.

Default workload: one school of N = 2^28 fish (seed 2), streamed from HBM,
one bench step = one step of the method over the whole school.  Prints one
JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload stream|small|resident] [--precision ...]

value      fish-steps/s over all ranks, inputs resident in HBM
e2e        the same metric through the C ABI with host buffers: host->device
           copy of the initial state, K steps with per-step statistics read
           back, device->host copy of the final state
roofline   the fused per-step pass: algorithmic bytes (32 B per fish-step in
           binary32, 64 B in binary64 state) / its average launch time, taken
           with CUDA events on the launching stream during the timed region
cpu_baseline  the CPU oracle (single thread) on a bounded sample of the
           same workload
--impl reference  times the CPU oracle, as it stands, on a bounded sample
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

import numpy as np  # noqa: E402

from paper_2507_20173_gb300 import workloads  # noqa: E402

METRIC = "fish-steps/sec and % HBM roofline on 1 GB300; batched vs per-school launches"
UNIT = "fish-steps/s"
L2_BYTES = 129 * (1 << 20)


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["stream", "small", "resident", "batch", "precision",
                                           "eat", "collective"],
                    default="stream")
    ap.add_argument("--precision-schools", type=int, default=1,
                    help="precision study: time this many schools of the 64-school "
                         "ensemble (seeds 100 + k) per mode; errors on the first")
    ap.add_argument("--batch-schools", type=int, default=None,
                    help="use only the first N schools of the batched ensemble")
    ap.add_argument("--batch-cluster", type=int, default=0)
    ap.add_argument("--no-per-school", action="store_true")
    ap.add_argument("--precision", choices=["FP32", "FP32_KAHAN", "FP64_ACC", "FP64_STATE"],
                    default="FP32_KAHAN")
    ap.add_argument("--n-fish", type=int, default=None,
                    help="override the school size (profiling on a smaller case)")
    ap.add_argument("--stream-kernel", type=int, default=0,
                    help="0 library choice, 1 vector loads, 2 bulk-copy ring, "
                         "3 warp-specialised bulk-copy ring, 4 steps blocked by recompute, "
                         "5 the same keeping the positions of the blocked steps")
    ap.add_argument("--stream-block", type=int, default=0)
    ap.add_argument("--stream-stages", type=int, default=0)
    ap.add_argument("--stream-blocks-per-sm", type=int, default=0,
                    help="blocks per SM of the streaming pass (kernels 1-3)")
    ap.add_argument("--stream-block-steps", type=int, default=0,
                    help="stream kernels 4, 5: steps per pair of passes (2, 4, 8)")
    ap.add_argument("--reference-fish", type=int, default=1 << 22,
                    help="fish per bench step of the CPU reference arm")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-runs", type=int, default=5,
                    help="end-to-end runs; the median is reported")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-sub", action="store_true",
                    help="skip the sub-records (resident school, batched ensemble, "
                         "allocation-free entry point) of the default line")
    return ap.parse_args()


def workload_of(name):
    return {"stream": workloads.STREAM, "small": workloads.SMALL,
            "resident": workloads.RESIDENT, "collective": workloads.COLLECTIVE}[name]


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def reduce_max(value, pg):
    """Max of a float over all ranks (identity on one rank).  NCCL reduces a
    CUDA tensor, gloo a CPU one."""
    if pg is None:
        return float(value)
    import torch
    dev = "cuda" if pg.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _code_only(text):
    """Source text without comments and blank runs: the profile records are
    keyed to the code, so a comment edit does not void them."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def _sources_hash(names):
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2507_20173_gb300", "csrc")
    for name in names:
        with open(os.path.join(csrc, name)) as f:
            h.update(_code_only(f.read()).encode())
    return h.hexdigest()[:16]


def kernel_source_hash():
    return _sources_hash(("fsb_stream.cu", "fsb_stream_tma.cu", "fsb_stream_ws.cu",
                          "fsb_bulk_copy.cuh", "fsb_stream_common.cuh", "fsb_device.cuh",
                          "fsb_reduce.cuh"))


# Sources of the kernels whose roofline is instruction issue (the two on-chip
# kernels and the collective-movement pass).
ALU_KERNEL_SOURCES = {
    "resident": ("fsb_resident.cu", "fsb_onchip.cuh", "fsb_check.cuh", "fsb_device.cuh",
                 "fsb_reduce.cuh"),
    "batch": ("fsb_batch.cu", "fsb_batch_wide.cu", "fsb_batch_kernel.cuh", "fsb_onchip.cuh",
              "fsb_check.cuh", "fsb_device.cuh", "fsb_reduce.cuh"),
    "collective": ("fsb_collective.cu", "fsb_device.cuh", "fsb_reduce.cuh"),
    "blocked": ("fsb_stream_blocked.cu", "fsb_stream_common.cuh", "fsb_device.cuh",
                "fsb_reduce.cuh"),
    "blocked5": ("fsb_stream_blocked.cu", "fsb_stream_common.cuh", "fsb_device.cuh",
                 "fsb_reduce.cuh"),
}


def launches_per_call(steps, coll, resident, tuning):
    """Kernel launches of one fsb_step(steps) call: the resident kernel once;
    the collective movements two passes per step and a first swim; streaming
    kernels 4 and 5 a first swim, a pair of passes per k steps after it and
    a last eat; the other streaming kernels one pass per step and a last
    eat."""
    if resident:
        return 1
    if coll:
        return 2 * steps + 1
    if tuning.get("stream_kernel") in (4, 5):
        k = tuning["stream_block_steps"]
        return 2 + 2 * ((steps - 1 + k - 1) // k)
    return steps + 1


def alu_source_hash(kernel):
    return _sources_hash(ALU_KERNEL_SOURCES[kernel])


def alu_record(kernel, precision, steps_per_pair=None):
    """The committed ncu summary of an issue-bound kernel
    (profiles/<kernel>_instr.json); None if the kernel changed since, or the
    precision or the steps per pair of passes differ."""
    p = os.path.join(ROOT, "profiles", "%s_instr.json" % kernel)
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    if d.get("kernel_source_hash") != alu_source_hash(kernel) or d.get("precision") != precision:
        return None
    if steps_per_pair is not None and d.get("steps_per_pair") != steps_per_pair:
        return None
    return d


def alu_instr_per_fish_step(kernel, precision, steps_per_pair=None):
    """Lane instructions per fish-step from the kernel's ncu summary."""
    d = alu_record(kernel, precision, steps_per_pair)
    return float(d["lane_instr_per_fish_step"]) if d else None


def issue_peak(sms, clocks):
    """Lane-instructions per second the SMs can issue: 4 schedulers x 32
    lanes per SM per clock, at the median SM clock seen in the timed region."""
    mhz = clocks.get("sm_mhz") or 2070.0
    return sms * 4 * 32 * mhz * 1e6 / 1e9


def ncu_traffic(n_fish, precision, stream_kernel):
    """DRAM bytes of one fused-pass launch of n_fish fish, from the committed
    ncu fit (profiles/stream_fused_traffic.json): bytes = slope x N +
    intercept, fitted to single launches captured at several school sizes
    (the intercept is the L2-held remainder of a launch, which does not grow
    with N).  None if no fit matches this stream kernel and precision, or the
    kernels changed since it was taken."""
    p = os.path.join(ROOT, "profiles", "stream_fused_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        records = json.load(f)["records"]
    for d in records:
        if (d.get("kernel_source_hash") == kernel_source_hash() and d.get("precision") == precision
                and d.get("stream_kernel") == stream_kernel and "slope_bytes_per_fish" in d):
            return float(d["slope_bytes_per_fish"]) * n_fish + float(d["intercept_bytes"])
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for name, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(rows),
                "power_w_max": max((num(r[3]) or 0.0) for r in rows)}


def cpu_oracle_rate(n_fish, seed, steps, collective=False):
    """Time the CPU oracle (single thread) on n_fish x steps fish-steps."""
    import oracle
    cfg = oracle.Config(n_fish=n_fish, seed=seed, collective_mode=1 if collective else 0)
    school = oracle.init(cfg)
    t0 = time.perf_counter()
    oracle.run(cfg, school, 0, steps)
    dt = time.perf_counter() - t0
    return n_fish * steps / dt, dt


def host_cpu():
    """The host's CPU model (lscpu's "Model name", else /proc/cpuinfo's
    "model name", else the machine type) and its core counts."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None and os.path.exists("/proc/cpuinfo"):
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    import platform
    return {"model": model or platform.machine(), "machine": platform.machine(),
            "nproc": os.cpu_count(), "usable": len(os.sched_getaffinity(0))}


def cpu_openmp_rate(n_fish, seed, seconds=8.0):
    """Time the oracle's step on every host core (its per-fish loops on
    OpenMP threads, the paper's parallelisation): a two-step probe sizes a
    run of about `seconds`.  Returns (rate, seconds, steps, threads)."""
    import oracle
    threads = len(os.sched_getaffinity(0))
    cfg = oracle.Config(n_fish=n_fish, seed=seed)
    school = oracle.init(cfg)
    t0 = time.perf_counter()
    oracle.run_omp(cfg, school, 0, 2, threads=threads)
    per_step = (time.perf_counter() - t0) / 2
    steps = max(1, min(100_000, int(round(seconds / per_step))))
    t0 = time.perf_counter()
    oracle.run_omp(cfg, school, 2, steps, threads=threads)
    dt = time.perf_counter() - t0
    return n_fish * steps / dt, dt, steps, threads


def measure_batch(args, world, rank, local, pg):
    """The ragged ensemble (4096 schools, log-uniform sizes in [256, 65536],
    T = 500): one graph-captured persistent launch, against the same schools
    run one launch per school (the single-school path, serially on one
    stream).  Returns the bench line (every rank)."""
    import torch

    import paper_2507_20173_gb300 as fsb
    from paper_2507_20173_gb300 import build as fsb_build

    torch.cuda.set_device(local)
    fsb_build.build()
    fsb.lib()
    wl = workloads.BATCH
    offsets, seeds = wl.offsets(), wl.seeds()
    if args.batch_schools:
        seeds = seeds[:args.batch_schools]
        offsets = offsets[:args.batch_schools + 1]
    seeds = seeds + np.uint64(rank * 100000)
    n_schools = seeds.size
    total = int(offsets[-1])
    steps = args.steps if args.steps is not None else wl.steps
    warmup = max(3, args.warmup)
    prec = getattr(fsb, "FSB_" + args.precision)
    tmpl = fsb.fsb_config_init(1, 0, precision=prec)
    stream = torch.cuda.current_stream()
    ts = [torch.zeros(total, dtype=torch.float32, device="cuda") for _ in range(4)]
    state = fsb.FsbStateDev(*(t.data_ptr() for t in ts))

    def barrier():
        torch.cuda.synchronize()
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize()

    b = fsb.fsb_batch_create(tmpl, offsets, seeds, state, init=True, stream=stream.cuda_stream)
    if args.batch_cluster:
        fsb.fsb_batch_set_cluster(b, args.batch_cluster)
    fsb.fsb_batch_step(b, warmup)
    fsb.fsb_batch_step(b, steps)          # captures the timed call's graph
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        fsb.fsb_batch_step(b, warmup)     # warm again after the sampler's start-up pause
        fsb.fsb_batch_set_timing(b, True)
        barrier()
        start.record(stream)
        fsb.fsb_batch_step(b, steps)
        stop.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms = start.elapsed_time(stop)
    kms, kl = fsb.fsb_batch_kernel_time(b)
    info = fsb.fsb_batch_info(b)
    plan = fsb.fsb_batch_plan(b)
    fsb.fsb_batch_destroy(b)
    ms_max = reduce_max(ms, pg)
    value = world * total * steps / (ms_max / 1e3)

    per_school = None
    if not args.no_per_school:
        # a stream of their own, so the calls can also be captured in a graph
        ps_stream = torch.cuda.Stream()
        handles = []
        for k in range(n_schools):
            lo, hi = int(offsets[k]), int(offsets[k + 1])
            cfg = fsb.fsb_config_init(hi - lo, int(seeds[k]), school_id=k, precision=prec)
            bufs = fsb.FsbStateDev(*(t_.data_ptr() + 4 * lo for t_ in ts))
            handles.append(fsb.fsb_create(cfg, bufs, None, 0, ps_stream.cuda_stream))
        for h in handles:
            fsb.fsb_step(h, warmup)
        barrier()
        start.record(ps_stream)
        for h in handles:
            fsb.fsb_step(h, steps)
        stop.record(ps_stream)
        torch.cuda.synchronize()
        ps_ms = start.elapsed_time(stop)
        per_school = {"value": total * steps / (ps_ms / 1e3), "unit": UNIT,
                      "ms": ps_ms, "launches": n_schools,
                      "what": "one fsb_step(T) launch per school on the single-school "
                              "path (library's choice: resident), serially on one stream"}
        # the same calls captured once into a CUDA graph and replayed: no
        # host launch cost between schools (a replay repeats the captured
        # steps' counters on the evolved state; the work per school is the
        # same)
        try:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=ps_stream):
                for h in handles:
                    fsb.fsb_step(h, steps)
            g.replay()
            torch.cuda.synchronize()
            start.record(ps_stream)
            g.replay()
            stop.record(ps_stream)
            torch.cuda.synchronize()
            gms = start.elapsed_time(stop)
            per_school["graph"] = {"value": total * steps / (gms / 1e3), "unit": UNIT,
                                   "ms": gms, "what": "the per-school calls captured in "
                                                     "one CUDA graph, one replay timed"}
            del g
        except Exception as e:  # report, do not fail the bench line
            torch.cuda.synchronize()
            per_school["graph"] = {"unavailable": str(e).splitlines()[0][:200]}
        for h in handles:
            fsb.fsb_destroy(h)
    clocks = clk.summary()
    ipfs = alu_instr_per_fish_step("batch", args.precision)
    avg_s = (kms / kl) / 1e3 if kl else None
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    roof = {"bound": "alu", "kernel": "batch_kernel", "launches": kl,
            "avg_launch_ms": avg_s * 1e3 if avg_s else None,
            "fish_steps_per_launch": total * steps, "lane_instr_per_fish_step": ipfs,
            "achieved": total * steps / avg_s * ipfs / 1e9 if (avg_s and ipfs) else None,
            "peak": issue_peak(sms, clocks), "unit": "Glane-instr/s", "traffic": None,
            "peak_source": "issue peak %d SMs x 128 lanes x measured median SM clock" % sms}
    roof["frac"] = roof["achieved"] / roof["peak"] if roof["achieved"] else None
    del ts
    torch.cuda.empty_cache()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": steps, "warmup": warmup, "ms_per_step": ms_max / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl.name if n_schools == wl.n_schools else
                       "%s (first %d schools)" % (wl.name, n_schools),
                       "n_schools": n_schools, "total_fish": total,
                       "precision": args.precision, "batch": info,
                       "launch_plan": plan,
                       "l2": "state %.2f GB; each school's state stays on chip for the call"
                             % (16 * total / 1e9),
                       "parallelism": "replicas x%d" % world},
            "roofline": roof,
            "per_school": per_school,
            "batched_over_per_school": (value / world) / per_school["value"]
            if per_school else None,
            "batched_over_per_school_graph": (value / world) / per_school["graph"]["value"]
            if per_school and "value" in per_school.get("graph", {}) else None,
            "cpu_baseline": None, "e2e": None,
            "gpu_launches": len(plan["launches"]) + 1, "clocks": clocks}
    return line


def run_batch(args, world, rank, local, pg):
    line = measure_batch(args, world, rank, local, pg)
    if rank == 0:
        print(json.dumps(line), flush=True)


def exact_sums(w, x, y):
    """Reference sums of the read-back state: binary64 products (exact for
    binary32 inputs), summed pairwise in binary64 in 4096 chunks whose sums
    are added exactly by math.fsum; relative error about 1e-15 of sum |w x|,
    far below the 1e-12 the binary64 modes are held to."""
    import math
    w64, x64, y64 = (np.asarray(a, dtype=np.float64) for a in (w, x, y))
    wx, wy = w64 * x64, w64 * y64

    def fsum_chunked(v):
        return math.fsum(np.sum(c) for c in np.array_split(v, 4096))
    return {"sum_w": fsum_chunked(w64), "sum_wx": fsum_chunked(wx), "sum_wy": fsum_chunked(wy),
            "abs_wx": float(np.sum(np.abs(wx))), "abs_wy": float(np.sum(np.abs(wy)))}


def run_precision(args, world, rank, local):
    """Precision study: schools of N = 2^24 fish from the 64-school study
    ensemble (seeds 100 + k; --precision-schools of them, one by default),
    T = 1000 steps, in each arithmetic mode.  Reports each mode's throughput
    over those schools, the error of the first school's barycentre sums at
    steps 1, 10, 100 and 1000 against the exact sums of its read-back state
    (normalised by sum |w x|), and the drift between the binary32 and the
    binary64 trajectories (the same draws, different rounding).  Beside them,
    the CPU oracle runs the first school's first 100 steps (its OpenMP step,
    binary32 and binary64 state, sums compensated in binary64 over exact
    products): every step's sums of each mode against it, its maxima, the
    whole state at step 100 bit for bit, and the binary32 modes' drift from
    the binary64 oracle's trajectory."""
    import torch

    import paper_2507_20173_gb300 as fsb
    from paper_2507_20173_gb300 import build as fsb_build

    torch.cuda.set_device(local)
    fsb_build.build()
    fsb.lib()
    n = args.n_fish or (1 << 24)
    total = args.steps if args.steps is not None else 1000
    marks = [m for m in (1, 10, 100, 1000) if m <= total]
    stream = torch.cuda.current_stream()
    modes = {}
    finals = {}
    # the oracle's trajectories of school 0 (seed 100) over the first steps
    import oracle
    ostep = min(100, total)
    if ostep not in marks:
        marks = sorted(set(marks) | {ostep})
    ocfg = oracle.Config(n_fish=n, seed=100)
    oref, ostats, otime = {}, {}, {}
    for prec in ("f32", "f64"):
        t0 = time.perf_counter()
        oref[prec] = oracle.init(ocfg, prec)
        ostats[prec] = oracle.run_omp(ocfg, oref[prec], 0, ostep)
        otime[prec] = time.perf_counter() - t0
    for name in ("FP32", "FP32_KAHAN", "FP64_ACC", "FP64_STATE"):
        cfg = fsb.fsb_config_init(n, 100, precision=getattr(fsb, "FSB_" + name),
                                  path=fsb.FSB_PATH_STREAM)
        s = fsb.School.create(cfg, stream=stream)
        errs = {}
        done = 0
        elapsed = 0.0
        gstats = []
        at_ostep = None
        start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for m in marks:
            k = m - done
            torch.cuda.synchronize()
            start.record(stream)
            st = s.step(k, stats=True)
            stop.record(stream)
            torch.cuda.synchronize()
            elapsed += start.elapsed_time(stop) / 1e3
            done = m
            gstats.append(st)
            got = s.read()
            if m == ostep:
                at_ostep = got
            ex = exact_sums(got["w"], got["x"], got["y"])
            last = st[-1]
            errs[str(m)] = {
                "sum_w": abs(last["sum_w"] - ex["sum_w"]) / abs(ex["sum_w"]),
                "sum_wx": abs(last["sum_wx"] - ex["sum_wx"]) / ex["abs_wx"],
                "sum_wy": abs(last["sum_wy"] - ex["sum_wy"]) / ex["abs_wy"],
                "bary_x_abs_err": abs(last["sum_wx"] / last["sum_w"] - ex["sum_wx"] / ex["sum_w"])}
        finals[name] = got
        s.destroy()
        # against the oracle of the same state precision, steps 1 .. ostep
        prec = "f64" if name == "FP64_STATE" else "f32"
        g = np.concatenate(gstats)[:ostep]
        o = ostats[prec]
        r = oref[prec]
        same = {k: bool(np.array_equal(at_ostep[k], r[f])) for k, f in
                (("x", "x"), ("y", "y"), ("w", "weight"), ("prev", "prevObjective"),
                 ("cur", "currentObjective"))}
        vs_oracle = {
            "steps": ostep, "oracle_state": prec,
            "max_err_sum_w": float(np.max(np.abs(g["sum_w"] - o["sum_w"]) / np.abs(o["sum_w"]))),
            "max_err_sum_wx": float(np.max(np.abs(g["sum_wx"] - o["sum_wx"]) / o["sum_abs_wx"])),
            "max_err_sum_wy": float(np.max(np.abs(g["sum_wy"] - o["sum_wy"]) / o["sum_abs_wy"])),
            "max_abs_delta_every_step_equal": bool(np.array_equal(g["max_abs_delta"],
                                                                  o["max_abs_delta"])),
            "eat_max_diff_every_step_equal": bool(np.array_equal(g["eat_max_diff"],
                                                                 o["eat_max_diff"])),
            "state_bitwise_equal_at_last_step": same}
        if prec == "f32":
            r64 = oref["f64"]
            vs_oracle["drift_from_binary64_oracle"] = {
                k: float(np.max(np.abs(at_ostep[k].astype(np.float64) - r64[f])))
                for k, f in (("x", "x"), ("y", "y"), ("w", "weight"))}
        # the ensemble's other schools, timed over the whole call
        for k in range(1, max(1, args.precision_schools)):
            cfg_k = fsb.fsb_config_init(n, 100 + k, precision=getattr(fsb, "FSB_" + name),
                                        path=fsb.FSB_PATH_STREAM)
            sk = fsb.School.create(cfg_k, stream=stream)
            torch.cuda.synchronize()
            start.record(stream)
            sk.step(total)
            stop.record(stream)
            torch.cuda.synchronize()
            elapsed += start.elapsed_time(stop) / 1e3
            sk.destroy()
        schools = max(1, args.precision_schools)
        modes[name] = {"fish_steps_per_s": schools * n * total / elapsed, "errors": errs,
                       "schools_timed": schools, "vs_oracle": vs_oracle}
    drift = {f: float(np.max(np.abs(finals["FP32_KAHAN"][f].astype(np.float64) -
                                    finals["FP64_STATE"][f])))
             for f in ("x", "y", "w")}
    drift["mean_abs_x"] = float(np.mean(np.abs(finals["FP32_KAHAN"]["x"].astype(np.float64) -
                                               finals["FP64_STATE"]["x"])))
    if rank == 0:
        line = {"metric": "precision study: barycentre error and throughput per arithmetic mode",
                "value": modes["FP32_KAHAN"]["fish_steps_per_s"], "unit": UNIT, "n_gpus": 1,
                "steps": total, "warmup": 0, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32/f64", "data": "synthetic",
                "config": {"workload": "precision %d x N=2^%d T=%d seeds 100+k"
                                       % (max(1, args.precision_schools), n.bit_length() - 1,
                                          total),
                           "note": "schools of the 64-school ensemble, timed per mode; errors "
                                   "of the first against exact host sums of its read-back "
                                   "state, and every step of its first %d against the CPU "
                                   "oracle (OpenMP step; %.1f s binary32, %.1f s binary64)"
                                   % (ostep, otime["f32"], otime["f64"])},
                "modes": modes, "trajectory_drift_fp32_vs_fp64_state": drift}
        print(json.dumps(line), flush=True)


def run_eat(args, world, rank, local):
    """The GPU analogue of the paper's Experiment 3 (reduction vs critical):
    the eat() reduction max(prev - cur) over a school's state under each
    reduction construct, timed with CUDA events (median of 5)."""
    import torch

    import paper_2507_20173_gb300 as fsb
    from paper_2507_20173_gb300 import build as fsb_build

    torch.cuda.set_device(local)
    fsb_build.build()
    fsb.lib()
    n = args.n_fish or (1 << 26)
    cfg = fsb.fsb_config_init(n, 2, path=fsb.FSB_PATH_STREAM)
    s = fsb.School.create(cfg)
    s.step(1)
    st = s.read()
    s.destroy()
    prev = torch.from_numpy(st["prev"]).cuda()
    cur = torch.from_numpy(st["cur"]).cuda()
    del st
    out = {}
    for name, c in (("reduction", fsb.FSB_EAT_REDUCTION), ("per_warp", fsb.FSB_EAT_PER_WARP),
                    ("critical", fsb.FSB_EAT_CRITICAL)):
        times, val = [], None
        for _ in range(6):
            val, ms = fsb.fsb_eat_max(prev.data_ptr(), cur.data_ptr(), n, c)
            times.append(ms)
        t = statistics.median(times[1:])
        out[name] = {"ms": t, "value": val, "GB_per_s": 8 * n / (t * 1e-3) / 1e9}
    if rank == 0:
        line = {"metric": "eat() reduction time per construct (paper Experiment 3 analogue)",
                "value": out["reduction"]["ms"], "unit": "ms", "n_gpus": 1, "steps": 5,
                "warmup": 1, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": {"workload": "eat() over N=%d fish (prev, cur of step 1, seed 2)" % n},
                "constructs": out,
                "critical_over_reduction": out["critical"]["ms"] / out["reduction"]["ms"]}
        print(json.dumps(line), flush=True)


def run_reference(args, world, rank):
    """The oracle as it stands, each bench step a bounded sample of the
    workload (2^22 fish of the same school rule, one step)."""
    wl = workload_of(args.workload)
    if rank != 0:
        return
    import oracle
    n = min(wl.n_fish, args.reference_fish)
    steps = args.steps if args.steps is not None else wl.steps
    cfg = oracle.Config(n_fish=n, seed=wl.seed,
                        collective_mode=1 if args.workload == "collective" else 0)
    school = oracle.init(cfg)
    oracle.run(cfg, school, 0, args.warmup)
    t0 = time.perf_counter()
    oracle.run(cfg, school, args.warmup, steps)
    dt = time.perf_counter() - t0
    value = n * steps / dt
    sample = "first %d fish of the %s school (same init rule), %d steps" % (n, wl.name, steps)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl.name, "n_fish_sample": n, "impl_kind": "cpu oracle"},
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def barrier(torch, pg):
    torch.cuda.synchronize()
    if pg is not None:
        pg.barrier()
    torch.cuda.synchronize()


def time_single(fsb, torch, cfg, steps, warmup, local, pg, tuning):
    """Device-resident timing of one school: `warmup` untimed steps, then one
    fsb_step(steps) call bracketed by CUDA events on the school's stream,
    with the clocks sampled meanwhile.  Each fused-pass (or resident) launch
    is also bracketed by events on that stream (fsb_set_kernel_timing)."""
    stream = torch.cuda.current_stream()
    school = fsb.School.create(cfg, stream=stream)
    if any(tuning.values()):
        fsb.fsb_set_tuning(school.handle, **tuning)
    tuning = fsb.fsb_get_tuning(school.handle)
    # the warm-up runs timed too, so the timed call reuses its timing events;
    # enabling again clears the warm-up's times
    fsb.fsb_set_kernel_timing(school.handle, True)
    school.step(warmup)
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        # warm again after the sampler's start-up pause (an idle GPU timed
        # short calls slow), then clear the warm-up's kernel times
        school.step(warmup)
        fsb.fsb_set_kernel_timing(school.handle, True)
        fsb.fsb_kernel_time(school.handle)
        barrier(torch, pg)
        start.record(stream)
        fsb.fsb_step(school.handle, steps)
        stop.record(stream)
        torch.cuda.synchronize()
    barrier(torch, pg)
    ms = start.elapsed_time(stop)
    fused_ms, fused_n = fsb.fsb_kernel_time(school.handle)
    path = fsb.fsb_handle_path(school.handle)
    school.destroy()
    return {"ms": ms, "fused_ms": fused_ms, "fused_n": fused_n, "path": path, "tuning": tuning,
            "clocks": clk.summary()}


def alu_roofline(kernel, name, precision, fish_steps_per_launch, avg_s, sms, clocks,
                 steps_per_pair=None):
    """Instruction-issue roofline of an issue-bound kernel: fish-steps per
    launch / the launch's event time x the lane-instructions per fish-step ncu
    counted (profiles/<kernel>_instr.json), against the issue peak at the
    median SM clock sampled during the timed region.  traffic: the DRAM bytes
    per fish-step of that summary (when it has them) x fish-steps per launch."""
    rec = alu_record(kernel, precision, steps_per_pair)
    ipfs = float(rec["lane_instr_per_fish_step"]) if rec else None
    bpfs = rec.get("dram_bytes_per_fish_step") if rec else None
    rate = fish_steps_per_launch / avg_s if avg_s else None
    roof = {"bound": "alu", "unit": "Glane-instr/s", "kernel": name,
            "avg_launch_ms": avg_s * 1e3 if avg_s else None,
            "fish_steps_per_launch": fish_steps_per_launch, "lane_instr_per_fish_step": ipfs,
            "traffic": bpfs * fish_steps_per_launch if bpfs else None,
            "achieved": rate * ipfs / 1e9 if (rate and ipfs) else None,
            "peak": issue_peak(sms, clocks),
            "peak_source": "issue peak %d SMs x 128 lanes x measured median SM clock" % sms}
    roof["frac"] = roof["achieved"] / roof["peak"] if roof["achieved"] else None
    return roof


def resident_record(fsb, torch, local, pg):
    """The resident school of the metric's configurations (N = 2^20, seed 1,
    T = 1000, the on-chip kernel): one call timed as the main line's."""
    wl = workloads.RESIDENT
    cfg = fsb.fsb_config_init(wl.n_fish, wl.seed, precision=fsb.FSB_FP32_KAHAN)
    # warm-up: one untimed call as long as the timed one (a call of 1000
    # steps is 4 ms; after a 3-step warm-up it timed about 7% slow)
    t = time_single(fsb, torch, cfg, wl.steps, wl.steps, local, pg, {})
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    avg_s = (t["fused_ms"] / t["fused_n"]) / 1e3 if t["fused_n"] else None
    roof = alu_roofline("resident", "resident_kernel", "FP32_KAHAN", wl.n_fish * wl.steps, avg_s,
                        sms, t["clocks"])
    roof["launches"] = t["fused_n"]
    return {"workload": wl.name, "value": wl.n_fish * wl.steps / (t["ms"] / 1e3), "unit": UNIT,
            "steps": wl.steps, "warmup": wl.steps, "ms_per_step": t["ms"] / wl.steps,
            "path": {1: "stream", 2: "resident"}.get(t["path"], str(t["path"])),
            "tuning": t["tuning"], "roofline": roof, "gpu_launches": 1, "clocks": t["clocks"]}


def static_record(fsb, torch, cfg, steps, warmup, local):
    """fsb_step_static, the allocation-free entry point, on the main line's
    school: `warmup` steps, then one call of `steps` steps on caller-owned
    arrays timed with CUDA events (its scratch is the library's static
    array; nothing is allocated)."""
    stream = torch.cuda.current_stream()
    school = fsb.School.create(cfg, stream=stream)   # its arrays, initialised
    state = fsb.FsbStateDev(*(t.data_ptr() for t in school.tensors))
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        fsb.fsb_step_static(cfg, state, 0, warmup, None, stream.cuda_stream)
        torch.cuda.synchronize()
        start.record(stream)
        fsb.fsb_step_static(cfg, state, warmup, steps, None, stream.cuda_stream)
        stop.record(stream)
        torch.cuda.synchronize()
    ms = start.elapsed_time(stop)
    school.destroy()
    del school, state
    torch.cuda.empty_cache()
    return {"value": cfg.n_fish * steps / (ms / 1e3), "unit": UNIT, "steps": steps,
            "ms_per_step": ms / steps, "gpu_launches": steps + 1,
            "what": "fsb_step_static(K) on caller-owned arrays, same school and steps",
            "clocks": clk.summary()}


def run_ours(args, world, rank, local, pg):
    import torch

    import paper_2507_20173_gb300 as fsb
    from paper_2507_20173_gb300 import build as fsb_build

    if not torch.cuda.is_available():
        raise SystemExit("bench.py: no CUDA device")
    torch.cuda.set_device(local)
    fsb_build.build()
    fsb.lib()
    wl = workload_of(args.workload)
    steps = args.steps if args.steps is not None else wl.steps
    warmup = max(3, args.warmup)
    prec = getattr(fsb, "FSB_" + args.precision)
    dbl = prec == fsb.FSB_FP64_STATE
    elem = 8 if dbl else 4
    n = args.n_fish or wl.n_fish
    coll = args.workload == "collective"
    cfg = fsb.fsb_config_init(n, wl.seed + rank, precision=prec, school_id=wl.school_id,
                              collective_mode=1 if coll else 0)
    stream = torch.cuda.current_stream()

    tuning = {"stream_kernel": args.stream_kernel, "stream_block": args.stream_block,
              "stream_stages": args.stream_stages, "stream_block_steps": args.stream_block_steps,
              "stream_blocks_per_sm": args.stream_blocks_per_sm}
    tuning_args = dict(tuning)  # as asked (tuning below becomes the handle's)

    # ---- device-resident timing
    t = time_single(fsb, torch, cfg, steps, warmup, local, pg, tuning)
    ms, fused_ms, fused_n, path, tuning = t["ms"], t["fused_ms"], t["fused_n"], t["path"], \
        t["tuning"]
    clocks = t["clocks"]
    ms_max = reduce_max(ms, pg)
    value = world * n * steps / (ms_max / 1e3)
    sms = torch.cuda.get_device_properties(local).multi_processor_count

    # ---- roofline of the dominant kernel
    peak, peak_kind = measured_peaks()
    # per fish-step: 16 B in, 16 B out; with the collective movements the
    # step's two passes move 28 B in and 20 B out (eat: x y w prev in, x y w
    # out; move: x y in, x y prev out)
    bytes_per_fish_step = (12 if coll else 8) * elem
    avg_fused_s = (fused_ms / fused_n) / 1e3 if fused_n else None
    if coll:
        # two passes per step, bound by instruction issue (grid terms, two
        # draws and three square roots per fish); HBM fraction kept beside
        roof = alu_roofline("collective", "coll_kernel<eat> + coll_kernel<move> (one step)",
                            args.precision, n, avg_fused_s, sms, clocks)
        hbm = bytes_per_fish_step * n / avg_fused_s / 1e9 if avg_fused_s else None
        roof.update({"launches": fused_n, "hbm_achieved_gbs": hbm,
                     "hbm_frac_of_measured": hbm / peak if hbm else None,
                     "algorithmic_bytes_per_launch": bytes_per_fish_step * n})
    elif tuning["stream_kernel"] in (4, 5):
        # steps blocked by recompute: each timed unit is a pair of passes
        # (maxima, step) covering up to K steps; the pairs cover steps - 1
        # steps of the call.  Bound by instruction issue; the HBM fraction of
        # its algorithmic bytes beside (x, y read by the maxima pass; x, y, w,
        # prev read and written by the step pass: 40 B per fish per pair;
        # kernel 5 also writes and reads the positions of the K steps, 16 K B)
        pair_steps = steps - 1
        per_step_s = (fused_ms / 1e3) / pair_steps if pair_steps and fused_n else None
        five = tuning["stream_kernel"] == 5
        roof = alu_roofline("blocked5" if five else "blocked",
                            "blocked_maxima_kernel + blocked_step_kernel (pairs%s)"
                            % (", positions kept" if five else ""),
                            args.precision, n, per_step_s, sms, clocks,
                            steps_per_pair=tuning["stream_block_steps"])
        pair_bytes = 40 * n * fused_n + (16 * n * pair_steps if five else 0)
        hbm = pair_bytes / (fused_ms / 1e3) / 1e9 if fused_n else None
        roof.update({"launches": fused_n, "steps_per_pair": tuning["stream_block_steps"],
                     "hbm_achieved_gbs": hbm, "hbm_frac_of_measured": hbm / peak if hbm else None,
                     "what": "avg_launch_ms and achieved are per fish-step of the pairs"})
    elif path == fsb.FSB_PATH_RESIDENT:
        # one launch advances all `steps` steps with the state on chip: bound
        # by instruction issue, 152 SMs x 4 schedulers x 32 lanes per clock
        roof = alu_roofline("resident", "resident_kernel", args.precision, n * steps,
                            avg_fused_s, sms, clocks)
        roof["launches"] = fused_n
    else:
        achieved = bytes_per_fish_step * n / avg_fused_s / 1e9 if avg_fused_s else None
        traffic = ncu_traffic(n, args.precision, tuning["stream_kernel"])
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak if achieved else None, "traffic": traffic,
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one "
                                  "fused launch, slope x N + intercept fitted over captured "
                                  "school sizes (profiles/stream_fused_traffic.json)",
                "peak_source": peak_kind + " hbm_gbs (STREAM copy)",
                "kernel": {1: "stream_pass_kernel<fused>", 2: "stream_pass_tma_kernel<fused>",
                           3: "stream_pass_ws_kernel<fused>"}[tuning["stream_kernel"]],
                "launches": fused_n,
                "avg_launch_ms": avg_fused_s * 1e3 if avg_fused_s else None,
                "algorithmic_bytes_per_launch": bytes_per_fish_step * n}

    # ---- the metric's other configurations and the allocation-free entry
    # point, measured in the same run (N = 1, default workload only)
    subs = None
    if world == 1 and args.workload == "stream" and not args.no_sub:
        subs = {"no_alloc": static_record(fsb, torch, cfg, steps, warmup, local)}
        subs["no_alloc"]["over_fsb_step"] = subs["no_alloc"]["value"] / value
        subs["resident"] = resident_record(fsb, torch, local, pg)
        bargs = argparse.Namespace(**{**vars(args), "steps": None, "warmup": 3,
                                      "batch_schools": None, "batch_cluster": 0,
                                      "no_per_school": False, "precision": "FP32_KAHAN"})
        bl = measure_batch(bargs, world, rank, local, pg)
        subs["batch"] = {k: bl[k] for k in ("value", "unit", "steps", "warmup", "ms_per_step",
                                            "config", "roofline", "per_school",
                                            "batched_over_per_school",
                                            "batched_over_per_school_graph", "gpu_launches",
                                            "clocks")}

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        npdt = np.float64 if dbl else np.float32
        init_school = fsb.School.create(cfg, stream=stream)
        host0 = init_school.read()
        init_school.destroy()
        pin = {k: torch.from_numpy(host0[k]).pin_memory() for k in ("x", "y", "w", "prev")}
        outs = {k: torch.empty(n, dtype=torch.float64 if dbl else torch.float32).pin_memory()
                for k in ("x", "y", "w", "prev", "cur")}
        dev = [torch.empty(n, dtype=torch.float64 if dbl else torch.float32, device="cuda")
               for _ in range(4)]
        bufs = fsb.FsbStateDev(*(d.data_ptr() for d in dev))
        host = fsb.FsbStateHost(*(pin[k].data_ptr() for k in ("x", "y", "w", "prev")))
        stats = np.zeros(steps, fsb.STATS_DTYPE)
        runs = []
        # one untimed round first: the pinned pages' first transfers and the
        # handle's first graph instantiation are warm-up, like the device
        # steps' warm-up
        for r_i in range(1 + args.e2e_runs):
            barrier(torch, pg)
            t0 = time.perf_counter()
            h = fsb.fsb_create(cfg, bufs, host, 0, stream.cuda_stream)
            if any(tuning_args.values()):
                fsb.fsb_set_tuning(h, **tuning_args)
            stream.synchronize()  # the state's host->device copies are in
            t1 = time.perf_counter()
            fsb.fsb_step(h, steps, stats)
            t2 = time.perf_counter()
            fsb.fsb_read_state(h, *(outs[k].numpy() for k in ("x", "y", "w", "prev", "cur")))
            t3 = time.perf_counter()
            fsb.fsb_destroy(h)
            if r_i > 0:
                runs.append((reduce_max(t3 - t0, pg), 1e3 * (t1 - t0), 1e3 * (t2 - t1),
                             1e3 * (t3 - t2)))
        med = sorted(runs)[len(runs) // 2]
        e2e = {"value": world * n * steps / med[0], "unit": UNIT,
               "h2d_bytes_per_step": int(4 * elem * n / steps),
               "d2h_bytes_per_step": int((5 * elem * n + 40 * steps) / steps),
               "what": "fsb_create from pinned host state + fsb_step(K) with host stats + "
                       "fsb_read_state to pinned host, wall clock; median of %d runs "
                       "after one untimed run" % len(runs),
               "runs_s": [r[0] for r in runs],
               "phases_ms": {"create_h2d": med[1], "step": med[2], "read_d2h": med[3]}}
        del pin, outs, dev

    # ---- CPU oracle baseline (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        # about 10 s of single-thread oracle work (~3.3e7 fish-steps/s on
        # the machine's host core): up to 2^22 fish, as many steps as that takes
        cn = min(n, 1 << 22)
        cs = max(1, min(100_000, int(round(3.2e8 / cn))))
        rate, dt = cpu_oracle_rate(cn, wl.seed, cs, collective=coll)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "%d fish x %d steps of the %s school (same init rule), %.1f s"
                         % (cn, cs, wl.name, dt), "host": host_cpu()}
        if not coll:
            # the multi-core CPU baseline beside it: the same per-fish step
            # on every host core
            orate, odt, osteps, othreads = cpu_openmp_rate(cn, wl.seed)
            cpu["openmp"] = {"value": orate, "unit": UNIT, "cores": othreads,
                             "kind": "oracle step, per-fish loops on OpenMP threads "
                                     "(static schedule, max reductions)",
                             "sample": "%d fish x %d steps of the %s school, %.1f s"
                                       % (cn, osteps, wl.name, odt)}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": steps, "warmup": warmup, "ms_per_step": ms_max / steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if dbl else "f32", "data": "synthetic",
                "config": {"workload": wl.name if n == wl.n_fish else
                           "%s (resized to N=%d)" % (wl.name, n), "n_fish": n, "seed": wl.seed,
                           "precision": args.precision,
                           "path": {1: "stream", 2: "resident"}.get(path, str(path)),
                           "l2": "inputs larger than L2 (%.1f GB state vs 129 MB L2)"
                                 % (4 * elem * n / 1e9) if 4 * elem * n > L2_BYTES
                                 else "state fits in L2 (reused across steps)",
                           "parallelism": "replicas x%d" % world, "tuning": tuning},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches_per_call(steps, coll, path == fsb.FSB_PATH_RESIDENT,
                                                  tuning),
                "clocks": clocks}
        if subs is not None:
            line["sub_records"] = subs
        print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    world, rank, local, pg = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.workload == "batch":
        run_batch(args, world, rank, local, pg)
    elif args.workload == "precision":
        run_precision(args, world, rank, local)
    elif args.workload == "eat":
        run_eat(args, world, rank, local)
    else:
        run_ours(args, world, rank, local, pg)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
