"""Benchmark of GPU Bucket Sort (deterministic sample sort) on GB300.

One step = one full sort (Algorithm 1, Steps 1-9) of a fixed synthetic array
already resident in HBM.  Default workload: n = 2^28 uint32 keys drawn
uniformly (SplitMix64), keys only.  Prints ONE JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--n N] [--dist uniform] [--key-type u32|f32|u64] [--pairs]
                  [--no-dists] [--batch-arrays 20000] [--batch-cap 2^30]
                  [--batch-u64-arrays 400]
                  [--serve-seconds 60] [--serve-rate 2000] [--serve-budget B]
                  [--merge-sort] [--cpu-sample 2^24] [--no-cpu-full]

"roofline" is the HBM roofline of the dominant kernel: its algorithmic bytes
(one read and one write of every item it moves) over its CUDA-event time,
against the measured copy bandwidth; "distributions" times the seven key
distributions and reports their spread; "cpu_baseline" is the CPU oracle on
all host cores (on a 2^24-key sample; once on the whole workload when host
memory allows; and on one core as "single_thread"); "plans" times the
measured plan table against the analytic cost model at 2^24, 2^26, 2^28.

The line also carries "served": a Poisson stream of sort jobs (2,000 per
second for 60 s, 50/50 uint32/uint64, sizes log-uniform in [2^10, 2^24],
50/50 uniform/Zipf keys, pinned host buffers in and out, 40 GB device
budget) through bsort_submit/bsort_poll, against the same arrivals sorted
one at a time (bsort_sort_keys_host, then a wait); latency = the time the
sorted keys are in host memory minus the scheduled arrival.  Its "capacity"
runs the first 4,000 jobs back to back both ways, in this process and (as
"fresh_process") in a new one started with --serve-capacity, then in this
process again, with the same buffers and with freshly pinned ones.

And "batched": the batched workload (20,000 independent
uint32 arrays, sizes log-uniform in [2^7, 2^20], scaled to at most 2^30 keys
in all, uniform keys) sorted by one bsort_sort_batch call, against the same
arrays sorted by one plain bsort_sort_keys call each, on the same stream;
"batched_u64" likewise for 400 uint64 arrays of 2^18 to 2^20 keys.

--impl reference times the CPU oracle (a plain C statement of Algorithm 1)
on the host cores, on a bounded sample of the same workload per step.
Multi-GPU: one process per GPU (torchrun); every rank sorts its own array
(independent replicas, weak scaling); no collective on the data path.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Gkeys/s (uint32, n=2^28) & HBM-roofline %"
# kernels of the launch sequence (library names -> CUDA kernel names)
KERNEL_FN = {
    "step1_3_sublist_sort": "k_sublist_sort", "step4_sample_chunks": "k_records_sort",
    "step4_sample_merge": "k_merge_pass", "step5_splitters": "k_select_splitters",
    "step4_sample_hist": "k_rec_hist", "step4_sample_radix": "k_rec_pass",
    "step4_5_radix_splitters": "k_rec_pass",
    "step6_sample_index": "k_sample_index", "step7_prefix_sum": "k_row_scan",
    "step8_relocate": "k_relocate", "step7_8_scan_relocate": "k_bucket_relocate",
    "step9_pack_units": "k_pack_units",
    "step9_bucket_sort": "k_bucket_sort", "step9_single_unit": "k_bucket_sort",
}
ALU_KERNELS = ("step1_3_sublist_sort", "step9_bucket_sort", "step9_single_unit")
UNIT = "Gkeys/s"
# the sources each kernel is built from (a traffic record is valid while they
# are unchanged)
_CSRC = "paper_1002_4464_gb300/csrc/"
KERNEL_SOURCES = {
    "k_sublist_sort": [_CSRC + "bsort_sort.cuh", _CSRC + "bsort_device.cuh",
                       _CSRC + "bsort_radix.cuh", _CSRC + "bsort_sort_keys_radix.cu"],
    "k_bucket_sort": [_CSRC + "bsort_sort.cuh", _CSRC + "bsort_device.cuh",
                      _CSRC + "bsort_radix.cuh", _CSRC + "bsort_sort_keys_radix.cu"],
}
KERNEL_SOURCES_DEFAULT = [_CSRC + "bsort_kernels.cu", _CSRC + "bsort_device.cuh"]


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=1 << 28)
    p.add_argument("--dist", default="uniform")
    p.add_argument("--key-type", default="u32", choices=["u32", "f32", "u64"],
                   help="u64: uniform 64-bit keys (the --dist option is ignored)")
    p.add_argument("--small-reps", type=int, default=200,
                   help="2^20-key sorts repeated with and without CUDA-graph replay (0: skip)")
    p.add_argument("--pairs", action="store_true",
                   help="key-value pairs: uint32 keys with uint32 values = original index "
                        "(bsort_sort_pairs); e2e is not taken")
    p.add_argument("--no-dists", dest="dists", action="store_false",
                   help="skip timing every distribution (the spread across distributions)")
    p.add_argument("--dists", dest="dists", action="store_true",
                   help="time every distribution (the default)")
    p.add_argument("--e2e-steps", type=int, default=3)
    p.add_argument("--cpu-sample", type=int, default=1 << 24,
                   help="keys per CPU-oracle sample (all host cores)")
    p.add_argument("--no-cpu-full", dest="cpu_full", action="store_false",
                   help="skip timing the CPU oracle once on the whole workload")
    p.add_argument("--no-plans", dest="plans", action="store_false",
                   help="skip timing the tabled plans against the cost model's")
    p.add_argument("--merge-sort", action="store_true",
                   help="sort the 32768-key chunks of Steps 2 and 9 by comparisons "
                        "(BSORT_FLAG_MERGE_SORT) instead of by digits")
    p.add_argument("--tile", type=int, default=0, help="force the sublist size t (0: planner)")
    p.add_argument("--samples", type=int, default=0, help="force s (0: planner)")
    p.add_argument("--buckets", type=int, default=0,
                   help="force the bucket count b (0: b = s if --samples, else planner)")
    p.add_argument("--batch-arrays", type=int, default=20000,
                   help="batched workload: number of arrays (0: skip the batched line)")
    p.add_argument("--batch-cap", type=int, default=1 << 30,
                   help="batched workload: total keys at most")
    p.add_argument("--batch-steps", type=int, default=3)
    p.add_argument("--batch-u64-arrays", type=int, default=400,
                   help="64-bit batched workload: number of arrays, sizes log-uniform in "
                        "[2^18, 2^20] (0: skip the batched_u64 line)")
    p.add_argument("--serve-seconds", type=float, default=60.0,
                   help="served stream: seconds of Poisson arrivals (0: skip the served line)")
    p.add_argument("--serve-rate", type=float, default=2000.0, help="arrivals per second")
    p.add_argument("--serve-budget", type=int, default=40 << 30, help="device bytes")
    p.add_argument("--serve-capacity", action="store_true",
                   help="only the closed-loop capacity of the served workload (one JSON line); "
                        "the served section runs it this way in a fresh process")
    return p.parse_args()


def _dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _kernel_hash(kernel):
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES.get(kernel, KERNEL_SOURCES_DEFAULT):
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _traffic_for(kernel, workload):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    e = d.get("kernels", {}).get(kernel)
    if not e or e.get("workload") != workload:
        return None
    if e.get("sources_sha256_16") != _kernel_hash(kernel):
        return None
    return e.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def _cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_oracle_rate(keys_np, key_type, t, s, threads=1):
    """Time the CPU oracle (Algorithm 1 in plain C; with threads > 1 its
    per-sublist and per-bucket loops spread over that many threads) on one
    sample; returns (Gkeys/s, seconds)."""
    import oracle
    t0 = time.perf_counter()
    oracle.paper_sort(keys_np, t, s, key_type, intermediates=False, threads=threads)
    dt = time.perf_counter() - t0
    return keys_np.size / dt / 1e9, dt


def _mem_available_bytes():
    try:
        with open("/proc/meminfo") as f:
            for ln in f:
                if ln.startswith("MemAvailable:"):
                    return int(ln.split()[1]) * 1024
    except OSError:
        pass
    return 0


def _oracle_plan(n):
    """Sublist size and sample count for the CPU oracle sample: the paper's
    own choice for its Tesla-era runs, n/m = 2K items and s = 64
    (Section 4)."""
    return 2048, 64


def _sample_keys(args, rank, count):
    import synth
    if args.key_type == "f32":
        return synth.keys_f32(args.dist, count, synth.seed_for(2, _dist_index(args.dist), rank))
    if args.key_type == "u64":
        return synth.keys_u64(count, synth.seed_for(2, _dist_index(args.dist), rank))
    return synth.keys_u32(args.dist, count, synth.seed_for(2, _dist_index(args.dist), rank))


def _kb(args):
    """Bytes per item of the workload (key, plus the value of a pair)."""
    return 8 if args.key_type == "u64" or getattr(args, "pairs", False) else 4


def _dist_index(name):
    import synth
    if name in synth.DISTRIBUTIONS:
        return synth.DISTRIBUTIONS.index(name)
    return len(synth.DISTRIBUTIONS) + ("zipf", "16distinct").index(name)


def job_time_ms(local_ms, world, device):
    """Time of the whole job: the slowest rank's timed region (max over ranks)."""
    if world <= 1:
        return float(local_ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(n_per_rank, world, steps, ms_total):
    """Whole-job keys per second in G: every rank sorts its own n keys per
    step (independent replicas), over the slowest rank's time."""
    return n_per_rank * world * steps / (ms_total / 1e3) / 1e9


def _cpu_baseline(args, keys):
    """The CPU oracle on the machine's host cores: all cores on a bounded sample
    of this workload (the reported value), one core on a smaller sample, and
    all cores once on the whole workload when host memory allows."""
    import numpy as np
    cores = _cpu_cores()
    ktype = {"u32": np.uint32, "f32": np.uint32, "u64": np.uint64}[args.key_type]

    def rates(count, threads, budget_s, max_reps):
        t_o, s_o = _oracle_plan(count)
        knp = keys[:count].cpu().numpy().view(ktype)
        rs, spent = [], 0.0
        while spent < budget_s and len(rs) < max_reps:
            r, dt = cpu_oracle_rate(knp, args.key_type, t_o, s_o, threads)
            rs.append(r)
            spent += dt
        return statistics.median(rs), len(rs), t_o, s_o

    n_mt = min(args.cpu_sample, args.n)
    v_mt, reps_mt, t_o, s_o = rates(n_mt, cores, 10.0, 5)
    n_st = min(1 << 22, args.n)
    v_st, reps_st, _, _ = rates(n_st, 1, 5.0, 3)
    cpu = {"value": v_mt, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": "first %d keys of this workload, %d repetitions (median), Algorithm 1 "
                     "with t=%d, s=%d, its per-sublist and per-bucket loops on %d threads%s"
                     % (n_mt, reps_mt, t_o, s_o, cores, ", keys only" if args.pairs else ""),
           "single_thread": {"value": v_st, "unit": UNIT, "cores": 1,
                             "sample": "first %d keys, %d repetitions (median)"
                                       % (n_st, reps_st)}}
    # the whole workload once: about 64 bytes of oracle state per key
    need = args.n * 64
    if args.cpu_full and args.n > n_mt and _mem_available_bytes() > 2 * need:
        try:
            t_o, s_o = _oracle_plan(args.n)
            knp = keys.cpu().numpy().view(ktype)
            r, dt = cpu_oracle_rate(knp, args.key_type, t_o, s_o, cores)
            cpu["full_workload"] = {"value": r, "unit": UNIT, "cores": cores,
                                    "seconds": dt, "n": args.n}
            del knp
        except (MemoryError, ValueError) as e:
            cpu["full_workload"] = {"error": "%s: %s" % (type(e).__name__, str(e)[:120])}
    return cpu


def run_reference(args):
    rank, world, local = _dist_env()
    if rank != 0:
        return 0
    sample_n = min(args.cpu_sample, args.n)
    keys = _sample_keys(args, 0, sample_n)
    t, s = _oracle_plan(sample_n)
    cores = _cpu_cores()
    for _ in range(args.warmup):
        cpu_oracle_rate(keys, args.key_type, t, s, cores)
    times = []
    for _ in range(args.steps):
        _, dt = cpu_oracle_rate(keys, args.key_type, t, s, cores)
        times.append(dt)
    total = sum(times)
    value = sample_n * len(times) / total / 1e9
    sample_desc = ("first %d keys of the %s %s workload (n=%d), Algorithm 1 with t=%d, s=%d, "
                   "per-sublist and per-bucket loops on %d threads, per step"
                   % (sample_n, args.dist, args.key_type, args.n, t, s, cores))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total / len(times) * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.key_type,
        "data": "synthetic", "config": _config(args, world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample_desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)
    return 0


def _config(args, world):
    what = ("key-value (uint32 value = original index) sort" if getattr(args, "pairs", False)
            else "keys-only sort")
    return {"workload": "%s %s %s, n=2^%d per GPU" % (
                args.dist, args.key_type, what, max(args.n.bit_length() - 1, 0))
            if args.n & (args.n - 1) == 0
            else "%s %s %s, n=%d per GPU" % (args.dist, args.key_type, what, args.n),
            "n": args.n, "key_type": args.key_type, "distribution": args.dist,
            "global_keys": args.n * world, "parallelism": "replicas x%d" % world,
            "l2_policy": "input (%d MB) larger than the 129 MB L2; no flush" % (args.n * _kb(args) >> 20)
            if args.n * _kb(args) > 129 * 2 ** 20 else "input smaller than L2 (resident)"}


def _small_sorts(args, pkg, synth, dev, local, rank, stream, sorter):
    """2^20 uint32 keys sorted args.small_reps times on the same buffers,
    with a launch per kernel and with one CUDA-graph launch per sort."""
    import torch
    ns = 1 << 20
    ks = synth.keys_u32_torch("uniform", ns, synth.seed_for(2, 0, rank), device=dev)
    os_ = torch.empty_like(ks)
    side = torch.cuda.Stream(device=dev)
    side.wait_stream(stream)
    out = {"n": ns, "reps": args.small_reps,
           "kernels_per_sort": sorter.plan(ns, "u32").num_kernels}
    with torch.cuda.stream(side):
        for graphs in (False, True):
            s2 = pkg.BucketSorter(device=local, graphs=graphs)
            for _ in range(5):
                s2.sort_keys(ks, out=os_)
            s2.sync()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(side)
            for _ in range(args.small_reps):
                s2.sort_keys(ks, out=os_)
            b.record(side)
            side.synchronize()
            s2.sync()
            out["ms_per_sort_graph" if graphs else "ms_per_sort_launches"] = \
                a.elapsed_time(b) / args.small_reps
            s2.close()
    stream.wait_stream(side)
    out["speedup"] = out["ms_per_sort_launches"] / out["ms_per_sort_graph"]
    return out


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_1002_4464_gb300 as pkg
    import synth

    rank, world, local = _dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    def make_keys(dname):
        seed = synth.seed_for(2, _dist_index(dname), rank)
        if dname in ("zipf", "16distinct"):  # heavy-duplicate uint32 keys
            kn = synth.keys_zipf(args.n, seed) if dname == "zipf" else synth.keys_16distinct(args.n, seed)
            return torch.from_numpy(kn.view(np.int32)).to(dev)
        if args.key_type == "f32":
            return synth.keys_f32_torch(dname, args.n, seed, device=dev)
        if args.key_type == "u64":
            return synth.draws64_torch(seed, args.n, device=dev)
        return synth.keys_u32_torch(dname, args.n, seed, device=dev)

    if args.pairs and args.key_type != "u32":
        raise SystemExit("--pairs takes uint32 keys")
    keys = make_keys(args.dist)
    out = torch.empty_like(keys)
    vals = torch.arange(args.n, dtype=torch.int32, device=dev) if args.pairs else None
    out_v = torch.empty_like(vals) if args.pairs else None
    sorter = pkg.BucketSorter(device=local, timing=True, tile=args.tile, samples=args.samples,
                              buckets=args.buckets, merge_sort=args.merge_sort)
    plan = sorter.plan(args.n, args.key_type)
    stream = torch.cuda.current_stream(dev)

    def one_step(k_in):
        if args.pairs:
            sorter.sort_pairs(k_in, vals, out_keys=out, out_vals=out_v)
        else:
            sorter.sort_keys(k_in, out=out, key_type=args.key_type)

    for _ in range(max(args.warmup, 3)):
        one_step(keys)
    sorter.sync()
    # correctness gate (outside the timed region): nondecreasing and same multiset
    o = out.view(torch.int32).to(torch.int64) & 0xFFFFFFFF if args.key_type == "u32" else None
    if o is not None:
        assert bool((o[1:] >= o[:-1]).all()), "output not sorted"
        kin = keys.view(torch.int32).to(torch.int64) & 0xFFFFFFFF
        assert int(kin.sum()) == int(o.sum()), "multiset changed"
        del kin
        if args.pairs:  # stable: equal keys keep their original order (value = index)
            same = o[1:] == o[:-1]
            assert bool((out_v[1:][same] > out_v[:-1][same]).all()), "not stable"
            assert bool((keys[out_v.long()] == out).all()), "values do not follow keys"
            del same
    if args.key_type == "u64":  # unsigned order = signed order with the top bit flipped
        o = out ^ torch.tensor(-(1 << 63), dtype=torch.int64, device=dev)
        assert bool((o[1:] >= o[:-1]).all()), "output not sorted"
        assert int(keys.sum()) == int(out.sum()), "multiset changed"
    del o
    sorter.kernel_times()  # reset the timing ring

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        one_step(keys)
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms_total = ev0.elapsed_time(ev1)
    sorter.sync()
    ktimes, kcalls = sorter.kernel_times()
    ms_total = job_time_ms(ms_total, world, dev)
    ms_step = ms_total / args.steps
    value = job_throughput(args.n, world, args.steps, ms_total)

    # per-kernel breakdown and the dominant kernel's roofline
    per_kernel = {}
    launches_per_kernel = {}
    for name, ms in ktimes:
        per_kernel[name] = per_kernel.get(name, 0.0) + ms / max(kcalls, 1)
        launches_per_kernel[name] = launches_per_kernel.get(name, 0) + 1
    dom = max(per_kernel, key=per_kernel.get) if per_kernel else None
    hbm_peak, peak_kind = _peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    roofline = None
    if dom is not None:
        dom_ms = per_kernel[dom] / launches_per_kernel[dom]
        # HBM roofline of the dominant kernel: its algorithmic bytes are the
        # one read and one write of every item it moves (Steps 2, 8 and 9
        # each pass the whole array once), over its CUDA-event time
        alg = 2 * plan.n_padded * _kb(args)
        achieved = alg / (dom_ms / 1e3) / 1e9
        roofline = {"bound": "hbm", "kernel": KERNEL_FN.get(dom, dom), "achieved": achieved,
                    "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                    "peak_kind": peak_kind, "alg_bytes_per_launch": alg,
                    "ms_per_launch": dom_ms, "sm_count": sm_count}
        roofline["traffic"] = _traffic_for(KERNEL_FN.get(dom, dom), _config(args, 1)["workload"])
        if args.merge_sort and dom in ALU_KERNELS:
            # the comparison sort's own ceiling: 2 integer ops (compare +
            # select) per item per merge level on the integer ALU pipe
            # (16 lanes x 4 sub-partitions per SM) at the sampled clock
            unit = plan.unit_capacity if dom != "step1_3_sublist_sort" else plan.t
            levels = max(1, (int(unit) - 1).bit_length())
            ops = 2.0 * args.n * levels
            mhz = clk.get("sm_mhz") or 2070.0
            alu_peak = sm_count * 64 * mhz * 1e6 / 1e12
            roofline["alu_view"] = {"achieved": ops / (dom_ms / 1e3) / 1e12, "peak": alu_peak,
                                    "unit": "Tops/s",
                                    "frac": ops / (dom_ms / 1e3) / 1e12 / alu_peak,
                                    "peak_kind": "derived: %d SMs x 64 int ops/clk x %.0f MHz"
                                                 % (sm_count, mhz)}
        # whole-step HBM roofline: three read+write passes (Steps 2, 8, 9)
        whole = 6 * args.n * _kb(args) / (ms_step / 1e3) / 1e9
        roofline["step_hbm_achieved_gbs"] = whole
        roofline["step_hbm_peak_gbs"] = hbm_peak
        roofline["step_hbm_frac"] = whole / hbm_peak

    # end to end through the C ABI with host buffers (pinned), copies inside
    e2e = None
    if args.e2e_steps > 0 and not args.pairs:
        h_in = keys.cpu().pin_memory()
        h_out = torch.empty_like(h_in).pin_memory()
        sorter.sort_keys_host(h_in, h_out, key_type=args.key_type)  # warm-up (workspace)
        sorter.sync()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.e2e_steps):
            sorter.sort_keys_host(h_in, h_out, key_type=args.key_type)
        e1.record(stream)
        torch.cuda.synchronize()
        sorter.sync()
        ems = e0.elapsed_time(e1) / args.e2e_steps
        e2e = {"value": args.n / (ems / 1e3) / 1e9 * world, "unit": UNIT,
               "h2d_bytes_per_step": args.n * _kb(args),
               "d2h_bytes_per_step": args.n * _kb(args),
               "ms_per_step": ems}
        del h_in, h_out

    # a small sort repeated on the same buffers: one launch per kernel
    # against one graph launch per sort (BSORT_FLAG_GRAPHS), on a created
    # stream (the legacy default stream cannot be captured)
    small = None
    if args.small_reps > 0:
        try:
            small = _small_sorts(args, pkg, synth, dev, local, rank, stream, sorter)
        except Exception as e:  # reported, not fatal: the headline stands
            small = {"error": "%s: %s" % (type(e).__name__, str(e)[:200])}

    # the measured plan table against the analytic cost model on prefixes
    # of this workload (keys-only 32-bit sorts; the table covers them)
    plans = None
    if args.plans and not args.pairs and args.key_type != "u64":
        plans = {}
        for lg in (24, 26, 28):
            nn = 1 << lg
            if nn > args.n:
                continue
            row = {}
            for label, flags in (("table", 0), ("cost_model", pkg.BSORT_FLAG_PLAN_MODEL)):
                srt = pkg.BucketSorter(device=local, flags=flags)
                pl = srt.plan(nn, args.key_type)
                ki, ko = keys[:nn], out[:nn]
                for _ in range(3):
                    srt.sort_keys(ki, out=ko, key_type=args.key_type)
                srt.sync()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                reps = max(5, (1 << 28) // nn * 2)
                a.record(stream)
                for _ in range(reps):
                    srt.sort_keys(ki, out=ko, key_type=args.key_type)
                b.record(stream)
                torch.cuda.synchronize()
                srt.sync()
                pms = a.elapsed_time(b) / reps
                row[label] = {"ms_per_sort": pms, "gkeys_s": nn / (pms / 1e3) / 1e9,
                              "t": pl.t, "s": pl.s, "b": pl.b}
                srt.close()
            plans["2^%d" % lg] = row

    dists = None
    if args.dists:
        dists = {}
        for dname in (("uniform", "zipf", "16distinct") if args.pairs else synth.DISTRIBUTIONS):
            kd = make_keys(dname)
            for _ in range(3):
                one_step(kd)
            torch.cuda.synchronize()
            sorter.sync()
            sorter.kernel_times()  # drop the warm-up calls from the timing ring
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            reps = max(3, args.steps // 2)
            a.record(stream)
            for _ in range(reps):
                one_step(kd)
            b.record(stream)
            torch.cuda.synchronize()
            dms = a.elapsed_time(b) / reps
            sorter.sync()
            kt, kc = sorter.kernel_times()
            dk = {}
            for name, ms in kt:
                dk[name] = round(dk.get(name, 0.0) + ms / max(kc, 1), 4)
            dists[dname] = {"ms_per_step": dms, "gkeys_s": args.n / (dms / 1e3) / 1e9,
                            "per_kernel_ms": dk}
            del kd
        rates = [v["ms_per_step"] for v in dists.values()]
        dists["spread"] = (max(rates) - min(rates)) / (sum(rates) / len(rates))

    cpu = None
    if rank == 0 and args.cpu_sample > 0:
        cpu = _cpu_baseline(args, keys)

    sorter.close()
    del keys, out, vals, out_v
    batched = run_batched(args, pkg, synth, dev, stream, rank, world) if args.batch_arrays else None
    batched_u64 = None
    if args.batch_u64_arrays:
        try:
            batched_u64 = run_batched(args, pkg, synth, dev, stream, rank, world, wide=True)
        except Exception as exc:  # reported in the line; the headline stands
            if world > 1:
                raise  # the other ranks wait in its collectives
            import traceback
            traceback.print_exc()
            batched_u64 = {"error": "%s: %s" % (type(exc).__name__, exc)}
    served = run_served(args, pkg, synth, dev, rank) if args.serve_seconds > 0 else None

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": args.key_type + ("+u32" if args.pairs else ""),
            "data": "synthetic (SplitMix64 %s keys)" % args.dist,
            "config": _config(args, world), "roofline": roofline, "cpu_baseline": cpu,
            "e2e": e2e, "gpu_launches": plan.num_kernels * args.steps,
            "clocks": clk, "per_kernel_ms": per_kernel,
            "plan": {k: v for k, v in plan.as_dict().items()
                     if k in ("t", "s", "b", "m", "w", "bucket_bound", "unit_capacity",
                              "tile_ctas", "unit_ctas", "num_kernels")},
        }
        if small is not None:
            line["small_sort"] = small
        if dists is not None:
            line["distributions"] = dists
        if plans is not None:
            line["plans"] = plans
        if batched is not None:
            line["batched"] = batched
        if batched_u64 is not None:
            line["batched_u64"] = batched_u64
        if served is not None:
            line["served"] = served
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def _batched_graph(pkg, dev, stream, keys, off, out, ref, ktype, steps, world):
    """The batch through the batch-graph cache (BSORT_FLAG_GRAPHS) on a
    created stream (the legacy default stream cannot be captured): after the
    first call, one graph launch per call and no planning on the host."""
    import torch

    side = torch.cuda.Stream(device=dev)
    side.wait_stream(stream)
    gsort = pkg.BucketSorter(device=dev.index, graphs=True)
    with torch.cuda.stream(side):
        for _ in range(2):
            gsort.sort_batch(keys, off, out=out, key_type=ktype)
        gsort.sync()
        torch.cuda.synchronize()
        assert torch.equal(out, ref), "graph replay differs from the plain batch"
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        t_host = time.perf_counter()
        g0.record(side)
        for _ in range(steps):
            gsort.sort_batch(keys, off, out=out, key_type=ktype)
        g1.record(side)
        g_host_ms = (time.perf_counter() - t_host) * 1e3 / steps
        torch.cuda.synchronize()
        gsort.sync()
    g_ms = g0.elapsed_time(g1) / steps
    gsort.close()
    stream.wait_stream(side)
    return {"value": keys.numel() * world / (g_ms / 1e3) / 1e9, "unit": UNIT,
            "ms_per_batch": g_ms, "host_ms_per_call": g_host_ms,
            "launch": "one CUDA-graph launch per call (BSORT_FLAG_GRAPHS)"}


def run_batched(args, pkg, synth, dev, stream, rank, world, wide=False):
    """The batched workload: one bsort_sort_batch call per step against one
    plain bsort_sort_keys call per array (same arrays, same stream).  wide:
    the 64-bit workload (args.batch_u64_arrays uint64 arrays, sizes
    log-uniform in [2^18, 2^20]: the segments sorted by the 64-bit
    segment-aware sample sort)."""
    import numpy as np
    import torch

    ktype = "u64" if wide else "u32"
    kb = 8 if wide else 4
    if wide:
        sizes = synth.batch_sizes(args.batch_u64_arrays, synth.seed_for(4, 9, rank),
                                  lo_log2=18, hi_log2=20, cap=1 << 40)
    else:
        sizes = synth.batch_sizes(args.batch_arrays, synth.seed_for(4, 0, rank),
                                  cap=args.batch_cap)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    nb = int(off[-1])
    if wide:
        keys = synth.draws64_torch(synth.seed_for(4, 9, 1000 + rank), nb, device=dev)
    else:
        keys = synth.keys_u32_torch("uniform", nb, synth.seed_for(4, 0, 1000 + rank), device=dev)
    out = torch.empty_like(keys)
    sorter = pkg.BucketSorter(device=dev.index, timing=True)
    bplan = sorter.plan_batch(off, ktype)
    for _ in range(3):
        sorter.sort_batch(keys, off, out=out, key_type=ktype)
    sorter.sync()
    # correctness gate: nondecreasing inside every array (unsigned order),
    # same multiset (sums of the 32-bit halves)
    if wide:
        o = out ^ (-(1 << 63))  # unsigned order as signed order
        halves = [(out & 0xFFFFFFFF, (out >> 32) & 0xFFFFFFFF),
                  (keys & 0xFFFFFFFF, (keys >> 32) & 0xFFFFFFFF)]
        sums_out = [int(h.sum()) for h in halves[0]]
        sums_in = [int(h.sum()) for h in halves[1]]
        del halves
    else:
        o = out.view(torch.int32).to(torch.int64) & 0xFFFFFFFF
        kin = keys.view(torch.int32).to(torch.int64) & 0xFFFFFFFF
        sums_out, sums_in = [int(o.sum())], [int(kin.sum())]
        del kin
    starts = torch.zeros(nb, dtype=torch.bool, device=dev)
    starts[torch.from_numpy(off[:-1].astype(np.int64)).to(dev)] = True
    assert bool(((o[1:] >= o[:-1]) | starts[1:]).all()), "a batched array is not sorted"
    assert sums_in == sums_out, "multiset changed"
    del o, starts
    ref = out.clone()
    sorter.kernel_times()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    t_host = time.perf_counter()
    e0.record(stream)
    for _ in range(args.batch_steps):
        sorter.sort_batch(keys, off, out=out, key_type=ktype)
    e1.record(stream)
    host_ms = (time.perf_counter() - t_host) * 1e3 / args.batch_steps
    torch.cuda.synchronize()
    sorter.sync()
    kt, kc = sorter.kernel_times()
    per_kernel = {}
    for name, ms in kt:
        per_kernel[name] = round(per_kernel.get(name, 0.0) + ms / max(kc, 1), 4)
    b_ms = job_time_ms(e0.elapsed_time(e1), world, dev) / args.batch_steps
    sorter.close()

    graph = None
    if not wide:
        graph = _batched_graph(pkg, dev, stream, keys, off, out, ref, ktype, args.batch_steps,
                               world)
    del ref

    # the same arrays, one plain sort call each
    plain = pkg.BucketSorter(device=dev.index)
    plain._ensure(int(sizes.max()), ktype, 0)
    h, st = plain.h, plain._stream()
    kp, op = keys.data_ptr(), out.data_ptr()
    bounds = [(int(off[q]) * kb, int(off[q + 1] - off[q])) for q in range(len(sizes))]
    kcode = pkg.BSORT_U64 if wide else pkg.BSORT_U32

    def sequential():
        for a, n in bounds:
            pkg.bsort_sort_keys(h, kcode, kp + a, op + a, n, st)

    sequential()
    plain.sync()
    torch.cuda.synchronize()
    e0.record(stream)
    sequential()
    e1.record(stream)
    torch.cuda.synchronize()
    plain.sync()
    s_ms = job_time_ms(e0.elapsed_time(e1), world, dev)
    plain.close()
    if wide:
        workload = ("%d uint64 arrays, sizes log-uniform in [2^18, 2^20], uniform keys, per GPU"
                    % len(sizes))
    else:
        workload = ("%d uint32 arrays, sizes log-uniform in [2^7, 2^20] scaled to <= %d keys "
                    "in all, uniform keys, per GPU" % (len(sizes), args.batch_cap))
    return {"workload": workload,
            "keys": nb, "value": nb * world / (b_ms / 1e3) / 1e9, "unit": UNIT,
            "ms_per_batch": b_ms, "steps": args.batch_steps,
            "sequential": {"value": nb * world / (s_ms / 1e3) / 1e9, "unit": UNIT,
                           "ms_per_batch": s_ms,
                           "launch": "one bsort_sort_keys call per array, same stream"},
            "speedup_vs_sequential": s_ms / b_ms, "gpu_launches": bplan.num_kernels,
            "host_ms_per_call": host_ms,
            **({"graph": graph} if graph is not None else {}),
            "plan": bplan.as_dict(), "per_kernel_ms": per_kernel}


def _serve_capacity(args, pkg, dev, job, ring, maxn, ncap, cap_keys):
    """The first ncap jobs of the served trace back to back (closed loop):
    through the request loop with up to `ring` jobs in flight, and one at a
    time through bsort_sort_keys_host.  Each way first runs the first
    quarter of the jobs untimed (warm-up: after the open-loop runs the GPU
    has been mostly idle for minutes)."""
    def capacity_served(count):
        srv2 = pkg.SortServer(device=dev.index, budget_bytes=args.serve_budget)
        kt, a, b, n, _, _ = job(0, 0)
        w = pkg.bsort_submit(srv2.h, kt, a, b, min(n, 4096))
        while pkg.bsort_poll(srv2.h, w) is None:
            time.sleep(1e-4)
        free2, infl2 = list(range(ring)), {}
        c0 = pkg.bsort_clock_ns()
        k = fin = 0
        while fin < count:
            while k < count and free2:
                slot = free2.pop()
                kt, a, b, n, _, _ = job(k, slot)
                infl2[pkg.bsort_submit(srv2.h, kt, a, b, n)] = slot
                k += 1
            finished = pkg.bsort_poll_any(srv2.h, 256)
            for t, _ in finished:
                free2.append(infl2.pop(t))
                fin += 1
            if not finished:
                time.sleep(1e-5)
        dt = (pkg.bsort_clock_ns() - c0) / 1e9
        srv2.close()
        return dt

    def capacity_one(count):
        one2 = pkg.BucketSorter(device=dev.index)
        one2._ensure(maxn, "u64", 0, extra=maxn * 8 + 512)
        s2 = one2._stream()
        c0 = pkg.bsort_clock_ns()
        for k in range(count):
            kt, a, b, n, _, _ = job(k, 0)
            pkg.bsort_sort_keys_host(one2.h, kt, a, b, n, s2)
            one2.sync()
        dt = (pkg.bsort_clock_ns() - c0) / 1e9
        one2.close()
        return dt

    capacity_served(max(1, ncap // 4))
    dt_s = capacity_served(ncap)
    capacity_one(max(1, ncap // 4))
    dt_o = capacity_one(ncap)
    return {"jobs": ncap, "keys": cap_keys,
            "served_gkeys_s": cap_keys / dt_s / 1e9,
            "one_at_a_time_gkeys_s": cap_keys / dt_o / 1e9,
            "speedup": dt_o / dt_s,
            "how": "the first jobs of the trace back to back (closed loop), after an untimed "
                   "warm-up on the first quarter of them"}


def _serve_capacity_subprocess(args):
    """_serve_capacity in a fresh process (this script with --serve-capacity):
    in a process that has already run the other sections, the request loop's
    closed-loop capacity measures lower with the pinned buffers the open-loop
    runs used (freshly pinned buffers restore it; reported beside it)."""
    cmd = [sys.executable, os.path.abspath(__file__), "--serve-capacity",
           "--serve-seconds", repr(args.serve_seconds), "--serve-rate", repr(args.serve_rate),
           "--serve-budget", str(args.serve_budget)]
    try:
        out = subprocess.run(cmd, capture_output=True, text=True, timeout=900, check=True).stdout
        return json.loads([ln for ln in out.splitlines() if ln.startswith("{")][-1])["capacity"]
    except Exception as e:  # reported, not fatal: the in-process numbers stand
        return {"error": "%s: %s" % (type(e).__name__, str(e)[:200])}


def run_served(args, pkg, synth, dev, rank, capacity_only=False):
    """The served workload: a Poisson stream of jobs through the request loop
    (bsort_submit / bsort_poll) and, for comparison, the same arrivals sorted
    one at a time.  Inputs come from pinned pools (each job sorts the first
    n keys of the pool of its key width and distribution); each job in
    flight owns one of a ring of pinned output buffers."""
    import numpy as np
    import torch

    rate, secs = args.serve_rate, args.serve_seconds
    cap = int(secs * rate * 1.5) + 16
    arr = synth.poisson_arrivals(cap, rate, synth.seed_for(5, 0, rank))
    njobs = int((arr < secs).sum())
    arr = arr[:njobs]
    sizes = synth.batch_sizes(njobs, synth.seed_for(5, 1, rank), lo_log2=10, hi_log2=24,
                              cap=1 << 62)
    bits = synth.draws64(synth.seed_for(5, 2, rank), njobs)
    wide = (bits & np.uint64(1)) != 0          # 64-bit keys
    zipf = (bits & np.uint64(2)) != 0          # Zipf(1.1) keys
    maxn = 1 << 24
    pools = {}
    for w in (False, True):
        for z in (False, True):
            seed = synth.seed_for(5, 3 + 2 * int(w) + int(z), rank)
            if w:
                a = synth.keys_zipf_u64(maxn, seed) if z else synth.keys_u64(maxn, seed)
                pools[(w, z)] = torch.from_numpy(a.view(np.int64)).pin_memory()
            else:
                a = synth.keys_zipf(maxn, seed) if z else synth.keys_u32("uniform", maxn, seed)
                pools[(w, z)] = torch.from_numpy(a.view(np.int32)).pin_memory()
    ring = 96
    slots = [torch.empty(maxn, dtype=torch.int64).pin_memory() for _ in range(ring)]
    kt_of = {False: pkg.BSORT_U32, True: pkg.BSORT_U64}

    def job(k, slot):
        w, z, n = bool(wide[k]), bool(zipf[k]), int(sizes[k])
        src = pools[(w, z)]
        dst = slots[slot] if w else slots[slot].view(torch.int32)
        return kt_of[w], src.data_ptr(), dst.data_ptr(), n, src, dst

    def check(k, slot):
        kt, _, _, n, src, dst = job(k, slot)
        if kt == pkg.BSORT_U64:
            flip = torch.tensor(-(1 << 63), dtype=torch.int64)
            want = torch.sort(src[:n] ^ flip).values ^ flip
        else:
            want = (torch.sort(src[:n].to(torch.int64) & 0xFFFFFFFF).values).to(torch.int32)
        return torch.equal(dst[:n], want)

    ncap = min(njobs, 4000)
    cap_keys = int(sizes[:ncap].sum())
    if capacity_only:
        return _serve_capacity(args, pkg, dev, job, ring, maxn, ncap, cap_keys)

    # served: arrivals submitted at their scheduled times, results polled
    srv = pkg.SortServer(device=dev.index, budget_bytes=args.serve_budget)
    # correctness gate, untimed: the first 48 jobs of the trace, 8 at a time,
    # each checked against torch.sort
    for g0 in range(0, min(njobs, 48), 8):
        tick = {}
        for k in range(g0, min(njobs, g0 + 8)):
            kt, a, b, n, _, _ = job(k, k - g0)
            tick[pkg.bsort_submit(srv.h, kt, a, b, n)] = k
        for t, k in tick.items():
            r = srv.wait(t)
            assert r.status == pkg.BSORT_OK and check(k, k - g0), "served job %d wrong" % k
    lat = np.zeros(njobs)
    done_at = np.zeros(njobs, np.int64)
    free, inflight = list(range(ring)), {}
    t0 = pkg.bsort_clock_ns() + 50_000_000
    nxt = done = 0
    while done < njobs:
        now = pkg.bsort_clock_ns()
        while nxt < njobs and t0 + int(arr[nxt] * 1e9) <= now and free:
            slot = free.pop()
            kt, a, b, n, _, _ = job(nxt, slot)
            inflight[pkg.bsort_submit(srv.h, kt, a, b, n)] = (nxt, slot)
            nxt += 1
        finished = pkg.bsort_poll_any(srv.h, 256)
        for t, r in finished:
            k, slot = inflight.pop(t)
            assert r.status == pkg.BSORT_OK, "served job failed"
            free.append(slot)
            lat[k] = (r.done_ns - (t0 + int(arr[k] * 1e9))) / 1e6
            done_at[k] = r.done_ns
            done += 1
        if not finished:
            time.sleep(2e-5)
    st = srv.stats()
    srv.close()
    span = (int(done_at.max()) - t0) / 1e9
    keys_total = int(sizes.sum())

    # one at a time: the same arrivals, each sorted and copied back before the next
    one = pkg.BucketSorter(device=dev.index)
    one._ensure(maxn, "u64", 0, extra=maxn * 8 + 512)
    lat1 = np.zeros(njobs)
    t1 = pkg.bsort_clock_ns() + 50_000_000
    last = t1
    strm = one._stream()
    for k in range(njobs):
        at = t1 + int(arr[k] * 1e9)
        while pkg.bsort_clock_ns() < at:
            pass
        kt, a, b, n, _, _ = job(k, 0)
        pkg.bsort_sort_keys_host(one.h, kt, a, b, n, strm)
        one.sync()
        last = pkg.bsort_clock_ns()
        lat1[k] = (last - at) / 1e6
    one.close()
    span1 = (last - t1) / 1e9

    # capacity: the first jobs of the trace back to back (closed loop), both
    # ways, in this process and in a fresh one
    import gc
    import torch
    gc.collect()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()  # device memory the earlier sections left cached
    capacity = _serve_capacity(args, pkg, dev, job, ring, maxn, ncap, cap_keys)
    capacity["fresh_process"] = _serve_capacity_subprocess(args) if rank == 0 else None
    # the same measurement once more in this process, after the fresh one
    again = _serve_capacity(args, pkg, dev, job, ring, maxn, ncap, cap_keys)
    capacity["again_in_process"] = {k: again[k] for k in ("served_gkeys_s",
                                                           "one_at_a_time_gkeys_s", "speedup")}
    # and with freshly pinned host buffers (same contents): the drop in this
    # process follows the pinned buffers the open-loop runs used
    try:
        kept = (pools, slots)
        pools = {key: val.clone().pin_memory() for key, val in kept[0].items()}
        slots = [torch.empty(maxn, dtype=torch.int64).pin_memory() for _ in range(ring)]
        nb = _serve_capacity(args, pkg, dev, job, ring, maxn, ncap, cap_keys)
        capacity["new_pinned_buffers_in_process"] = {
            k: nb[k] for k in ("served_gkeys_s", "one_at_a_time_gkeys_s", "speedup")}
        pools, slots = kept
    except Exception as e:  # reported, not fatal
        capacity["new_pinned_buffers_in_process"] = {"error": "%s: %s" % (type(e).__name__,
                                                                          str(e)[:200])}

    def pct(x, q):
        return float(np.percentile(x, q)) if len(x) else None

    # the tail by job kind: 64-bit keys or not, and size class (log2 n)
    by_kind = {}
    for w in (False, True):
        for lo, hi in ((10, 17), (17, 20), (20, 22), (22, 25)):
            sel = (wide == w) & (sizes >= (1 << lo)) & (sizes < (1 << hi))
            if sel.any():
                by_kind["%s_2^%d-2^%d" % ("u64" if w else "u32", lo, hi)] = {
                    "jobs": int(sel.sum()), "served_p99_ms": pct(lat[sel], 99),
                    "one_at_a_time_p99_ms": pct(lat1[sel], 99)}

    return {"workload": "Poisson arrivals %.0f/s for %.0f s, %d jobs, 50/50 uint32/uint64, "
                        "sizes log-uniform in [2^10, 2^24], 50/50 uniform/Zipf(1.1), pinned host "
                        "buffers, %d GB budget" % (rate, secs, njobs, args.serve_budget >> 30),
            "jobs": njobs, "keys": keys_total,
            "value": keys_total / span / 1e9, "unit": UNIT,
            "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99), "mean_ms": float(lat.mean()),
            "jobs_per_s": njobs / span, "batches": st["batches"],
            "mean_batch": njobs / max(st["batches"], 1), "max_batch": st["max_batch"],
            "arena_peak_bytes": st["arena_peak_bytes"],
            "one_at_a_time": {"value": keys_total / span1 / 1e9, "unit": UNIT,
                              "p50_ms": pct(lat1, 50), "p99_ms": pct(lat1, 99),
                              "mean_ms": float(lat1.mean()), "jobs_per_s": njobs / span1},
            "capacity": capacity, "p99_by_kind": by_kind,
            "latency": "sorted keys in host memory minus scheduled arrival"}


def run_capacity_only(args):
    import torch
    import paper_1002_4464_gb300 as pkg
    import synth
    _, _, local = _dist_env()
    torch.cuda.set_device(local)
    cap = run_served(args, pkg, synth, torch.device("cuda", local), 0, capacity_only=True)
    print(json.dumps({"capacity": cap}))
    return 0


def main():
    args = _args()
    if args.impl == "reference":
        return run_reference(args)
    if args.serve_capacity:
        return run_capacity_only(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
