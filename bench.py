"""Benchmark: concrete data-race-freedom checking of a memory access protocol
on the GPU, in access tuples checked per second.

Workload (the grid-scale configuration, the largest that one GPU runs as one
protocol): 65,536 threads, four arrays of 2^24 cells, eight phases (seven
top-level syncs between loop nests of depth <= 2 with trip counts 1..32),
affine indices (tid + 65536*g(x, y) + d) mod 2^24 for the owned writes plus
read-only accesses with tid coefficients in [-8, 8], about 2.2x10^8 access
tuples; seeded synthetic input (generator seed 0) with one planted race.  A
step is one complete check of that protocol -- every kernel of the back end
the plan runs, launched as one CUDA graph with the protocol's device program
already resident -- and ends with the verdict and witness in device memory.
L2 is flushed (a 256 MiB write) before every timed step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  `--impl reference` times the oracle (the plain CPU
checker used by the tests, method B driven on every host core) on the same
workload.
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
sys.path.insert(0, ROOT)

METRIC = "access tuples checked/sec"
UNIT = "tuples/s"
WORKLOAD = ("grid-scale seeded protocol (generator seed 0, one planted race): 65,536 threads, 4 arrays x 2^24 cells, "
            "8 phases, loop depth <= 2, trip counts 1..32, affine indices mod 2^24, ~2.2e8 access tuples")


def _measured():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return None


def _peaks():
    d = _measured()
    if d and "hbm_gbs" in d:
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons.  Started before the
    warm-up so that the sampler runs steadily when the timed region opens;
    mark() brackets the timed region and summary() keeps the samples inside
    it (plus the one just before and just after, so that a timed region
    shorter than the sampling period still has its clock)."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap,utilization.gpu")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []
        self.window = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def wait_first(self, timeout=5.0):
        t0 = time.perf_counter()
        while self.proc and not self.lines and time.perf_counter() - t0 < timeout:
            time.sleep(0.01)

    def mark(self):
        return len(self.lines)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, window=None):
        lines = self.lines
        if window is not None:
            lo, hi = window
            lines = lines[max(0, lo - 1):min(len(lines), hi + 1)]
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for n, v in zip(names, parts[2:6]):
                if v.lower() in ("active", "1"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


KERNEL_SOURCES = ("paper_2203_12878_b300/csrc/cuda/pipeline.cu", "paper_2203_12878_b300/csrc/cuda/pipeline.cuh",
                  "paper_2203_12878_b300/csrc/cuda/radix.cuh", "paper_2203_12878_b300/csrc/cuda/owner.cuh",
                  "paper_2203_12878_b300/csrc/cuda/intmath.cuh", "paper_2203_12878_b300/csrc/batch_args.h",
                  "paper_2203_12878_b300/csrc/devprog.h", "paper_2203_12878_b300/csrc/host/jit.cpp")


def _pipeline_hash():
    """Hash of what the measured kernels are built from: the device sources,
    the code generator (its compile options included) and the CUDA source it
    generates for the benchmark protocol (which also fingerprints the host's
    lowering of that protocol, the program the interpreter runs)."""
    from paper_2203_12878_b300 import drf
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    p = workload()
    st, src, _ = drf.drf_protocol_specialize(drf.drf_protocol_compile(p.text), p.nthreads, p.cells, p.params,
                                             compile=False)
    h.update((src or st).encode())
    return h.hexdigest()[:16]


TRAFFIC_FILE = "dram_traffic_grid_scale.txt"


def _profiled_traffic(kernel):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, or
    None when there is none or the kernels changed since it was taken."""
    path = os.path.join(ROOT, "profiles", TRAFFIC_FILE)
    try:
        vals = {}
        for line in open(path):
            if ":" in line:
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
        if vals.get("pipeline_hash") != _pipeline_hash():
            return None
        return float(vals[f"{kernel}_dram_bytes_per_launch"])
    except Exception:
        return None


def workload(seed=0, racy=True):
    from paper_2203_12878_b300 import protogen
    return protogen.config3(seed, racy=racy)


def thread_sample(p, threads):
    """The same protocol restricted to its first `threads` threads."""
    from paper_2203_12878_b300 import protogen
    return protogen.Protocol(p.text, threads, p.cells, p.params, p.meta)


def time_oracle(p, min_seconds, workers, max_runs=None):
    """Oracle method B (per-cell records) on `workers` host threads, run on
    protocol `p` until `min_seconds` have passed (at least once)."""
    from oracle import oracle
    oracle.build()
    runs, tuples, t0 = 0, 0, time.perf_counter()
    while True:
        r = oracle.check_mt(p.text, p.nthreads, p.cells, p.params, workers)
        tuples += r["tuples"]
        runs += 1
        el = time.perf_counter() - t0
        if el >= min_seconds or (max_runs and runs >= max_runs):
            return tuples / el, runs, el, r


def cpu_baselines(p, args):
    """The oracle on the machine's host cores: every core on the whole workload,
    and one core on a bounded thread-prefix sample of it."""
    from oracle import oracle
    cores = oracle.host_cores()
    v, runs, el, r = time_oracle(p, args.cpu_seconds, cores)
    one_threads = max(32, min(p.nthreads, args.cpu_one_core_threads))
    v1, runs1, el1, _ = time_oracle(thread_sample(p, one_threads), args.cpu_seconds / 2, 1)
    return ({"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
             "sample": f"the whole workload ({r['tuples']} tuples, all {p.nthreads} threads), method B (per-cell "
                       f"records) driven on {cores} host threads, {runs} runs in {el:.1f} s",
             "verdict": r.get("verdict")},
            {"value": v1, "unit": UNIT, "cores": 1, "kind": "oracle",
             "sample": f"the same protocol restricted to its first {one_threads} of {p.nthreads} threads, "
                       f"method B on one host thread, {runs1} runs in {el1:.1f} s"})


# ------------------------------------------------------------------ ours --

WARMUP_MIN_S = 1.5   # default: the GPU leaves its idle clocks only after some sustained work


def time_steps(plan, steps, warmup, stream, flush, clk_dev=None, stages=False, warm_s=None):
    """Times `steps` graph launches of `plan` on `stream` (L2 flushed before
    each, outside the events), after at least `warmup` untimed steps and at
    least WARMUP_MIN_S seconds of them.  Returns per-step ms, per-stage
    launch lists {kind: [(name, ms), ...]} (when `stages`: the plan's graph
    then holds an event node between its kernels), the clock summary of the
    timed region, the wall time and the warm-up actually done (steps, seconds)."""
    import torch
    from paper_2203_12878_b300 import drf

    def step(evs):
        with torch.cuda.stream(stream):
            flush.fill_(1)
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record(stream)
            drf.drf_plan_launch(plan, stream)
            e.record(stream)
        if evs is not None:
            evs.append((s, e))

    sampler = ClockSampler(clk_dev) if clk_dev is not None else None
    if sampler:
        sampler.__enter__()
    warm_s = WARMUP_MIN_S if warm_s is None else warm_s
    w0, done = time.perf_counter(), 0
    while done < warmup or time.perf_counter() - w0 < warm_s:
        for _ in range(8):
            step(None)
            done += 1
        stream.synchronize()
    if sampler:
        sampler.wait_first()
    warm_s = time.perf_counter() - w0
    torch.cuda.synchronize()
    evs, kinds = [], {}
    mark0 = sampler.mark() if sampler else 0
    t0 = time.perf_counter()
    for _ in range(steps):
        step(evs)
        if stages:
            stream.synchronize()
            for name, t in drf.drf_plan_stage_times(plan):
                kind = "radix" if name.startswith("radix") else name
                kinds.setdefault(kind, []).append((name, t))
    stream.synchronize()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clocks = None
    if sampler:
        if wall < 0.1:
            time.sleep(0.06)      # let the sample after the region arrive
        mark1 = sampler.mark()
        sampler.__exit__(None, None, None)
        clocks = sampler.summary((mark0, mark1))
    return [s.elapsed_time(e) for s, e in evs], kinds, clocks, wall, (done, warm_s)


# Algorithmic integer work of the owner-table pass per access tuple: index
# update, post-operation (mask / remainder), phase add, range test, record
# offset (two operations), record read, saturation test.
TABLE_OPS_PER_TUPLE = 8
INT32_LANES_PER_SM = 128   # sm_100-family SM: four partitions of 32 INT32 lanes


def alu_peak(dev, clocks):
    """INT32 operations per second of the device: its SM count (queried) x
    INT32 lanes per SM x the maximum SM clock (the driver's measurement, else
    the clock sampler's, else nvidia-smi's)."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz, src = None, None
    m = _measured()
    if m and m.get("sm_max_mhz"):
        mhz, src = float(m["sm_max_mhz"]), "MEASURED_PEAKS sm_max_mhz"
    elif clocks and clocks.get("sm_max_mhz"):
        mhz, src = float(clocks["sm_max_mhz"]), "nvidia-smi clocks.max.sm"
    if mhz is None:
        mhz, src = 2032.0, "nominal maximum SM clock"
    return sms * INT32_LANES_PER_SM * mhz * 1e6, f"{sms} SMs x {INT32_LANES_PER_SM} INT32 lanes x {mhz:.0f} MHz ({src})"


def roofline(kinds, steps, n, info, dev, clocks):
    """Roofline entry of the dominant kernel (largest device time per step)."""
    totals = {k: sum(t for _, t in v) / steps for k, v in kinds.items()}
    dominant = max(totals, key=totals.get)
    peak, peak_kind = _peaks()
    # algorithmic bytes per launch: radix pass = read + write every key (16 B);
    # emit = write every key (8 B); detect = read every key (8 B).  A forced
    # sort path emits one key per distinct (thread, offset) of the range
    # accesses, so it may sort fewer keys than there are tuples.
    nk = info.get("keys") or n
    bytes_per = {"radix": 16 * nk, "emit": 8 * nk, "detect": 8 * nk}
    radix_launches = [t for _, t in kinds.get("radix", []) if t > 0.002]
    dom_ms = (statistics.mean(radix_launches) if dominant == "radix" and radix_launches
              else totals[dominant] / max(1, len(kinds[dominant]) // steps))
    traffic = _profiled_traffic(dominant)
    if dominant in bytes_per:
        achieved = bytes_per[dominant] / (dom_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": f"k_{dominant}", "achieved": round(achieved, 1), "peak": peak,
                "unit": "GB/s", "frac": round(achieved / peak, 4), "peak_source": f"{peak_kind} (MEASURED_PEAKS hbm_gbs)",
                "traffic": traffic, "launch_ms": round(dom_ms, 4),
                "algorithmic_bytes_per_launch": bytes_per[dominant]}
        # the sort pipeline as a whole: algorithmic key bytes per tuple
        # (emit writes 8, each radix pass reads and writes 16, detection
        # reads 8) and each stage's share of HBM at its measured time
        npass = len(radix_launches) // steps if radix_launches else 0
        roof["keys_per_launch"] = nk
        roof["bytes_per_tuple"] = round((8 + 16 * npass + 8) * nk / n, 2)
        roof["stage_hbm_frac"] = {
            k: round(bytes_per[k] * (npass if k == "radix" else 1) / (totals[k] * 1e-3) / 1e9 / peak, 4)
            for k in bytes_per if totals.get(k)}
    elif dominant in ("table", "emit", "count", "witness", "range"):
        # the range pass applies its share of the tuples (counted on the
        # device); the table pass then applies the rest
        units = n
        if info.get("range_tuples") is not None:
            units = info["range_tuples"] if dominant == "range" else n - info["range_tuples"]
        ops = TABLE_OPS_PER_TUPLE * units
        achieved = ops / (dom_ms * 1e-3) / 1e12
        peak_ops, src = alu_peak(dev, clocks)
        kernel = ("k_range" if dominant == "range"
                  else f"drf_{dominant} (specialized)" if info.get("specialized") and dominant == "table"
                  else f"k_interp<{dominant}>")
        roof = {"bound": "alu", "kernel": kernel, "achieved": round(achieved, 3), "peak": round(peak_ops / 1e12, 2),
                "unit": "Tops/s", "frac": round(achieved * 1e12 / peak_ops, 4), "peak_source": f"derived: {src}",
                "traffic": traffic, "launch_ms": round(dom_ms, 4),
                "algorithmic_ops_per_launch": ops, "ops_per_tuple": TABLE_OPS_PER_TUPLE, "tuples_per_launch": units}
        if traffic:
            # the same kernel against HBM: its measured DRAM bytes per launch
            roof["dram_gbs"] = round(traffic / (dom_ms * 1e-3) / 1e9, 1)
            roof["dram_frac_of_hbm"] = round(traffic / (dom_ms * 1e-3) / 1e9 / peak, 4)
    else:
        roof = {"bound": "alu", "kernel": f"k_{dominant}", "achieved": None, "peak": None, "unit": None,
                "frac": None, "traffic": traffic, "launch_ms": round(dom_ms, 4)}
    return roof, {k: round(v, 4) for k, v in sorted(totals.items())}


def materialize_scan_fractions(tuples_per_s, sort_bits, peak_gbs):
    """The throughput as HBM fractions of a materialize-and-scan checker of
    the same protocol: one 8-byte key per tuple written, sorted by
    ceil(S / 8) LSD passes of 8-bit digits over its S sorted bits (16 B per
    key and pass) and read once by detection, i.e. 16 (1 + ceil(S / 8)) B per
    tuple (pipeline_frac), and the 16 B per tuple no such design moves less
    than (lower_bound_frac: one key written and read once).  Above 1 means the
    check ran faster than that design could at the measured copy bandwidth."""
    passes = -(-int(sort_bits) // 8) if sort_bits else 0
    per_tuple = 16 * (1 + passes)
    return {"sort_bits": sort_bits, "reference_passes": passes, "reference_bytes_per_tuple": per_tuple,
            "pipeline_frac": round(tuples_per_s * per_tuple / (peak_gbs * 1e9), 4),
            "lower_bound_frac": round(tuples_per_s * 16 / (peak_gbs * 1e9), 4), "peak_gbs": peak_gbs}


def run_ours(args, rank, world):
    import torch
    from paper_2203_12878_b300 import drf

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream()
    # each rank checks its own seeded protocol of the same shape
    p = workload(seed=rank)
    if args.threads:            # a smaller case of the same protocol (profiling captures)
        p = thread_sample(p, min(args.threads, p.nthreads))
    bc = drf.drf_protocol_compile(p.text)
    bounds = [(p.nthreads, p.cells, p.params)]
    flags = {"auto": drf.OPT_AUTOTUNE | drf.OPT_SPECIALIZE, "sort": drf.OPT_PATH_SORT,
             "table": drf.OPT_PATH_TABLE, "specialized": drf.OPT_PATH_TABLE | drf.OPT_SPECIALIZE}[args.path]
    ctx = drf.drf_ctx_create(dev, flags=flags)
    t_plan = time.perf_counter()
    plan = drf.drf_plan_create(ctx, [bc], bounds)
    plan_s = time.perf_counter() - t_plan
    info = drf.drf_plan_info(plan)
    path = drf.drf_plan_path(plan)
    specialized, _ = drf.drf_plan_specialized(plan)
    n = info["tuples"]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    drf.drf_plan_launch(plan, stream)
    torch.cuda.synchronize()
    res = drf.result_dict(drf.drf_plan_results(plan)[0])
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    step_ms, _, clocks, wall, warm = time_steps(plan, args.steps, args.warmup, stream, flush, clk_dev=dev,
                                                warm_s=args.warmup_seconds)
    if world > 1:
        dist.barrier()
    ms = statistics.mean(step_ms)
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    # per-stage times: the same configuration (the tuning cache returns the
    # timed plan's choice) recorded with an event node between its kernels;
    # those nodes cost time of their own, so the step above is timed without
    prof_steps = max(20, min(args.steps, 300))
    pctx = drf.drf_ctx_create(dev, flags=flags | drf.OPT_PROFILE_STAGES)
    pplan = drf.drf_plan_create(pctx, [bc], bounds)
    assert (drf.drf_plan_config(pplan), drf.drf_plan_path(pplan), drf.drf_plan_specialized(pplan)[0]) == \
        (drf.drf_plan_config(plan), path, specialized)
    pms, kinds, _, _, _ = time_steps(pplan, prof_steps, 3, stream, flush, stages=True, warm_s=args.warmup_seconds)
    assert drf.result_dict(drf.drf_plan_results(pplan)[0]) == res
    drf.drf_plan_destroy(pplan)
    drf.drf_ctx_destroy(pctx)
    range_tuples, range_updates = drf.drf_plan_range_tuples(plan)     # interpreted plans may run it too
    if not range_tuples:
        range_tuples, range_updates = None, None
    roof, stages = roofline(kinds, prof_steps, n, {**info, "specialized": specialized, "range_tuples": range_tuples,
                                                   "keys": drf.drf_plan_keys(plan)}, dev, clocks)

    # the interpreted back ends on the same protocol, for comparison
    others = []
    if rank == 0 and not args.quick and args.path == "auto":
        for oflags in (drf.OPT_PATH_SORT, drf.OPT_PATH_TABLE):
            try:
                osteps = max(20, min(args.steps // 5, 300))
                octx = drf.drf_ctx_create(dev, flags=oflags)
                oplan = drf.drf_plan_create(octx, [bc], bounds)
                oms, _, _, _, _ = time_steps(oplan, osteps, 3, stream, flush, warm_s=args.warmup_seconds)
                assert drf.result_dict(drf.drf_plan_results(oplan)[0]) == res
                drf.drf_plan_destroy(oplan)
                drf.drf_ctx_destroy(octx)
                octx = drf.drf_ctx_create(dev, flags=drf.OPT_PROFILE_STAGES | oflags)
                oplan = drf.drf_plan_create(octx, [bc], bounds)
                _, okinds, _, _, _ = time_steps(oplan, osteps, 3, stream, flush, stages=True, warm_s=args.warmup_seconds)
                ort = drf.drf_plan_range_tuples(oplan)[0] or None
                oroof, ostages = roofline(okinds, osteps, n, {**drf.drf_plan_info(oplan), "range_tuples": ort,
                                                              "keys": drf.drf_plan_keys(oplan)}, dev, clocks)
                ovalue = n / (statistics.mean(oms) * 1e-3)
                others.append({"path": drf.drf_plan_path(oplan), "specialized": False,
                               "ms_per_step": statistics.mean(oms), "value": ovalue,
                               "stages_ms": ostages, "roofline": oroof,
                               "materialize_scan_equivalent": materialize_scan_fractions(
                                   ovalue, info["sort_bits"], _peaks()[0])})
                drf.drf_plan_destroy(oplan)
                drf.drf_ctx_destroy(octx)
            except drf.DrfError as e:
                others.append({"flags": oflags, "unavailable": str(e)})

    # end to end through the public API: host bytecode in, host result out
    # (the context specializes: its first check of the protocol compiles the
    # kernels, untimed; the timed checks reuse them)
    drf.drf_check(ctx, bc, p.nthreads, p.cells, p.params, stream)
    e2e_t = []
    for i in range(max(5, min(args.steps, 50))):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        r = drf.drf_check(ctx, bc, p.nthreads, p.cells, p.params, stream)
        e2e_t.append(time.perf_counter() - t1)
        assert drf.result_dict(r) == res
    h2d, d2h = drf.drf_ctx_transfer_bytes(ctx)
    e2e_s = statistics.median(e2e_t)

    extra = {}
    if not args.quick and rank == 0:
        extra["race_free_variant"] = bench_one_protocol(stream, flush, workload(racy=False), "the same shape, "
                                                        "race-free variant (generator seed 0)")
        from paper_2203_12878_b300 import protogen
        extra["one_protocol_1024"] = bench_one_protocol(
            stream, flush, protogen.config2(0, "literal"),
            "one seeded protocol (generator seed 0): 1024 threads, 2 arrays x 2^20 cells, loop depth <= 3, trip counts "
            "1..64, affine indices mod 2^20 with coefficients in [-8,8], 1-6 syncs, rd/wr 50/50, ~1.2e7 tuples")
        extra["small_latency"] = bench_small_latency(stream)
        extra["batched"] = bench_batched(ctx, args)
        extra["served"] = [bench_served(args, rate=r, seconds=1.5) for r in args.rates]

    out = None
    if rank == 0:
        cpu, cpu1 = cpu_baselines(p, args)
        out = {
            "metric": METRIC, "value": world * n / (ms * 1e-3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": ("u32 owner records" if path == "table" else "u64 keys") + ", int32/int64 index arithmetic",
            "data": "synthetic",
            "config": {"workload": WORKLOAD if not args.threads else
                       f"{WORKLOAD}; restricted to its first {p.nthreads} threads",
                       "tuples_per_step": n, "path": path, "specialized": specialized,
                       "range_pass_tuples_per_step": range_tuples, "range_pass_record_updates_per_step": range_updates,
                       "path_choice": args.path,
                       "plan": {**drf.drf_plan_config(plan), "create_s": round(plan_s, 3)},
                       "sort_passes": info["sort_passes"], "sort_bits": info["sort_bits"],
                       "verdict": res.get("verdict"),
                       "l2": "flushed before every step (256 MiB write, outside the timed events); the owner "
                             "table alone (2.1 GB) is larger than L2",
                       "parallelism": f"replicas x{world}"},
            "roofline": roof,
            # the whole step (and the end-to-end call) against the HBM time a
            # materialize-and-scan checker needs for the same tuples
            "materialize_scan_equivalent": {
                "device": materialize_scan_fractions(world * n / (ms * 1e-3), info["sort_bits"], _peaks()[0]),
                "e2e": materialize_scan_fractions(n / e2e_s, info["sort_bits"], _peaks()[0])},
            "stages_ms": stages,
            "stages_note": (f"per-stage device times from {prof_steps} further steps of the same configuration "
                            f"with an event node between kernels (mean {statistics.mean(pms):.4f} ms per step "
                            f"with those nodes); value and ms_per_step come from the graph without them"),
            "alternatives": others,
            "cpu_baseline": cpu,
            "cpu_baseline_one_core": cpu1,
            "e2e": {"value": n / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": e2e_s * 1e3,
                    "path": "drf_check: host bytecode -> validate/lower -> H2D device program -> all kernels "
                            "(specialized kernels compiled by an earlier, untimed check) -> D2H result"},
            "gpu_launches": info["kernels_per_launch"] * args.steps,
            "clocks": clocks,
            "wall_s_timed_region": wall,
            "warmup_done": {"steps": warm[0], "seconds": round(warm[1], 3)},
        }
        out.update(extra)
    drf.drf_plan_destroy(plan)
    drf.drf_ctx_destroy(ctx)
    return out


def bench_small_latency(stream, calls=200):
    """The small workload (256 threads, one array of 2048 cells, 4096
    accesses: latency-bound): wall time of one drf_check (host bytecode in,
    result out) and of one plan launch with its results read back."""
    import torch
    from paper_2203_12878_b300 import drf, protogen
    out = {}
    ctx = drf.drf_ctx_create(0)
    try:
        for v in ("drf", "nosync"):
            p = protogen.config1(v)
            bc = drf.drf_protocol_compile(p.text)
            for _ in range(20):
                drf.drf_check(ctx, bc, p.nthreads, p.cells, p.params, stream)
            ts = []
            for _ in range(calls):
                t0 = time.perf_counter()
                r = drf.drf_check(ctx, bc, p.nthreads, p.cells, p.params, stream)
                ts.append(time.perf_counter() - t0)
            plan = drf.drf_plan_create(ctx, [bc], [(p.nthreads, p.cells, p.params)])
            tp = []
            for i in range(calls + 20):
                t0 = time.perf_counter()
                drf.drf_plan_launch(plan, stream)
                drf.drf_plan_results(plan)
                if i >= 20:
                    tp.append(time.perf_counter() - t0)
            drf.drf_plan_destroy(plan)
            ts.sort(); tp.sort()
            out[v] = {"verdict": drf.result_dict(r)["verdict"], "tuples": p.meta.get("accesses", 4096),
                      "drf_check_us_p50": round(ts[len(ts) // 2] * 1e6, 1), "drf_check_us_p99": round(ts[int(len(ts) * 0.99)] * 1e6, 1),
                      "plan_launch_us_p50": round(tp[len(tp) // 2] * 1e6, 1), "plan_launch_us_p99": round(tp[int(len(tp) * 0.99)] * 1e6, 1)}
    finally:
        drf.drf_ctx_destroy(ctx)
    return out


def bench_one_protocol(stream, flush, p, what):
    """One protocol as an autotuned plan (specialized kernels allowed):
    device time per check, L2 flushed before each; the result is checked
    against what the generator planted (or its absence)."""
    from paper_2203_12878_b300 import drf
    bc = drf.drf_protocol_compile(p.text)
    ctx = drf.drf_ctx_create(0, flags=drf.OPT_AUTOTUNE | drf.OPT_SPECIALIZE)
    try:
        plan = drf.drf_plan_create(ctx, [bc], [(p.nthreads, p.cells, p.params)])
        n = drf.drf_plan_info(plan)["tuples"]
        ms, _, _, _, _ = time_steps(plan, 50, 3, stream, flush, warm_s=0.5)
        r = drf.result_dict(drf.drf_plan_results(plan)[0])
        if p.meta.get("planted"):
            assert (r["verdict"], r["phase"], r["loc"], r["index"]) == ("RACY", p.meta["phase"], p.meta["loc"],
                                                                       p.meta["index"])
        elif p.meta.get("race_free_by_construction"):
            assert r["verdict"] == "DRF"
        out = {"workload": what, "tuples": n, "path": drf.drf_plan_path(plan),
               "specialized": drf.drf_plan_specialized(plan)[0], "verdict": r["verdict"],
               "ms_per_check": statistics.mean(ms), "tuples_per_s": n / (statistics.mean(ms) * 1e-3)}
        drf.drf_plan_destroy(plan)
        return out
    finally:
        drf.drf_ctx_destroy(ctx)


def bench_batched(ctx, args):
    """Protocols per second on the batched workload: 4096 seeded protocols in
    one pipeline pass (protocol id in the key's top bits), as a CUDA graph."""
    import torch
    from paper_2203_12878_b300 import drf, protogen
    ps = protogen.config4(master_seed=1, count=4096)
    bcs = [drf.drf_protocol_compile(p.text) for p in ps]
    tctx = drf.drf_ctx_create(0, flags=drf.OPT_AUTOTUNE)
    t0 = time.perf_counter()
    plan = drf.drf_plan_create(tctx, bcs, [(p.nthreads, p.cells, p.params) for p in ps])
    tune_s = time.perf_counter() - t0
    info = drf.drf_plan_info(plan)
    cfg = drf.drf_plan_config(plan)
    stream = torch.cuda.Stream()
    for _ in range(3):
        drf.drf_plan_launch(plan, stream)
    stream.synchronize()
    reps = 10
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record(stream)
    for _ in range(reps):
        drf.drf_plan_launch(plan, stream)
    e.record(stream)
    e.synchronize()
    ms = s.elapsed_time(e) / reps
    res = drf.drf_plan_results(plan)
    racy = sum(1 for r in res if r.verdict == 1)
    drf.drf_plan_destroy(plan)
    drf.drf_ctx_destroy(tctx)
    # the plain path: one protocol per launch (drf_check on a default
    # context), same protocols (a sample)
    sample = list(zip(bcs, ps))[:256]
    pctx = drf.drf_ctx_create(0)
    drf.drf_check(pctx, sample[0][0], sample[0][1].nthreads, sample[0][1].cells, sample[0][1].params, stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for bc, p in sample:
        drf.drf_check(pctx, bc, p.nthreads, p.cells, p.params, stream)
    plain_s = (time.perf_counter() - t0) / len(sample)
    drf.drf_ctx_destroy(pctx)
    return {"protocols": len(ps), "tuples": info["tuples"], "sort_passes": info["sort_passes"],
            "ms_per_batch": ms, "protocols_per_s": len(ps) / (ms * 1e-3), "tuples_per_s": info["tuples"] / (ms * 1e-3),
            "racy": racy, "plain_protocols_per_s": 1.0 / plain_s, "autotuned": cfg, "tuning_s": tune_s,
            "path": "one plan (CUDA graph) over all 4096 protocols; plain = drf_check per protocol"}


SERVER_POLL_US = 2000


def bench_served(args, rate=5000.0, seconds=2.0, warm_seconds=0.5):
    """Continuous-batching server under a Poisson stream: 90% batched-family
    protocols, 10% one-protocol-family (scaled to 3x10^5 accesses).  The
    first `warm_seconds` of the stream bring the server's device buffers to
    their working sizes and are not counted; latency percentiles and
    throughput cover the requests submitted after them."""
    import random
    from paper_2203_12878_b300 import drf, protogen
    arr = protogen.config5_arrivals(rate, warm_seconds + seconds)
    r = random.Random(9)
    pool_b = [drf.drf_protocol_compile(p.text) for p in protogen.config4(master_seed=5, count=512)]
    pool_b_meta = protogen.config4(master_seed=5, count=512)
    singles = [protogen.config2(s, target=3e5) for s in range(4)]
    pool_s = [(drf.drf_protocol_compile(p.text), p) for p in singles]
    ctx = drf.drf_ctx_create(0)
    # idle workers poll the queue for 2 ms before sleeping (low-latency mode)
    drf.drf_server_start(ctx, poll_us=SERVER_POLL_US)
    tickets = []
    t0 = time.perf_counter()
    for t, fam in arr:
        while time.perf_counter() - t0 < t:
            pass
        if fam == "batch":
            i = r.randrange(len(pool_b))
            p = pool_b_meta[i]
            tk = drf.drf_server_submit(ctx, pool_b[i], p.nthreads, p.cells, p.params)
        else:
            bc, p = pool_s[r.randrange(len(pool_s))]
            tk = drf.drf_server_submit(ctx, bc, p.nthreads, p.cells, p.params)
        tickets.append((t >= warm_seconds, tk))
    lat = []
    t_end = time.perf_counter()
    for counted, tk in tickets:
        got = drf.drf_server_poll(ctx, tk, 120_000_000)
        if counted:
            lat.append(got[1] / 1e6)
    wall = max(time.perf_counter(), t_end) - t0 - warm_seconds
    stats = drf.drf_server_stats(ctx)
    drf.drf_server_stop(ctx)
    drf.drf_ctx_destroy(ctx)
    lat.sort()
    return {"rate_req_s": rate, "requests": len(lat), "warmup_s": warm_seconds, "p50_ms": lat[len(lat) // 2],
            "p99_ms": lat[min(len(lat) - 1, int(len(lat) * 0.99))], "throughput_req_s": len(lat) / wall,
            "rounds": stats["rounds"], "max_round": stats["max_round"], "worker_poll_us": SERVER_POLL_US}


# ------------------------------------------------------------- reference --

REFERENCE_BUDGET_S = 240.0   # the whole reference run (warm-up and timed steps) stays within about this


def run_reference(args):
    """The oracle (method B on every host core) as the reference arm, on the
    benchmark's workload: each step one complete check of the whole
    protocol.  When (warm-up + timed steps) of the whole protocol would not
    fit REFERENCE_BUDGET_S, each step checks the protocol restricted to a
    thread prefix sized to fit (said in config.sample)."""
    from oracle import oracle
    oracle.build()
    cores = oracle.host_cores()
    full = workload()
    p = full
    t0 = time.perf_counter()
    r = oracle.check_mt(p.text, p.nthreads, p.cells, p.params, cores)    # first warm-up step, and a size probe
    one = time.perf_counter() - t0
    total_steps = args.steps + args.warmup
    if one * total_steps > REFERENCE_BUDGET_S:
        threads = max(32, int(full.nthreads * REFERENCE_BUDGET_S / (one * total_steps)) // 32 * 32)
        p = thread_sample(full, min(threads, full.nthreads))
    for _ in range(args.warmup - 1):
        oracle.check_mt(p.text, p.nthreads, p.cells, p.params, cores)
    times, n = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = oracle.check_mt(p.text, p.nthreads, p.cells, p.params, cores)
        times.append(time.perf_counter() - t0)
        n = r["tuples"]
    ms = statistics.mean(times) * 1e3
    v = n / (ms * 1e-3)
    sample = ("the whole workload" if p is full else f"the workload restricted to its first {p.nthreads} of "
              f"{full.nthreads} threads (the whole protocol would not fit the run's time budget)")
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample, "tuples_per_step": n, "verdict": r.get("verdict")},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{sample}; method B (per-cell records) on {cores} host threads"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--quick", action="store_true", help="skip the batched and served measurements")
    ap.add_argument("--sources-hash", action="store_true",
                    help="print the hash of the kernel sources (the key of the committed DRAM traffic summary) and exit")
    ap.add_argument("--path", choices=("auto", "sort", "table", "specialized"), default="auto",
                    help="back end of the timed plan: autotuned (specialized kernels allowed), or forced")
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="least wall time of the oracle's all-core timing (the one-core sample gets half)")
    ap.add_argument("--threads", type=int, default=0,
                    help="check the workload restricted to its first THREADS threads (a smaller case for "
                         "profiling captures; the JSON line's config says so); 0 = all 65,536")
    ap.add_argument("--cpu-one-core-threads", type=int, default=4096,
                    help="threads of the thread-prefix sample timed on one host core")
    ap.add_argument("--warmup-seconds", type=float, default=WARMUP_MIN_S,
                    help="least wall time of untimed steps before each timed region (besides --warmup steps)")
    ap.add_argument("--rates", type=float, nargs="*", default=[1000, 5000, 20000, 50000],
                    help="served-workload arrival rates (requests/s)")
    args = ap.parse_args()
    if args.sources_hash:
        print(_pipeline_hash())
        return
    args.warmup = max(3, args.warmup)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    out = run_ours(args, rank, world)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
