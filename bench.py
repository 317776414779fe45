"""Benchmark: GP operations per second (tree nodes x fitness cases / s) of one
generation step on a GB300, through libgp's C ABI.

Workload (one step): the resident population of 4000 seeded random trees
(odd sizes log-uniform on [31, 32767], 48 Sextic fitness cases, 127 seeded
constants) produces 4000 children by subtree crossover at uniformly chosen
points (Sec. 3.1), and every child is evaluated (Sec. 2.2) and reduced to its
mean absolute error (Table gp.details).  `value` = child nodes x 48 / step
time, inputs resident in HBM; `e2e` repeats the step from pinned host buffers
through the public API, copies included.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).
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
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1902_09215_gb300 import synth  # noqa: E402

N_TREES = 4000
SEED_POP, SEED_XO, CONST_SEED = 3, 11, 2
WORKLOAD = ("4000 seeded random prefix trees, odd sizes log-uniform 31..32767 nodes, "
            "48 Sextic cases, 127 constants; step = 4000 subtree crossovers + fitness "
            "evaluation of the 4000 children")
METRIC = "GPops/s (tree nodes x fitness cases per second), generation step"
L2_FLUSH_BYTES = 256 << 20


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest of every rank's x (the slowest rank sets the job's time)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(units_per_rank: float, world: int, max_ms: float) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return units_per_rank * world / (max_ms / 1e3)


def nearest_rank(values, q: float) -> float:
    """The q-quantile by the nearest-rank rule: the ceil(q n)-th smallest."""
    srt = sorted(values)
    return srt[max(0, min(len(srt) - 1, math.ceil(q * len(srt)) - 1))]


def make_workload(rank: int):
    x, y, c = synth.problem(const_seed=CONST_SEED)
    nodes, offs = synth.population_loguniform(seed=SEED_POP + 1000 * rank, count=N_TREES)
    sizes = np.diff(offs.astype(np.int64))
    ops = synth.crossover_points(SEED_XO + 1000 * rank, sizes, N_TREES)
    return x, y, c, nodes, offs, ops


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [v.strip() for v in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_source_sha():
    """Hash of what the level-0 launch of the step depends on: gp_eval.cu,
    gp_plan0.cu (which chunks the launch gets) and the types, constants and
    device helpers of gp_internal.cuh (launcher declarations after them do
    not change the kernels)."""
    csrc = os.path.join(ROOT, "paper_1902_09215_gb300", "csrc")
    h = hashlib.sha256()
    h.update(open(os.path.join(csrc, "gp_eval.cu"), "rb").read())
    h.update(open(os.path.join(csrc, "gp_plan0.cu"), "rb").read())
    hdr = open(os.path.join(csrc, "gp_internal.cuh"), "rb").read()
    cut = hdr.find(b"// Launchers")
    h.update(hdr if cut < 0 else hdr[:cut])
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def recorded_counters():
    """The level-0 evaluator's ncu record (DRAM bytes and warp instructions
    per launch), only if it was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "eval_kernel_traffic.json")
    if not os.path.exists(p):
        return {}
    d = json.load(open(p))
    if d.get("kernel_source_sha") != kernel_source_sha():
        return {}
    return d


def recorded_traffic():
    return recorded_counters().get("dram_bytes_per_launch")


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_ours(args):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    from paper_1902_09215_gb300 import gp
    gp.lib()

    x, y, c, nodes, offs, ops = make_workload(rank)
    stream = torch.cuda.Stream(dev)
    prob = gp.Problem(x, y, c)
    xo = gp.make_xo(*ops)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    with torch.cuda.stream(stream):
        parents = gp.gp_create_population(prob, nodes, offs, stream)

    redo_in_step = [False]

    def step():
        kids = gp.gp_crossover(parents, xo, stream)
        gp.gp_evaluate(kids, stream)
        if redo_in_step[0]:              # trees deferred to gp_fitness are part of the step
            gp.gp_fitness(kids)
        return kids

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # Clocks are sampled from before the warm-up to the end of the timed
    # steps, so the sampler's start-up pause does not leave the GPU idle
    # (its clocks falling) right before the first timed step.
    clk = ClockSampler(local).__enter__()
    try:
        # warm-up (also sizes the child population); as many populations
        # alive at once as in the timed loop, so the memory pool is at its
        # working size before timing starts
        keep = []
        for _ in range(args.warmup):         # the timed loop's pattern: no wait between steps
            with torch.cuda.stream(stream):
                flush.zero_()
                keep.append(step())
            if len(keep) > 1:
                keep.pop(0)
        barrier()
        gp.gp_fitness(keep[-1])
        child_nodes = int(gp.gp_population_get_info(keep[-1]).total_nodes)
        stats = gp.gp_eval_stats_get(keep[-1])
        # gp_evaluate leaves trees whose chunk fragments overflowed their
        # slots to gp_fitness; the children are the same every step, so if
        # any were deferred the timed step waits for gp_fitness too
        redo_in_step[0] = stats["redone"] > 0
        keep.clear()

        # ---- timed: K steps, L2 flushed before each, device time per step
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        keep = []
        host_ms = []
        barrier()
        launches0 = gp.gp_kernel_launch_count()
        t0 = time.perf_counter()
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
                ev[k][0].record(stream)
                h = time.perf_counter()
                keep.append(step())
                host_ms.append(1e3 * (time.perf_counter() - h))
                ev[k][1].record(stream)
            if len(keep) > 1:                # freed in stream order after its step
                keep.pop(0)
        barrier()
        wall = time.perf_counter() - t0
    finally:
        clk.__exit__(None, None, None)
    launches = gp.gp_kernel_launch_count() - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    keep.clear()
    total_ms = max_over_ranks(float(sum(step_ms)), world, dev)
    value = weak_scaling_value(child_nodes * prob.n_cases * args.steps, world, total_ms)

    # ---- evaluation alone and crossover alone (device time), same flushing
    def timed(fn, reps):
        out = []
        for _ in range(reps):
            with torch.cuda.stream(stream):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn()
                b.record(stream)
            out.append((a, b))
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in out]

    kids = step()
    gp.gp_fitness(kids)
    eval_ms = timed(lambda: gp.gp_evaluate(kids, stream), max(10, args.steps // 4))
    xo_ms = timed(lambda: gp.gp_crossover(parents, xo, stream), max(10, args.steps // 4))
    child_bytes = child_nodes

    # ---- roofline of the dominant kernel: CUDA events around each launch
    gp.gp_profile_read(reset=True)
    gp.gp_profile_enable(True)
    for _ in range(max(10, args.steps // 4)):
        with torch.cuda.stream(stream):
            flush.zero_()
            k2 = step()
    torch.cuda.synchronize()
    gp.gp_profile_enable(False)
    prof = gp.gp_profile_read(reset=True)
    del k2
    ev0 = prof["eval"]
    eval_launch_ms = ev0["ms"] / max(ev0["launches"], 1)
    # algorithmic work of one evaluation: (n-1)/2 binary FP32 operations per
    # tree per case; the level-0 launch does all but the spine operators it
    # sends up to the ropes (gp_eval_stats: upper_ops), which the rope
    # launch does
    upper_ops = int(stats["upper_ops"])
    n_bin_ops = ((child_nodes - N_TREES) // 2 - upper_ops) * prob.n_cases
    up = prof.get("eval_upper", {"ms": 0.0, "launches": 0})
    rope_launch_ms = up["ms"] / up["launches"] if up["launches"] else None
    peaks, peak_src = measured_peaks()
    clocks = clk.summary()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak = n_sm * 128 * sm_mhz * 1e6 / 1e12           # FP32 lanes x clock, Tops/s
    achieved = n_bin_ops / (eval_launch_ms / 1e3) / 1e12
    traffic = recorded_traffic()
    # the interpreter's own bound: warp instructions issued (ncu count of the
    # same launch) against 4 schedulers x SMs x clock
    inst = recorded_counters().get("warp_instructions")
    issue = None
    if inst:
        ipeak = 4.0 * n_sm * sm_mhz * 1e6
        issue = {"warp_instructions_per_launch": inst, "achieved_per_s": inst / (eval_launch_ms / 1e3),
                 "peak_per_s": ipeak, "frac": inst / (eval_launch_ms / 1e3) / ipeak,
                 "note": "4 warp schedulers x SMs x max clock; the bound the interpreter meets"}
    tot_ms = sum(v["ms"] for v in prof.values() if v["launches"])

    # ---- end to end through the public API from pinned host memory
    pin_nodes = torch.from_numpy(nodes).pin_memory()
    pin_offs = torch.from_numpy(offs.astype(np.uint64).view(np.int64)).pin_memory()
    nodes_h = pin_nodes.numpy()
    offs_h = pin_offs.numpy().view(np.uint64)
    e2e_steps = max(5, args.steps // 10)
    barrier()
    te = []
    for _ in range(e2e_steps):
        flush.zero_()
        torch.cuda.synchronize()
        a = time.perf_counter()
        p2 = gp.gp_create_population(prob, nodes_h, offs_h, stream)
        k3 = gp.gp_crossover(p2, ops, stream)        # records marshalled as a caller's arrays
        gp.gp_evaluate(k3, stream)
        fit, _, _ = gp.gp_fitness(k3)
        te.append(time.perf_counter() - a)
        del p2, k3
    e2e_s = float(np.median(te))
    e2e_value = child_nodes * prob.n_cases * world / e2e_s
    h2d = int(nodes.nbytes + offs.nbytes + 4 * (x.size + y.size + c.size) + 24 * N_TREES)
    d2h = int(4 * N_TREES)

    if world > 1:
        dist.barrier()
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    cpu = cpu_baseline(nodes, offs, ops, x, y, c, child_nodes) if world == 1 and not args.no_cpu else None
    batched = generations_compare(gp, prob, nodes, offs, stream, flush, 10, 5) if world == 1 else None
    configs = None
    if world == 1 and not args.no_extra:
        # the benchmark's other configurations, each measured once here
        def guarded(fn, *a):
            # a configuration that fails is reported in the line, not fatal to it
            try:
                return fn(*a)
            except Exception as e:            # noqa: BLE001
                return {"error": f"{type(e).__name__}: {e}"}
        configs = {"smallest_50_trees": guarded(config1_latency, gp, prob, stream, 300, not args.no_cpu),
                   "bloated_48_trees": guarded(config3_bloated, gp, prob, stream, not args.no_cpu),
                   "crossover_large_children": guarded(crossover_large, gp, prob, stream, flush),
                   "batched_4000_parents_1e2_1e8": guarded(config4_batched, gp, prob, stream, flush,
                                                           not args.no_cpu),
                   "serving_64_runs": guarded(config5_serving, gp, prob, stream)}
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "GPops/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {
            "workload": WORKLOAD,
            "trees": N_TREES, "child_nodes_per_step": child_nodes, "cases": int(prob.n_cases),
            "seeds": {"population": SEED_POP, "crossover": SEED_XO, "constants": CONST_SEED},
            "l2": f"flushed before every timed step ({L2_FLUSH_BYTES >> 20} MB write, outside the events)",
            "parallelism": f"replicas x{world} (independent populations)",
            "eval_levels": stats["levels"], "eval_items": stats["items"],
        },
        "latency_ms": {"p50": nearest_rank(step_ms, 0.5), "p99": nearest_rank(step_ms, 0.99),
                       "rule": f"nearest rank over {len(step_ms)} timed steps",
                       "max": max(step_ms), "slowest_step": int(step_ms.index(max(step_ms))),
                       "first_step": step_ms[0],
                       "host_enqueue_ms": {"p50": nearest_rank(host_ms, 0.5), "max": max(host_ms),
                                           "slowest_step": int(host_ms.index(max(host_ms)))}},
        "redone_trees": int(stats["redone"]),
        "eval_only": {"value": child_nodes * prob.n_cases / (statistics.median(eval_ms) / 1e3),
                      "unit": "GPops/s", "ms_p50": statistics.median(eval_ms)},
        "crossover": {"ms_p50": statistics.median(xo_ms),
                      "GB_per_s": 2 * child_bytes / (statistics.median(xo_ms) / 1e3) / 1e9},
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": "GPops/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "wall_s_p50": e2e_s},
        "gpu_launches": int(launches),
        "roofline": {"bound": "alu", "kernel": "eval_kernel (level 0)",
                     "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                     "frac": achieved / alu_peak, "traffic": traffic,
                     "peak_note": f"{n_sm} SMs x 128 FP32 lanes x {sm_mhz:.0f} MHz ({peak_src} max clock); "
                                  "achieved = the binary ops x 48 cases level 0 performs ((n-1)/2 per tree "
                                  "less the spine operators it sends to the ropes) / mean launch time",
                     "launch_ms": eval_launch_ms, "launches_profiled": ev0["launches"], "issue": issue,
                     "rope_launch": None if rope_launch_ms is None else {
                         "kernel": "eval_kernel (ropes)", "ops": upper_ops * prob.n_cases,
                         "launch_ms": rope_launch_ms,
                         "achieved": upper_ops * prob.n_cases / (rope_launch_ms / 1e3) / 1e12,
                         "frac": upper_ops * prob.n_cases / (rope_launch_ms / 1e3) / 1e12 / alu_peak},
                     "kernel_ms_per_launch": {k: v["ms"] / v["launches"] for k, v in prof.items() if v["launches"]},
                     "kernel_share": {k: v["ms"] / tot_ms for k, v in prof.items() if v["launches"]}},
        "wall_s": wall,
    }
    if cpu:
        line["cpu_baseline"] = cpu
    if batched:
        line["batched_vs_plain"] = batched
    if configs:
        line["configs"] = configs
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def generations_compare(gp, prob, nodes, offs, stream, flush, K, reps, chunk=0, arena=0, shape=None):
    """K consecutive generations from the same parents, made two ways, with
    identical results (checked): on the device (one gp_generation_step of K
    generations: tournaments, crossover and evaluation replayed from the
    captured graph, the host never waiting) and through the plain API as a
    host-driven GP loop must run it (per generation: gp_crossover on that
    generation's records, gp_evaluate, and gp_fitness, the read-back the
    host needs before it can choose the next parents; the records are
    given, so the host's own selection costs nothing here).  Wall clock
    around each block of K generations, L2 flushed before it.  Also the
    plain path replaying one generation's records without any read-back
    (device time), a bound no host-driven loop reaches."""
    import torch
    kw = dict(seed=SEED_GEN, use_graph=True, stream=stream)
    if arena:
        kw["arena_bytes"] = arena
    if shape:
        kw.update(warps_per_cta=shape[0], window_entries=shape[1], upper_window_entries=shape[2])
    G = gp.gp_generation_create(prob, nodes, offs, chunk_nodes=chunk, **kw)
    info0 = gp.gp_generation_get_info(G)
    chunk = int(info0["chunk_nodes"])
    # later creations take the chosen chunk and launch shapes (no autotuning)
    kw.update(warps_per_cta=info0["warps_per_cta"], window_entries=info0["window_entries"],
              upper_window_entries=info0["upper_window_entries"])
    # the records of each generation (untimed pass, one generation at a time)
    recs = []
    for _ in range(K):
        gp.gp_generation_step(G, 1, stream)
        recs.append(gp.make_xo(*gp.gp_generation_records(G)))
    want_nodes, want_offs = gp.gp_generation_trees(G)
    want_fit, _, _ = gp.gp_generation_fitness(G)
    child_nodes = []
    gp.gp_generation_destroy(G)
    del G

    def one_batched():
        G2 = gp.gp_generation_create(prob, nodes, offs, chunk_nodes=chunk, **kw)
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            flush.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        gp.gp_generation_step(G2, K, stream)
        torch.cuda.synchronize()
        el = time.perf_counter() - t
        return G2, el

    b_s = []
    for r in range(reps):
        G2, el = one_batched()
        b_s.append(el)
        if r == reps - 1:
            got_nodes, got_offs = gp.gp_generation_trees(G2)
            same_batched = bool(np.array_equal(got_nodes, want_nodes) and np.array_equal(got_offs, want_offs))
        gp.gp_generation_destroy(G2)
        del G2
    with torch.cuda.stream(stream):
        first = gp.gp_create_population(prob, nodes, offs, stream)
    gp.gp_evaluate(first, stream, chunk_nodes=chunk)
    gp.gp_fitness(first)
    p_s = []
    for r in range(reps):
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            flush.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        pop = first
        for g in range(K):
            kids = gp.gp_crossover(pop, recs[g], stream)
            gp.gp_evaluate(kids, stream, chunk_nodes=chunk)
            fit, _, _ = gp.gp_fitness(kids)           # the host loop's read-back
            if r == 0:
                child_nodes.append(int(gp.gp_population_get_info(kids).total_nodes))
            pop = kids
        el = time.perf_counter() - t
        p_s.append(el)
    plain_nodes, plain_offs = gp.read_all_trees(pop)
    same_plain = bool(np.array_equal(plain_nodes, want_nodes) and np.array_equal(plain_offs, want_offs)
                      and np.array_equal(np.asarray(fit).view(np.uint32), np.asarray(want_fit).view(np.uint32)))
    del pop, kids
    # one generation's records replayed with no read-back (device time)
    xo = recs[0]

    def replay():
        k = gp.gp_crossover(first, xo, stream)
        gp.gp_evaluate(k, stream, chunk_nodes=chunk)
        return k
    ms = []
    for k in range(max(3, reps) + 2):
        with torch.cuda.stream(stream):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            kk = replay()
            b.record(stream)
        b.synchronize()
        gp.gp_fitness(kk)
        if k >= 2:
            ms.append(a.elapsed_time(b))
        del kk
    del first
    torch.cuda.synchronize()
    units = sum(child_nodes) * prob.n_cases
    bs, ps = statistics.median(b_s), statistics.median(p_s)
    return {"generations": K, "blocks": reps, "chunk_nodes": chunk, "child_nodes": sum(child_nodes),
            "launch_shape": {"level0": [info0["warps_per_cta"], info0["window_entries"]],
                             "upper": [info0["upper_warps"], info0["upper_window_entries"]]},
            "identical_results": same_batched and same_plain,
            "batched_graph": {"ms_per_generation": 1e3 * bs / K, "GPops_per_s": units / bs},
            "plain_host_loop": {"ms_per_generation": 1e3 * ps / K, "GPops_per_s": units / ps},
            "speedup": ps / bs,
            "plain_records_replayed_no_readback": {
                "ms_per_generation": statistics.median(ms),
                "GPops_per_s": child_nodes[0] * prob.n_cases / (statistics.median(ms) / 1e3),
                "note": "one generation's records replayed, host never waiting (device time)"}}


def cpu_baseline(nodes, offs, ops, x, y, c, child_nodes):
    """The oracle as it stands, on this host's cores: children of a bounded
    sample of the crossover records, evaluated by the oracle's dynamic
    work queue over all cores, repeated for about 10 s."""
    from oracle import oracle
    cores = os.cpu_count() or 1
    sample = 1000
    mum, dad, mp, dp = (a[:sample] for a in ops)
    t0 = time.perf_counter()
    done_nodes, reps = 0, 0
    while True:
        rn, ro = oracle.crossover_population(nodes, offs, mum, dad, mp, dp)
        oracle.eval_population(rn, ro, x, y, c, n_threads=cores)
        done_nodes += int(ro[-1])
        reps += 1
        if time.perf_counter() - t0 > 10.0:
            break
    el = time.perf_counter() - t0
    # the same oracle on one thread, on a smaller sample (about 3 s)
    one = 100
    rn, ro = oracle.crossover_population(nodes, offs, *(a[:one] for a in ops))
    t1 = time.perf_counter()
    one_nodes, one_reps = 0, 0
    while True:
        oracle.eval_population(rn, ro, x, y, c, n_threads=1)
        one_nodes += int(ro[-1])
        one_reps += 1
        if time.perf_counter() - t1 > 3.0:
            break
    el1 = time.perf_counter() - t1
    return {"value": done_nodes * len(x) / el, "unit": "GPops/s", "cores": cores, "kind": "oracle",
            "sample": f"{reps} x (crossover of the first {sample} of the 4000 records + oracle "
                      f"evaluation of those children on {cores} threads), {el:.1f} s",
            "single_core": {"value": one_nodes * len(x) / el1, "unit": "GPops/s", "cores": 1,
                            "sample": f"{one_reps} x oracle evaluation of the children of the first "
                                      f"{one} records on 1 thread, {el1:.1f} s"}}


def config1_latency(gp, prob, stream, reps, cpu):
    """The smallest workload (50 trees of 1..63 nodes): it is launch-bound,
    so what counts is the time of one evaluation call, on the device (CUDA
    events around gp_evaluate) and through the API (gp_evaluate plus the
    gp_fitness that waits for it and copies the 50 fitness values back)."""
    import torch
    nodes, offs = synth.population_small(seed=1)
    x, y, c = prob.x, prob.y, prob.consts
    pop = gp.gp_create_population(prob, nodes, offs, stream)
    for _ in range(20):
        gp.gp_evaluate(pop, stream)
        gp.gp_fitness(pop)
    dev, wall = [], []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t = time.perf_counter()
        a.record(stream)
        gp.gp_evaluate(pop, stream)
        b.record(stream)
        gp.gp_fitness(pop)
        wall.append(1e6 * (time.perf_counter() - t))
        dev.append(1e3 * a.elapsed_time(b))
    gp.gp_destroy_population(pop)
    n = int(offs[-1])
    out = {"workload": "50 seeded random trees, odd sizes uniform on 1..63 (seed 1), 48 cases; one evaluation",
           "nodes": n, "device_us_p50": nearest_rank(dev, 0.5), "device_us_p99": nearest_rank(dev, 0.99),
           "call_us_p50": nearest_rank(wall, 0.5), "call_us_p99": nearest_rank(wall, 0.99),
           "rule": f"nearest rank over {reps} calls",
           "GPops_per_s_call": n * prob.n_cases / (nearest_rank(wall, 0.5) / 1e6)}
    if cpu:
        from oracle import oracle
        t = time.perf_counter()
        k = 0
        while time.perf_counter() - t < 2.0:
            oracle.eval_population(nodes, offs, x, y, c, n_threads=1)
            k += 1
        el = time.perf_counter() - t
        out["cpu_baseline"] = {"value": 1e6 * el / k, "unit": "us per evaluation", "cores": 1, "kind": "oracle",
                               "sample": f"{k} oracle evaluations of the 50 trees on 1 thread, {el:.1f} s"}
    return out


def config3_bloated(gp, prob, stream, cpu):
    """The 48 bloated trees (odd sizes log-uniform 1e6..4e8, 4.47e9 nodes, the
    largest grown into a stringy chain of depth above 1e5): every tree is cut
    into chunks and its upper trees are planned level by level.  Device time
    of gp_evaluate (the levels' host synchronisations included), the
    level-0 launches against the FP32 lane peak, and end to end from pinned
    host memory (upload and validation, evaluation, fitness read-back)."""
    import torch
    x, y, c = prob.x, prob.y, prob.consts
    t0 = time.perf_counter()
    nodes, offs, info = synth.graft_population(seed=4)
    build_s = time.perf_counter() - t0
    n_trees = offs.shape[0] - 1
    n = int(offs[-1])
    pop = gp.gp_create_population(prob, nodes, offs, stream)
    gp.gp_evaluate(pop, stream)
    gp.gp_fitness(pop)
    gp.gp_profile_read(reset=True)
    gp.gp_profile_enable(True)
    ms = []
    for _ in range(3):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        gp.gp_evaluate(pop, stream)
        b.record(stream)
        gp.gp_fitness(pop)
        ms.append(a.elapsed_time(b))
    gp.gp_profile_enable(False)
    prof = gp.gp_profile_read(reset=True)
    st = gp.gp_eval_stats_get(pop)
    gp.gp_destroy_population(pop)
    eval_ms = statistics.median(ms)
    l0 = prof["eval"]
    l0_ms = l0["ms"] / max(l0["launches"], 1)
    l0_ops = ((n - n_trees) // 2 - int(st["upper_ops"])) * prob.n_cases
    peaks, src = measured_peaks()
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    alu_peak = n_sm * 128 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
    # end to end: the trees from pinned host memory, through the public API
    pin = torch.from_numpy(nodes).pin_memory()
    pin_offs = torch.from_numpy(offs.astype(np.uint64).view(np.int64)).pin_memory()
    del nodes
    torch.cuda.synchronize()
    t = time.perf_counter()
    p2 = gp.gp_create_population(prob, pin.numpy(), pin_offs.numpy().view(np.uint64), stream)
    gp.gp_evaluate(p2, stream)
    gp.gp_fitness(p2)
    e2e_s = time.perf_counter() - t
    gp.gp_destroy_population(p2)
    out = {"workload": "48 bloated trees (seed 4), odd sizes log-uniform 1e6..4e8 grown by subtree-crossover "
                       "chains, the largest a stringy chain of depth above 1e5; 48 cases; one evaluation",
           "nodes": n, "depth_of_chain_tree": int(info["chain_depth"]), "population_build_s": build_s,
           "value": n * prob.n_cases / (eval_ms / 1e3), "unit": "GPops/s", "ms_p50": eval_ms, "runs": len(ms),
           "levels": int(st["levels"]), "items": int(st["items"]),
           "kernel_ms": {k: v["ms"] / len(ms) for k, v in prof.items() if v["launches"]},
           "roofline": {"bound": "alu", "kernel": "eval_kernel (level 0)", "launches": l0["launches"] // len(ms),
                        "achieved": l0_ops / (l0_ms / 1e3) / 1e12 if l0["launches"] else None,
                        "peak": alu_peak, "unit": "TFLOP/s",
                        "frac": l0_ops / (l0_ms / 1e3) / 1e12 / alu_peak if l0["launches"] else None,
                        "peak_note": f"{n_sm} SMs x 128 FP32 lanes x max clock ({src})"},
           "e2e": {"value": n * prob.n_cases / e2e_s, "unit": "GPops/s", "h2d_bytes_per_step": int(n + 8 * (n_trees + 1)),
                   "d2h_bytes_per_step": 4 * n_trees, "wall_s": e2e_s}}
    if cpu:
        from oracle import oracle
        sizes = np.diff(offs.astype(np.int64))
        order = np.argsort(sizes)
        pick, tot = [], 0
        for t_ in order:
            if len(pick) >= 16 and tot > 2 * 10 ** 7:
                break
            pick.append(int(t_))
            tot += int(sizes[t_])
        sub = np.concatenate([pin.numpy()[int(offs[t_]):int(offs[t_ + 1])] for t_ in pick])
        so = np.zeros(len(pick) + 1, np.uint64)
        np.cumsum(sizes[pick].astype(np.uint64), out=so[1:])
        cores = os.cpu_count() or 1
        t = time.perf_counter()
        k = 0
        while time.perf_counter() - t < 10.0:
            oracle.eval_population(sub, so, x, y, c, n_threads=cores)
            k += 1
        el = time.perf_counter() - t
        out["cpu_baseline"] = {"value": k * tot * prob.n_cases / el, "unit": "GPops/s", "cores": cores,
                               "kind": "oracle",
                               "sample": f"{k} x oracle evaluation of the {len(pick)} smallest trees "
                                         f"({tot} nodes) on {cores} threads, {el:.1f} s"}
    return out


def config4_batched(gp, prob, stream, flush, cpu, steps=3):
    """The batched generation at full size: 4000 parents of 1e2..1e8 nodes
    (2.9e10 nodes), generations made on the device (size-7 tournaments,
    4000 crossovers, evaluation of the children; graph replays) against the
    plain path as a host loop runs them (generations_compare).  End to end:
    from the parents in (page-locked) host memory to the children's fitness
    on the host, through gp_generation_create (upload, validation, the
    parents' evaluation), one step and gp_generation_fitness."""
    import torch
    x, y, c = prob.x, prob.y, prob.consts
    desc, make = BATCHED["batched"]
    t0 = time.perf_counter()
    nodes, offs = make()
    build_s = time.perf_counter() - t0
    n = offs.shape[0] - 1
    sizes = np.diff(offs.astype(np.int64))
    arena = int(int(np.sum((sizes + 15) // 16 * 16) + 64) * 1.3) + (64 << 20)
    t0 = time.perf_counter()
    G = gp.gp_generation_create(prob, nodes, offs, seed=SEED_GEN, arena_bytes=arena, use_graph=True, stream=stream)
    create_s = time.perf_counter() - t0
    info0 = gp.gp_generation_get_info(G)
    gp.gp_generation_step(G, 1, stream)
    recs = gp.gp_generation_records(G)
    info1 = gp.gp_generation_get_info(G)
    chunk = int(info0["chunk_nodes"])
    gp.gp_generation_destroy(G)
    del G
    torch.cuda.synchronize()
    cmp = generations_compare(gp, prob, nodes, offs, stream, flush, 2, 1, chunk=chunk, arena=arena,
                              shape=(info0["warps_per_cta"], info0["window_entries"], info0["upper_window_entries"]))
    child_nodes = int(info1["total_nodes"])
    # end to end from page-locked host memory (the parents' own pages registered)
    try:
        cudart = torch.cuda.cudart()
        reg = int(cudart.cudaHostRegister(nodes.ctypes.data, nodes.nbytes, 0)) == 0
    except (AttributeError, RuntimeError, TypeError):
        cudart, reg = None, False
    torch.cuda.synchronize()
    t = time.perf_counter()
    G = gp.gp_generation_create(prob, nodes, offs, seed=SEED_GEN, chunk_nodes=chunk, arena_bytes=arena,
                                use_graph=True, stream=stream, warps_per_cta=info0["warps_per_cta"],
                                window_entries=info0["window_entries"],
                                upper_window_entries=info0["upper_window_entries"])
    gp.gp_generation_step(G, 1, stream)
    gp.gp_generation_fitness(G)
    e2e_s = time.perf_counter() - t
    gp.gp_generation_destroy(G)
    del G
    if reg:
        cudart.cudaHostUnregister(nodes.ctypes.data)
    units = child_nodes * prob.n_cases
    out = {"workload": desc, "parent_nodes": int(offs[-1]), "child_nodes": child_nodes,
           "population_build_s": build_s, "create_s": create_s, "chunk_nodes": chunk,
           "autotune": {"chunk": {str(k): v for k, v in zip(info0["autotune_chunk"], info0["autotune_ms"]) if k},
                        "shape": {f"{lv} {w}x{k}": v for (w, k, lv), v in zip(info0["autotune_shape"],
                                                                              info0["autotune_shape_ms"]) if w}},
           "levels": int(info1["levels"]),
           "batched_vs_plain": cmp,
           "e2e": {"value": units / e2e_s, "unit": "GPops/s", "wall_s": e2e_s,
                   "h2d_bytes_per_step": int(nodes.nbytes + 8 * (n + 1)), "d2h_bytes_per_step": 4 * n,
                   "host_memory": "page-locked" if reg else "pageable",
                   "note": "upload, validation and evaluation of the parents, one generation, fitness read-back"}}
    if cpu:
        from oracle import oracle
        k = 20
        mum, dad, mp, dp = (np.asarray(a)[:k] for a in recs)
        cores = os.cpu_count() or 1
        t = time.perf_counter()
        reps, done = 0, 0
        while time.perf_counter() - t < 10.0:
            kn, ko = oracle.crossover_population(nodes, offs, mum, dad, mp, dp)
            oracle.eval_population(kn, ko, x, y, c, n_threads=cores)
            done += int(ko[-1])
            reps += 1
        el = time.perf_counter() - t
        out["cpu_baseline"] = {"value": done * prob.n_cases / el, "unit": "GPops/s", "cores": cores,
                               "kind": "oracle",
                               "sample": f"{reps} x (crossover of the first {k} of the generation's records + "
                                         f"oracle evaluation of those children on {cores} threads), {el:.1f} s"}
    return out


def crossover_large(gp, prob, stream, flush, reps=10):
    """Subtree crossover alone on large children: 2000 parents of 1e4..1e6
    nodes (crossover chains from 32 random donors of 1e4..1e5 nodes; seed 8),
    2000 children at uniform points (seed 13).  The copy kernel is bound by
    HBM: algorithmic bytes = the child bytes read + written."""
    import torch
    nodes, offs, _ = synth.graft_population(seed=8, count=2000, lo=10 ** 4, hi=10 ** 6, donor_lo=10 ** 4,
                                            donor_hi=10 ** 5, n_donors=32, chain_depth=0)
    with torch.cuda.stream(stream):
        parents = gp.gp_create_population(prob, nodes, offs, stream)
    sizes = np.diff(offs.astype(np.int64))
    xo = gp.make_xo(*synth.crossover_points(13, sizes, 2000))
    for _ in range(2):
        k = gp.gp_crossover(parents, xo, stream)
    child_bytes = int(gp.gp_population_get_info(k).total_nodes)
    del k
    torch.cuda.synchronize()
    gp.gp_profile_read(reset=True)
    gp.gp_profile_enable(True)
    ms = []
    for _ in range(reps):
        with torch.cuda.stream(stream):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            k = gp.gp_crossover(parents, xo, stream)
            b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
        del k
    gp.gp_profile_enable(False)
    prof = gp.gp_profile_read(reset=True)
    del parents
    copy_ms = prof["copy"]["ms"] / max(prof["copy"]["launches"], 1)
    peaks, src = measured_peaks()
    gbs = 2 * child_bytes / (copy_ms / 1e3) / 1e9
    return {"workload": "2000 parents, odd sizes log-uniform 1e4..1e6 (seed 8), 2000 children at uniform points "
                        "(seed 13), L2 flushed before each crossover",
            "child_bytes": child_bytes, "gp_crossover_ms_p50": statistics.median(ms),
            "kernel_ms_per_launch": {k_: v["ms"] / v["launches"] for k_, v in prof.items() if v["launches"]},
            "roofline": {"bound": "hbm", "kernel": "xo_copy_map_kernel", "achieved": gbs,
                         "peak": float(peaks["hbm_gbs"]), "unit": "GB/s", "frac": gbs / float(peaks["hbm_gbs"]),
                         "note": f"child bytes read + written / copy launch time; peak {src}"}}


SERVE_POOL = 2000


def config5_serving(gp, prob, stream, gens=1, n_runs=64, rate=200.0, budget=150 * 10 ** 9):
    """The serving loop at the benchmark's sizes: 64 independent runs, each
    population U{48..4000} trees drawn (with repeats) from a device pool of
    2000 seeded trees with odd sizes log-uniform on 11..1e8 (the initial
    populations average 1.4e10 nodes, 880 GB in all, so they are opened
    from the device pool, not staged on the host), an HBM budget of 150 GB
    for the runs' population buffers (a few runs fit at once), generation
    requests in a closed loop per run with exponential think times (Poisson
    at `rate` per second in aggregate).  Continuous batching against one
    run per batch on the same arrivals; two runs are then made alone from
    the same trees and must end identical (bytes and fitness)."""
    import threading
    import torch
    t0 = time.perf_counter()
    pn, po, _ = synth.graft_population(seed=6, count=SERVE_POOL, lo=11, hi=10 ** 8, donor_lo=10 ** 5,
                                       donor_hi=10 ** 6, n_donors=32, chain_depth=0)
    build_s = time.perf_counter() - t0
    with torch.cuda.stream(stream):
        pool = gp.gp_create_population(prob, pn, po, stream)
    psize = np.diff(po.astype(np.int64))
    rng = np.random.default_rng(66)
    picks = [rng.integers(0, SERVE_POOL, size=int(rng.integers(48, 4001))).astype(np.uint32) for _ in range(n_runs)]
    run_nodes = [int(np.sum(psize[p])) for p in picks]
    think = n_runs / rate
    # upper-level workspace from the pool's own fragment density at this
    # chunk size (codes and value entries per node, all levels summed) for
    # batches of at most the largest run's nodes, a fifth more to spare
    C = 16384
    gp.gp_evaluate(pool, stream, chunk_nodes=C)
    gp.gp_fitness(pool)
    es = gp.gp_eval_stats_get(pool)
    batch_nodes = int(max(run_nodes))
    ws_codes = int(1.2 * es["upper_codes"] / int(po[-1]) * batch_nodes) + (1 << 20)
    ws_values = int(1.2 * es["value_entries"] / int(po[-1]) * batch_nodes) + (1 << 18)
    torch.cuda.synchronize()

    free_b, total_b = torch.cuda.mem_get_info()
    print(f"serving: pool {int(po[-1])} nodes, stats {es}, largest run {max(run_nodes)}, batch_nodes {batch_nodes}, "
          f"workspace codes {ws_codes} ({4 * ws_codes / 1e9:.1f} GB) values {ws_values} "
          f"({192 * 1.125 * ws_values / 1e9:.1f} GB), device free {free_b / 1e9:.1f} of {total_b / 1e9:.1f} GB",
          file=sys.stderr, flush=True)

    def session(max_batch_runs):
        srv = gp.gp_server_create(prob, hbm_budget_bytes=budget, max_runs=n_runs, max_batch_trees=1 << 20,
                                  max_batch_runs=max_batch_runs, chunk_nodes=C, max_batch_nodes=batch_nodes,
                                  workspace_codes=ws_codes, workspace_values=ws_values)
        ids = []
        for k, p in enumerate(picks):
            used = int(np.sum((psize[p] + 15) // 16 * 16))
            ids.append(gp.gp_server_open_run_from(srv, pool, p, seed=9000 + k,
                                                  arena_bytes=int(1.3 * used) + (64 << 20)))
        errors = []

        def client(k, rid):
            r_ = np.random.default_rng(77 + k)
            try:
                for _ in range(gens):
                    time.sleep(float(r_.exponential(think)))
                    r = gp.gp_server_wait(srv, gp.gp_server_submit(srv, rid, 1), timeout_ms=300000.0)
                    if r["status"] != gp.GP_OK:
                        errors.append(r["status"])
                        break
            except gp.GpError as e:
                errors.append(e.status)
            if k not in check:                # a finished run frees room for the waiting ones
                gp.gp_server_close_run(srv, rid)

        t = time.perf_counter()
        th = [threading.Thread(target=client, args=(k, rid), daemon=True) for k, rid in enumerate(ids)]
        for x in th:
            x.start()
        for x in th:
            x.join(timeout=max(1.0, 600.0 - (time.perf_counter() - t)))
        if any(x.is_alive() for x in th):
            raise RuntimeError("serving session did not finish within 600 s")
        wall = time.perf_counter() - t
        st = gp.gp_server_get_stats(srv)
        return srv, ids, wall, st, errors

    out = {"workload": f"{n_runs} runs, populations U{{48..4000}} trees drawn from a device pool of {SERVE_POOL} "
                       "seeded trees (odd sizes log-uniform 11..1e8, grown by crossover chains above 1e6; seed 6); "
                       f"48 cases; {gens} generation(s) per run, one request each after an exponential think "
                       f"time (Poisson {rate:g}/s in aggregate); HBM budget {budget / 1e9:.0f} GB",
           "pool_nodes": int(po[-1]), "pool_build_s": build_s, "chunk_nodes": C,
           "workspace": {"batch_nodes": batch_nodes, "codes": ws_codes, "value_entries": ws_values,
                         "device_free_gb_before": free_b / 1e9, "device_total_gb": total_b / 1e9},
           "run_nodes": {"mean": float(np.mean(run_nodes)), "total": int(np.sum(run_nodes))},
           "generations_per_run": gens,
           "reduced": f"{gens} generation(s) per run instead of 100: one generation of a run averages about "
                      "0.5 s of GPU time here, so 64 runs x 100 generations would take about an hour"}
    check = set(sorted(range(n_runs), key=lambda k: run_nodes[k])[:2])   # made alone afterwards
    for name, mbr in (("continuous_batching", 0), ("one_run_per_batch", 1)):
        srv, ids, wall, st, errors = session(mbr)
        out[name] = {"wall_s": wall, "GPops_per_s_wall": st["child_nodes"] * prob.n_cases / wall,
                     "GPops_per_s_device": st["child_nodes"] * prob.n_cases / max(st["device_ms"] / 1e3, 1e-9),
                     "latency_p50_ms": st["latency_p50_ms"], "latency_p99_ms": st["latency_p99_ms"],
                     "batches": st["batches"], "mean_runs_per_batch": st["mean_runs_per_batch"],
                     "runs_admitted": st["runs_admitted"], "child_nodes": st["child_nodes"],
                     "runs_regrown": st["regrown"], "batch_retries": st["retries"], "failed_requests": len(errors)}
        if name == "continuous_batching":
            # the two smallest runs, made alone from the same trees, must end identical
            small = sorted(check)
            same = True
            for k in small:
                tn, to = gp.gp_server_run_trees(srv, ids[k])
                fa, _, _ = gp.gp_server_run_fitness(srv, ids[k])
                nodes_k, offs_k = synth.pack([pn[int(po[t]):int(po[t + 1])] for t in picks[k]])
                G = gp.gp_generation_create(prob, nodes_k, offs_k, seed=9000 + k, chunk_nodes=16384,
                                            use_graph=True, stream=stream)
                gp.gp_generation_step(G, gens, stream)
                an, ao = gp.gp_generation_trees(G)
                fb, _, _ = gp.gp_generation_fitness(G)
                gp.gp_generation_destroy(G)
                same = same and np.array_equal(tn, an) and np.array_equal(to, ao) and \
                    np.array_equal(fa.view(np.uint32), fb.view(np.uint32))
            out["alone_check"] = {"runs": [int(k) for k in small], "identical": bool(same)}
        for k in check:
            gp.gp_server_close_run(srv, ids[k])
        gp.gp_server_destroy(srv)
        del srv
    del pool
    return out


# ---------------------------------------------------------------------------
# reference arm: the oracle, timed as it stands on the host cores
# ---------------------------------------------------------------------------

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle
    oracle.build()
    x, y, c, nodes, offs, ops = make_workload(0)
    cores = os.cpu_count() or 1
    sample = 200
    mum, dad, mp, dp = (a[:sample] for a in ops)

    def step():
        rn, ro = oracle.crossover_population(nodes, offs, mum, dad, mp, dp)
        oracle.eval_population(rn, ro, x, y, c, n_threads=cores)
        return int(ro[-1])

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    n = 0
    times = []
    for _ in range(args.steps):
        a = time.perf_counter()
        n += step()
        times.append(time.perf_counter() - a)
    el = time.perf_counter() - t0
    value = n * len(x) / el
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GPops/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "trees": N_TREES,
                   "sample": f"each step: first {sample} of the 4000 crossover records"},
        "cpu_baseline": {"value": value, "unit": "GPops/s", "cores": cores, "kind": "oracle",
                         "sample": f"first {sample} of 4000 crossover records per step, oracle on {cores} threads"},
        "e2e": {"value": value, "unit": "GPops/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ---------------------------------------------------------------------------
# batched generations on the device (tournament selection + crossover +
# evaluation as one captured launch sequence per generation)
# ---------------------------------------------------------------------------

SEED_GEN = 21
BATCHED = {
    "generation4000": (
        "4000 seeded random prefix trees, odd sizes log-uniform 31..32767 nodes (seed 3), 48 Sextic "
        "cases, 127 constants; step = one generation on the device: size-7 tournaments for both "
        "parents of 4000 children, 4000 subtree crossovers at uniform points, evaluation of the children",
        lambda: synth.population_loguniform(seed=3, count=4000)),
    "batched": (
        "4000 parents, odd sizes log-uniform 1e2..1e8 nodes (seed 5; trees above 1e6 grown by crossover "
        "chains from a pool of 32 random donors of 1e5..1e6 nodes), 48 Sextic cases, 127 constants; "
        "step = one generation on the device (size-7 tournaments, 4000 crossovers, evaluation)",
        lambda: synth.graft_population(seed=5, count=4000, lo=100, hi=10**8, donor_lo=10**5,
                                       donor_hi=10**6, n_donors=32, chain_depth=0)[:2]),
    "batched-reduced": (
        "4000 parents, odd sizes log-uniform 1e2..1e6 nodes (seed 5; trees above 1e5 grown by crossover "
        "chains from 32 random donors of 1e4..1e5 nodes), 48 Sextic cases; step = one generation on "
        "the device (size-7 tournaments, 4000 crossovers, evaluation)",
        lambda: synth.graft_population(seed=5, count=4000, lo=100, hi=10**6, donor_lo=10**4,
                                       donor_hi=10**5, n_donors=32, chain_depth=0)[:2]),
}


def run_batched(args):
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1902_09215_gb300 import gp
    gp.lib()
    desc, make = BATCHED[args.workload]
    x, y, c = synth.problem(const_seed=CONST_SEED)
    t0 = time.perf_counter()
    nodes, offs = make()
    gen_s = time.perf_counter() - t0
    n = offs.shape[0] - 1
    sizes = np.diff(offs.astype(np.int64))
    used = int(np.sum((sizes + 15) // 16 * 16)) + 64
    stream = torch.cuda.Stream(dev)
    prob = gp.Problem(x, y, c)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    arena = int(used * 1.3) + (64 << 20)

    def measure(G, steps):
        """Generation 0 -> 1 repeated: step (timed), rewind (not timed)."""
        for _ in range(args.warmup):
            gp.gp_generation_step(G, 1, stream)
            gp.gp_generation_rewind(G, stream)
        ms = []
        l0 = gp.gp_kernel_launch_count()
        for _ in range(steps):
            with torch.cuda.stream(stream):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                gp.gp_generation_step(G, 1, stream)
                b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
            gp.gp_generation_rewind(G, stream)
        launches = gp.gp_kernel_launch_count() - l0
        return ms, launches

    t0 = time.perf_counter()
    G = gp.gp_generation_create(prob, nodes, offs, seed=SEED_GEN, chunk_nodes=args.chunk,
                                arena_bytes=arena, use_graph=True, stream=stream)
    create_s = time.perf_counter() - t0
    info0 = gp.gp_generation_get_info(G)
    with ClockSampler(0) as clk:
        ms, launches = measure(G, args.steps)
    gp.gp_generation_step(G, 1, stream)
    recs = gp.gp_generation_records(G)
    info1 = gp.gp_generation_get_info(G)
    child_nodes = int(info1["total_nodes"])
    # end to end through the API: one generation and the read-back of its fitness
    gp.gp_generation_rewind(G, stream)
    te = []
    for _ in range(max(3, args.steps // 2)):
        torch.cuda.synchronize()
        a = time.perf_counter()
        gp.gp_generation_step(G, 1, stream)
        gp.gp_generation_fitness(G)
        te.append(time.perf_counter() - a)
        gp.gp_generation_rewind(G, stream)
    gp.gp_generation_destroy(G)
    del G
    torch.cuda.synchronize()

    # the same launch sequence without the graph
    G = gp.gp_generation_create(prob, nodes, offs, seed=SEED_GEN, chunk_nodes=info0["chunk_nodes"],
                                arena_bytes=arena, use_graph=False, stream=stream)
    ms_ng, _ = measure(G, max(3, args.steps // 2))
    gp.gp_generation_destroy(G)
    del G
    torch.cuda.synchronize()

    # host-driven path: the same crossover records through gp_crossover +
    # gp_evaluate (host synchronisations to size children and upper trees)
    with torch.cuda.stream(stream):
        parents = gp.gp_create_population(prob, nodes, offs, stream)
    xo = gp.make_xo(*recs)
    ms_plain = []
    for k in range(max(3, args.steps // 2) + 1):
        with torch.cuda.stream(stream):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            kids = gp.gp_crossover(parents, xo, stream)
            gp.gp_evaluate(kids, stream)
            b.record(stream)
        gp.gp_fitness(kids)
        if k:                                         # first one warms the pool
            ms_plain.append(a.elapsed_time(b))
        del kids
    del parents
    torch.cuda.synchronize()

    med = statistics.median(ms)
    units = child_nodes * len(x)
    line = {
        "metric": "GPops/s (tree nodes x fitness cases per second), batched generation",
        "value": units / (med / 1e3), "unit": "GPops/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": med, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": desc, "trees": n, "parent_nodes": int(offs[-1]), "child_nodes": child_nodes,
                   "cases": len(x), "seeds": {"run": SEED_GEN, "constants": CONST_SEED},
                   "l2": "flushed before every timed step (256 MB write, outside the events)",
                   "chunk_nodes": info0["chunk_nodes"], "levels": info1["levels"],
                   "kernels_per_generation": info0["kernels_per_generation"],
                   "arena_bytes": arena, "workspace": [info0["workspace_codes"], info0["workspace_values"]],
                   "population_build_s": gen_s, "create_s": create_s},
        "latency_ms": {"p50": med, "p99": nearest_rank(ms, 0.99), "rule": f"nearest rank over {len(ms)} steps"},
        "autotune": {str(k): v for k, v in zip(info0["autotune_chunk"], info0["autotune_ms"]) if k},
        "autotune_shape": {f"{lv} {w}x{k}": v for (w, k, lv), v in zip(info0["autotune_shape"], info0["autotune_shape_ms"])
                           if w},
        "launch_shape": {"level0": [info0["warps_per_cta"], info0["window_entries"]],
                         "upper": [info0["upper_warps"], info0["upper_window_entries"]],
                         "ropes": [info0["rope_warps"], info0["rope_window_entries"]]},
        "clocks": clk.summary(),
        "e2e": {"value": units / statistics.median(te), "unit": "GPops/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 4 * n, "wall_s_p50": statistics.median(te),
                "note": "population resident on the device; per step: one generation + fitness read-back"},
        "gpu_launches": int(launches),
        "compare": {
            "device_sequence_no_graph": {"ms_p50": statistics.median(ms_ng),
                                         "value": units / (statistics.median(ms_ng) / 1e3)},
            "host_driven_crossover_then_evaluate": {"ms_p50": statistics.median(ms_plain),
                                                    "value": units / (statistics.median(ms_plain) / 1e3)},
        },
    }
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# serving: many independent runs, continuous batching, HBM-budget admission
# ---------------------------------------------------------------------------

SERVE_RUNS, SERVE_RATE = 64, 200.0


def serving_workload(n_runs, gens):
    """Populations of U{48..4000} trees drawn from a shared pool of seeded
    random trees (odd sizes log-uniform 11..1e5)."""
    rng = np.random.default_rng(6)
    pool_sizes = synth.loguniform_sizes(rng, 12000, 11, 100001)
    pool = [synth.random_tree(rng, int(n)) for n in pool_sizes]
    runs = []
    for r in range(n_runs):
        n = int(rng.integers(48, 4001))
        pick = rng.integers(0, len(pool), size=n)
        nodes, offs = synth.pack([pool[int(k)] for k in pick])
        runs.append((nodes, offs, 5000 + r))
    return runs


def serve_session(gp, prob, runs, gens, budget, max_batch_runs, think_mean_s, seed):
    """Every run: `gens` one-generation requests in a closed loop with an
    exponential think time before each; runs close when done (admitting the
    waiting ones).  Returns wall seconds and the server's statistics."""
    import threading
    srv = gp.gp_server_create(prob, hbm_budget_bytes=budget, max_runs=len(runs), max_batch_trees=1 << 20,
                              max_batch_runs=max_batch_runs, chunk_nodes=8192)
    ids = [gp.gp_server_open_run(srv, n, o, seed=s) for n, o, s in runs]
    errors = []

    def client(k, rid):
        rng = np.random.default_rng(seed + k)
        for _ in range(gens):
            if think_mean_s > 0:
                time.sleep(float(rng.exponential(think_mean_s)))
            r = gp.gp_server_wait(srv, gp.gp_server_submit(srv, rid, 1))
            if r["status"] != gp.GP_OK:
                errors.append(r["status"])
                break
        gp.gp_server_close_run(srv, rid)

    t0 = time.perf_counter()
    th = [threading.Thread(target=client, args=(k, rid)) for k, rid in enumerate(ids)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    wall = time.perf_counter() - t0
    st = gp.gp_server_get_stats(srv)
    gp.gp_server_destroy(srv)
    if errors:
        raise RuntimeError(f"serving requests failed: {errors[:5]}")
    return wall, st


def run_serving_full(args):
    """The serving configuration at the benchmark's sizes alone (the same leg
    as in the default line)."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1902_09215_gb300 import gp
    gp.lib()
    x, y, c = synth.problem(const_seed=CONST_SEED)
    prob = gp.Problem(x, y, c)
    stream = torch.cuda.Stream(torch.device("cuda", 0))
    with ClockSampler(0) as clk:
        out = config5_serving(gp, prob, stream, gens=args.serve_gens_full)
    b = out["continuous_batching"]
    print(json.dumps({"metric": "GPops/s (tree nodes x fitness cases per second), served generations; p50/p99 latency",
                      "value": b["GPops_per_s_wall"], "unit": "GPops/s", "n_gpus": 1, "higher_is_better": True,
                      "dtype": "f32", "data": "synthetic", "config": {"workload": out["workload"]},
                      "serving": out, "clocks": clk.summary()}))


def run_serving(args):
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1902_09215_gb300 import gp
    gp.lib()
    x, y, c = synth.problem(const_seed=CONST_SEED)
    prob = gp.Problem(x, y, c)
    gens = args.serve_gens
    t0 = time.perf_counter()
    runs = serving_workload(SERVE_RUNS, gens)
    build_s = time.perf_counter() - t0
    per_run = [2 * (2 * int(np.sum((np.diff(o.astype(np.int64)) + 15) // 16 * 16)) + 16 * (len(o) - 1) + (1 << 20))
               for _, o, _ in runs]
    budget = int(np.sum(per_run) / 4)                 # about a quarter of the runs fit at once
    think = SERVE_RUNS / SERVE_RATE
    with ClockSampler(0) as clk:
        out = {}
        for name, mbr, th in (("batched", 0, think), ("one_run_per_batch", 1, think),
                              ("batched_saturated", 0, 0.0), ("one_run_per_batch_saturated", 1, 0.0)):
            wall, st = serve_session(gp, prob, runs, gens, budget, mbr, th, 11)
            out[name] = {
                "wall_s": wall,
                "GPops_per_s_wall": st["child_nodes"] * len(x) / wall,
                "GPops_per_s_device": st["child_nodes"] * len(x) / (st["device_ms"] / 1e3),
                "latency_p50_ms": st["latency_p50_ms"], "latency_p99_ms": st["latency_p99_ms"],
                "batches": st["batches"], "mean_runs_per_batch": st["mean_runs_per_batch"],
                "run_generations": st["run_generations"], "child_nodes": st["child_nodes"],
                "runs_regrown": st["regrown"], "batch_retries": st["retries"],
            }
    b = out["batched_saturated"]
    line = {
        "metric": "GPops/s (tree nodes x fitness cases per second), served generations; p50/p99 latency",
        "value": b["GPops_per_s_wall"], "unit": "GPops/s", "n_gpus": 1, "steps": SERVE_RUNS * gens,
        "warmup": 0, "ms_per_step": 1e3 * b["wall_s"] / (SERVE_RUNS * gens), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{SERVE_RUNS} independent runs, populations U{{48..4000}} trees drawn from a "
                               "pool of 12000 seeded random trees (odd sizes log-uniform 11..1e5), 48 Sextic "
                               f"cases; each run makes {gens} generations, one request per generation in a "
                               f"closed loop (exponential think time, mean {think:.2f} s = Poisson "
                               f"{SERVE_RATE:.0f}/s in aggregate; none in the saturated phases)",
                   "hbm_budget_bytes": budget, "runs_fitting_at_once": "about 1/4",
                   "population_build_s": build_s},
        "phases": out,
        "clocks": clk.summary(),
    }
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# the paper's run loop: ramped half-and-half, tournaments, crossover, N gens
# ---------------------------------------------------------------------------

def run_ltee(args):
    """The paper's run loop on the device: a ramped half-and-half population,
    then generation after generation of size-7 tournaments, subtree crossover
    and evaluation, each generation replayed from the captured graph.  After
    every generation the host reads the fitness (which reports a generation
    that ran out of room) and the population's size; a generation that
    outgrew the buffers is made again after gp_generation_recover.  The
    throughput counts every child node evaluated on every case."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1902_09215_gb300 import gp
    gp.lib()
    x, y, c = synth.problem(const_seed=CONST_SEED)
    prob = gp.Problem(x, y, c)
    nodes, offs = synth.ramped_half_and_half(seed=1, count=4000)
    stream = torch.cuda.Stream(torch.device("cuda", 0))
    G = gp.gp_generation_create(prob, nodes, offs, seed=SEED_GEN, chunk_nodes=args.chunk, use_graph=True,
                                stream=stream)
    info0 = gp.gp_generation_get_info(G)
    sizes, best_fit = [int(offs[-1])], []
    recoveries, done, evaluated = 0, 0, 0
    t0 = time.perf_counter()
    while done < args.generations and time.perf_counter() - t0 < args.time_limit:
        gp.gp_generation_step(G, 1, stream)
        try:
            fit, _, _ = gp.gp_generation_fitness(G)
        except gp.GpError as e:
            if e.status != gp.GP_ENOMEM:
                raise
            gp.gp_generation_recover(G, stream)        # bloat: larger buffers, the same generation again
            recoveries += 1
            continue
        info = gp.gp_generation_get_info(G)
        done = int(info["generation"])
        evaluated += int(info["total_nodes"])
        sizes.append(int(info["total_nodes"]))
        best_fit.append(float(np.nanmin(fit)))
        if done % 200 == 0:
            print(f"ltee: generation {done}, {sizes[-1]} nodes, {time.perf_counter() - t0:.1f} s, "
                  f"{recoveries} recoveries", file=sys.stderr, flush=True)
    wall = time.perf_counter() - t0
    fit, _, hits = gp.gp_generation_fitness(G, hits=True)
    best = int(np.argmin(np.where(np.isnan(fit), np.inf, fit)))
    info = gp.gp_generation_get_info(G)
    every = max(1, len(sizes) // 20)
    line = {
        "metric": "GPops/s (tree nodes x fitness cases per second), the paper's run loop",
        "value": evaluated * len(x) / wall, "unit": "GPops/s", "n_gpus": 1,
        "steps": done, "warmup": 0, "ms_per_step": 1e3 * wall / max(done, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"4000 ramped half-and-half trees (depths 2..6, seed 1), 48 Sextic cases, "
                               f"size-7 tournaments, subtree crossover on every child, {done} "
                               "generations made on the device from a captured graph, the host reading "
                               "fitness and sizes after each",
                   "stop": f"{args.generations} generations or {args.time_limit:g} s, whichever came first",
                   "seeds": {"population": 1, "run": SEED_GEN, "constants": CONST_SEED},
                   "timed": "wall clock around the whole loop, host reads and recoveries included"},
        "population_nodes": {"initial": sizes[0], "final": sizes[-1], "every": every,
                             "samples": sizes[::every]},
        "best_fitness": {"every": every, "samples": best_fit[::every]},
        "recoveries": recoveries,
        "chunk_nodes": int(info0["chunk_nodes"]), "levels_last": int(info["levels"]),
        "autotune": {str(k): v for k, v in zip(info0["autotune_chunk"], info0["autotune_ms"]) if k},
        "arena_bytes": int(info["arena_bytes"]),
        "workspace": {"codes": int(info["workspace_codes"]), "values": int(info["workspace_values"])},
        "best": {"tree": best, "fitness": float(fit[best]), "hits": int(hits[best])},
        "wall_s": wall,
    }
    gp.gp_generation_destroy(G)
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline leg")
    ap.add_argument("--no-extra", action="store_true",
                    help="time the 4000-tree step only (not the benchmark's other configurations)")
    ap.add_argument("--serve-gens", type=int, default=10, help="generations per run in the serving workload")
    ap.add_argument("--generations", type=int, default=200, help="generations of the ltee workload")
    ap.add_argument("--time-limit", type=float, default=120.0,
                    help="the ltee workload stops after this many seconds (bloat makes generations slower)")
    ap.add_argument("--serve-gens-full", type=int, default=1,
                    help="generations per run in the serving-full workload")
    ap.add_argument("--workload", choices=["step4000", "serving", "serving-full", "ltee"] + sorted(BATCHED),
                    default="step4000",
                    help="step4000 (default): crossover + evaluation of the 4000-tree population; "
                         "the others time whole generations made on the device")
    ap.add_argument("--chunk", type=int, default=0, help="evaluator chunk for the batched workloads (0 = autotune)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.workload != "step4000":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the reference arm times the step4000 workload only"}))
            return
        {"serving": run_serving, "serving-full": run_serving_full, "ltee": run_ltee}.get(args.workload,
                                                                                       run_batched)(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
