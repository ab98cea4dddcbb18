"""Benchmark: bottom-up semantic enumeration of LTLf formulae on GB300.

One step = one complete synthesis of the mid-scale workload (5 propositions,
64 + 64 traces of length 8..32 labelled by a hidden size-11 formula, 512-byte
characteristic matrices, 64 GiB language cache): atoms, every level until the
first separating formula, and the formula's reconstruction. The metric is
unique formulas (new characteristic matrices) per second over the timed steps;
per-level HBM GB/s and the roofline of the dominant kernel come with it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl lsyn|reference]

Under torchrun every rank solves its own replica of the problem: problems are
independent, so there is no collective on the data path (weak scaling); ranks
meet only at the barrier and the max-over-ranks timing reduction.
``--impl reference`` times the CPU oracle on a bounded sample of the same
workload on the host cores.
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
import types

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "mid-scale plain solve: 5 props, 64+64 traces, len U[8,32], Bernoulli(0.5), hidden size 11, " \
           "128 x uint32 words (512 B) per CM, 64 GiB cache, until first solution (seed 2: minimal size 11)"
METRIC = "unique formulas/sec"
CACHE_BYTES = 64 << 30
MAX_SIZE = 16
LARGE_CACHE_BYTES = 150 * 10**9
LARGE_WORKLOAD = ("large plain solve: 10 props, 1024+1024 traces, len U[16,64], Bernoulli(p) with p U[0.2,0.8] per "
                  "prop, hidden size 15, 2048 x uint64 words (16 KiB) per CM, 150 GB cache; every level built "
                  "completely until the cache fills (the cache-full path; seed 0 separates at size 5 already)")
E3_WORKLOAD = ("the paper's worked example: 7 positive + 7 negative traces of length 6 over {a, b}, the paper's "
               "grammar (atoms, not, and, X, F, U), minimal size 16, 16 GiB cache")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:  # noqa: BLE001
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={','.join(self.FIELDS)}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:  # noqa: BLE001
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
            except Exception:  # noqa: BLE001
                self.proc.kill()

    def summary(self):
        rows = []
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) != len(self.FIELDS):
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[4:]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _reduce_max(value: float, world: int, device=None) -> float:
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _reduce_sum(value: float, world: int, device=None) -> float:
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:  # noqa: BLE001
        return os.cpu_count() or 1


def cpu_baseline(problem, max_level: int, threads: int = 1, op_mask: int = 0x7F):
    """The oracle, as it stands, on a bounded sample of the timed problem:
    levels 1..max_level built completely, on one host core (the sequential
    listing) or on `threads` cores (each level's candidates shared out among
    threads, thread-local sets merged per level)."""
    import oracle
    spec = oracle.Spec.from_problem(problem)
    t0 = time.perf_counter()
    run = spec.enumerate(max_level, op_mask) if threads == 1 else spec.enumerate_threads(max_level, threads, op_mask)
    dt = time.perf_counter() - t0
    uniq = sum(run.size(k) for k in range(1, max_level + 1))
    del run
    return {"value": uniq / dt, "unit": METRIC, "cores": threads, "kind": "oracle",
            "sample": f"levels 1..{max_level} of the timed problem built completely ({uniq} unique formulas, "
                      f"{dt:.1f} s on {threads} host core{'s' if threads > 1 else ''})",
            "seconds": dt}


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    from paper_2504_18943_gb300 import workloads as W
    import oracle
    problem = W.mid_problem(args.seed, oracle.labeller)
    cores = host_cores()
    for _ in range(args.warmup):
        cpu_baseline(problem, args.ref_levels, cores)
    total_u, total_t = 0.0, 0.0
    for _ in range(args.steps):
        b = cpu_baseline(problem, args.ref_levels, cores)
        total_u += b["value"] * b["seconds"]
        total_t += b["seconds"]
    value = total_u / total_t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "unique formulas/sec",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * total_t / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "seed": args.seed, "sample_levels": args.ref_levels},
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": cores, "kind": "oracle",
                             "sample": f"levels 1..{args.ref_levels} of the mid-scale problem per step, each "
                                       f"level's candidates shared out among {cores} host threads"},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# One-problem workloads: (problem maker, cache bytes, max size, op mask, word type, description,
# default steps, CPU-baseline levels (one core, all cores)).
def _one_problem_workloads():
    return {
        "mid": dict(make=lambda W, lab, seed: W.mid_problem(seed, lab), cache=CACHE_BYTES, max_size=MAX_SIZE,
                    op_mask=0x7F, dtype="u32", desc=WORKLOAD, steps=30, cpu_levels=(7, 8),
                    kernels={"unary": "k_unary_c (not/X/F/G level kernel, 512-byte CMs)",
                             "binary": "k_binary_c + k_binary_small_c (and/or/U level kernels, 512-byte CMs)"}),
        "large": dict(make=lambda W, lab, seed: W.large_problem(seed, lab), cache=LARGE_CACHE_BYTES, max_size=15,
                      op_mask=0x7F, dtype="u64", desc=LARGE_WORKLOAD, steps=3, cpu_levels=(4, 5), fill=True,
                      kernels={"unary": "k_unary_d (not/X/F/G level kernel, 16 KiB CMs)",
                               "binary": "k_binary_d (and/or/U level kernel, 16 KiB CMs)"}),
        "e3": dict(make=lambda W, lab, seed: _paper_example(W), cache=16 << 30, max_size=16,
                   op_mask=0x1B | 0x40, dtype="u32", desc=E3_WORKLOAD, steps=5, cpu_levels=(12, 14),
                   kernels={"unary": "k_unary_a (not/X/F/G level kernel, 64-byte CMs)",
                            "binary": "k_binary_a (and/U level kernel, 64-byte CMs)"}),
    }


def _paper_example(W):
    g = _golden()["size16"]
    return W.problem_from_strings("e3", g["positive"], g["negative"], g["props"])


def _golden():
    with open(os.path.join(ROOT, "tests", "golden", "paper_examples.json")) as f:
        return json.load(f)


def run_lsyn(args):
    import numpy as np
    import torch

    world, rank, local = _dist()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    from paper_2504_18943_gb300 import build
    build.build()
    from paper_2504_18943_gb300 import lsyn as L
    from paper_2504_18943_gb300 import workloads as W

    wl = _one_problem_workloads()[args.workload]
    seed = args.seed if args.workload != "large" else args.large_seed
    # every rank solves the same problem: replicas, fixed work per GPU
    problem = wl["make"](W, L.labeller, seed)
    packed = L.pack_problem(problem)
    stream = torch.cuda.current_stream(dev)
    cache = wl["cache"]
    fill = wl.get("fill", False)
    cfg = L.torch_config(op_mask=wl["op_mask"], cache_bytes=cache, timing=True, stream=stream, device=local,
                         full_levels=fill)
    ctx = L.lsyn_create(packed, cfg)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)  # > L2 (129 MB)

    def run_on(c):
        if not fill:
            return L.lsyn_solve(c, wl["max_size"])
        # every level completely, until the cache is full (or max_size)
        levels = []
        for k in range(1, wl["max_size"] + 1):
            levels.append(L.lsyn_enumerate_level(c, k))
            if levels[-1].cache_full:
                break
        solved = [lv.level for lv in levels if lv.solved]
        res = types.SimpleNamespace(unique=levels[-1].total, launches=sum(lv.launches for lv in levels),
                                    constructed=sum(lv.candidates for lv in levels),
                                    size=solved[0] if solved else 0)
        return (L.LSYN_E_CACHE_FULL if levels[-1].cache_full else L.LSYN_NOT_FOUND), res, None, levels

    def step():
        L.lsyn_reset(ctx)
        return run_on(ctx)

    for _ in range(max(args.warmup, 0)):
        st, res, formula, levels = step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()

    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    uniques, launches, all_levels, constructed = 0, 0, [], 0
    kbytes = {"unary": 0.0, "binary": 0.0}
    kms = {"unary": 0.0, "binary": 0.0}
    klaunch = {"unary": 0, "binary": 0}
    results = []
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:  # noqa: BLE001
        gpu_id = str(local)
    with ClockSampler(gpu_id) as clocks:
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.zero_()
            ev0[i].record(stream)
            st, res, formula, levels = step()
            ev1[i].record(stream)
            results.append((st, res.size, formula))
            uniques += res.unique
            launches += res.launches
            constructed += res.constructed
            for lv in levels:
                for name, idx, b in (("unary", 0, lv.bytes_unary), ("binary", 1, lv.bytes_binary)):
                    if lv.kernel_ms[idx] > 0:
                        kbytes[name] += b
                        kms[name] += lv.kernel_ms[idx]
                        klaunch[name] += 1
            all_levels = levels
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    elapsed_ms = sum(a.elapsed_time(b) for a, b in zip(ev0, ev1))
    max_ms = _reduce_max(elapsed_ms, world, dev)
    total_uniques = _reduce_sum(float(uniques), world, dev)
    value = total_uniques / (max_ms / 1000.0)

    L.lsyn_destroy(ctx)  # its memory goes back to the allocator for the end-to-end contexts
    ctx = None
    # End to end through the public API from pinned host buffers: create
    # (host->device copy of the traces), solve, read the formula back, destroy;
    # L2 flushed before each step as for the device-timed steps.
    pinned_atoms = torch.from_numpy(packed.atom_words.view(np.int32 if packed.word_bits == 32 else np.int64))
    pinned_atoms = pinned_atoms.pin_memory()
    pinned_len = torch.from_numpy(packed.lengths).pin_memory()
    host_problem = L.PackedProblem(packed.n_props, packed.n_pos, packed.n_neg, packed.word_bits,
                                   pinned_len.numpy(), pinned_atoms.numpy().view(packed.word_dtype))
    e2e_uniques, e2e_ms = 0, 0.0
    e2e_steps = max(1, min(args.steps, 5))
    for i in range(e2e_steps + 1):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c2 = L.lsyn_create(host_problem, L.torch_config(op_mask=wl["op_mask"], cache_bytes=cache, stream=stream,
                                                        device=local, full_levels=fill))
        st2, r2, f2, _ = run_on(c2)
        L.lsyn_destroy(c2)
        dt = (time.perf_counter() - t0) * 1000.0
        if i > 0:  # the first call warms the allocator cache
            e2e_uniques += r2.unique
            e2e_ms += dt
    e2e_ms = _reduce_max(e2e_ms, world, dev)
    e2e_total = _reduce_sum(float(e2e_uniques), world, dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle  # the CPU-baseline leg only  # noqa: F401
        one_lv, all_lv = wl["cpu_levels"]
        cores = host_cores()
        cpu = cpu_baseline(problem, all_lv, cores, wl["op_mask"])
        one = cpu_baseline(problem, one_lv, 1, wl["op_mask"])
        cpu.pop("seconds", None)
        one.pop("seconds", None)
        cpu["single_core"] = one

    peak, peak_kind = _peaks()
    # The dominant kernel: the level-kernel family with the most device time in
    # the timed region (CUDA events around each launch, on the library's stream).
    dom = max(kms, key=lambda n: kms[n])
    achieved = (kbytes[dom] / 1e9) / (kms[dom] / 1e3) if kms[dom] > 0 else 0.0
    alg_per_launch = kbytes[dom] / max(1, klaunch[dom])
    traffic = None
    try:
        # DRAM bytes per algorithmic byte from an ncu capture of the same
        # kernel source, scaled to this run's average launch.
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            tj = json.load(f).get(f"{args.workload}:{dom}", {})
        if tj.get("source_sha") == _kernel_sha():
            traffic = alg_per_launch * tj["dram_bytes"] / tj["alg_bytes"]
    except Exception:  # noqa: BLE001
        pass
    per_level = [{"level": lv.level, "unique": lv.unique, "candidates": lv.candidates, "ms": round(lv.ms, 3),
                  "binary_ms": round(lv.kernel_ms[1], 3), "unary_ms": round(lv.kernel_ms[0], 3),
                  "gbs_alg": round(lv.bytes_alg / 1e9 / (max(lv.ms, 1e-6) / 1e3), 1),
                  "binary_gbs_alg": round(lv.bytes_binary / 1e9 / (lv.kernel_ms[1] / 1e3), 1)
                  if lv.kernel_ms[1] > 0.05 else None,
                  "unary_gbs_alg": round(lv.bytes_unary / 1e9 / (lv.kernel_ms[0] / 1e3), 1)
                  if lv.kernel_ms[0] > 0.05 else None,
                  "unique_per_s": round(lv.unique / (max(lv.ms, 1e-6) / 1e3), 1),
                  "cache_full": lv.cache_full} for lv in all_levels]
    if rank == 0:
        st, size, formula = results[-1]
        line = {
            "metric": METRIC, "value": value, "unit": "unique formulas/sec", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": max_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": wl["dtype"],
            "data": "synthetic",
            "config": {"workload": wl["desc"], "seed": seed, "min_size": size, "l2_flush": True,
                       "parallelism": f"replicas{world}" if world > 1 else "single",
                       "formula": formula, "status": st, "cache_bytes": cache},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak if peak else None, "traffic": traffic,
                         "kernel": wl["kernels"][dom], "peak_source": peak_kind,
                         "alg_bytes_per_launch": alg_per_launch, "launches": klaunch[dom],
                         "other": {n: {"achieved": (kbytes[n] / 1e9) / (kms[n] / 1e3) if kms[n] else None,
                                       "ms": kms[n]} for n in kms if n != dom}},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_total / (e2e_ms / 1000.0) if e2e_ms > 0 else None, "unit": "unique formulas/sec",
                    "h2d_bytes_per_step": packed.h2d_bytes, "d2h_bytes_per_step": 1 << 16,
                    "steps": e2e_steps, "l2_flush": True},
            "gpu_launches": launches,
            "clocks": clocks.summary(),
            "levels": per_level,
        }
        if args.workload == "e3":
            g = _golden()["size16"]
            line["time_to_formula_ms"] = max_ms / args.steps
            line["constructed_per_solve"] = constructed / args.steps
            line["paper_context"] = {
                "formulae_constructed": g["formulae_constructed_paper"], "seconds": g["seconds_paper"],
                "hardware": "not named in the paper", "note": "context only: the paper builds every ordered pair "
                "and names no GPU; this library builds and/or once per unordered pair"}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# Batched and served workloads (problems/s, time-to-formula)
# ---------------------------------------------------------------------------

BATCH_N = 256
BATCH_MAX_SIZE = 13
BATCH_CACHE = 8 << 30  # each problem's cap: the same for the batch, the server and the plain path
BATCH_WORKLOAD = ("batched: 256 seeded problems (base seed 1000) of the batched distribution: props U[2,8], "
                  "traces U[8,512] split evenly, lengths U[8,64] (uint64 words), hidden size U[5,13]; "
                  "max size 13, 8 GiB cache cap per problem")


def _batched_problems(L, W, n=BATCH_N):
    return [L.pack_problem(W.batched_problem(1000, i, L.labeller)) for i in range(n)]


def _percentile(xs, q):
    xs = sorted(xs)
    return xs[min(len(xs) - 1, int(q * len(xs)))] if xs else None


def _plain_service_times(L, packed, max_size, cache):
    """Each problem alone through the plain path (create, solve, destroy), warm
    allocator: (status, size, seconds) per problem."""
    import torch
    cfg = L.torch_config(cache_bytes=cache)
    out = []
    for q in packed:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with L.Synthesizer(q, cfg) as s:
            st, res, f, _ = s.solve(max_size)
        torch.cuda.synchronize()
        out.append((st, res.size, time.perf_counter() - t0))
    return out


def run_batched(args):
    import torch
    world, rank, local = _dist()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    from paper_2504_18943_gb300 import build
    build.build()
    from paper_2504_18943_gb300 import lsyn as L
    from paper_2504_18943_gb300 import workloads as W
    packed = _batched_problems(L, W)
    cfg = L.make_config(cache_bytes=BATCH_CACHE, device=local)
    b = L.Batch(packed, cfg)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(clocks=None):
        total, lat, out = 0.0, [], None
        for _ in range(args.steps):
            torch.cuda.synchronize()
            ev0.record()
            out = b.solve(BATCH_MAX_SIZE)
            ev1.record()
            torch.cuda.synchronize()
            total += ev0.elapsed_time(ev1)
            lat += [r.ms for r in out[1]]
        return total, lat, out

    tuned, default_ms = None, None
    if args.autotune:
        # the defaults first, then the autotuner's point, on the same batch
        for _ in range(args.warmup):
            b.solve(BATCH_MAX_SIZE)
        default_ms, _, _ = timed()
        tuned = b.autotune(BATCH_MAX_SIZE)  # keeps its choice for the solves below
    for _ in range(args.warmup):
        b.solve(BATCH_MAX_SIZE)
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:  # noqa: BLE001
        gpu_id = str(local)
    with ClockSampler(gpu_id) as clocks:
        total_ms, lat, (statuses, results, formulas) = timed()
    stats, trace = b.stats(), b.trace()
    b.close()
    max_ms = _reduce_max(total_ms, world)
    value = world * BATCH_N * args.steps / (max_ms / 1000.0)
    # end to end through the public API: create from host arrays, solve, read answers, destroy
    t0 = time.perf_counter()
    with L.Batch(packed, cfg, tuned) as b2:
        b2.solve(BATCH_MAX_SIZE)
    e2e_s = time.perf_counter() - t0
    plain = _plain_service_times(L, packed, BATCH_MAX_SIZE, BATCH_CACHE) if not args.no_plain else None
    line = None
    if rank == 0:
        same = None
        plain_d = None
        if plain:
            same = all((statuses[i] == plain[i][0]) for i in range(BATCH_N))
            t_all = sum(p[2] for p in plain)
            finish, acc = [], 0.0
            for p in plain:
                acc += p[2]
                finish.append(acc * 1000.0)
            plain_d = {"problems_per_s": BATCH_N / t_all, "total_s": t_all,
                       "p50_ms": _percentile(finish, 0.5), "p99_ms": _percentile(finish, 0.99),
                       "how": "each problem alone through lsyn_create + lsyn_solve + lsyn_destroy, one after another "
                              "(time-to-formula = its finish time when all 256 arrive at once)"}
        steps_tr = [t for t in trace if t["lane"] == 0]
        large_tr = [t for t in trace if t["lane"] == 1]
        line = {
            "metric": "problems/sec", "value": value, "unit": "problems/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": BATCH_WORKLOAD, "problems": BATCH_N, "max_size": BATCH_MAX_SIZE,
                       "l2_flush": False, "inputs": "caches far larger than L2 (GBs per step)"},
            "p50_ms": _percentile(lat, 0.5), "p99_ms": _percentile(lat, 0.99),
            "statuses": {str(k): statuses.count(k) for k in sorted(set(statuses))},
            "plain_serial": plain_d, "same_answers_as_plain": same,
            "vs_plain": (value / plain_d["problems_per_s"]) if plain_d else None,
            "tuning": {k: getattr(tuned, k) for k, _ in tuned._fields_} if tuned else None,
            "defaults_problems_per_s": (BATCH_N * args.steps / (default_ms / 1000.0)) if default_ms else None,
            "tuning_gain": (default_ms / total_ms) if default_ms else None,
            "sched": stats,
            "trace_totals": {"batch_steps": len(steps_tr), "large_levels": len(large_tr),
                             "host_ms": sum(t["plan_ms"] + t["settle_ms"] for t in trace)},
            "roofline": None, "roofline_note": "the level kernels' roofline is reported by the default (mid) workload",
            "e2e": {"value": BATCH_N / e2e_s, "unit": "problems/s",
                    "h2d_bytes_per_step": sum(q.h2d_bytes for q in packed), "d2h_bytes_per_step": BATCH_N * 4096},
            "gpu_launches": None, "clocks": clocks.summary(),
        }
        print(json.dumps(line), flush=True)
    return 0


def _plain_fifo_live(L, packed, arrivals, order, max_size, cache):
    """The plain path as a serial FIFO server under the same arrivals, run for
    real: each problem starts when it has arrived and the previous one is
    done, and goes through lsyn_create + lsyn_solve + lsyn_destroy. Returns
    (latencies in ms, (status, size) per arrival, seconds until the last
    answer)."""
    import torch
    cfg = L.torch_config(cache_bytes=cache)
    lat, answers = [], []
    t0 = time.perf_counter()
    for ta, pi in zip(arrivals, order):
        d = t0 + ta - time.perf_counter()
        if d > 0:
            time.sleep(d)
        with L.Synthesizer(packed[pi], cfg) as s:
            st, res, f, _ = s.solve(max_size)
        torch.cuda.synchronize()
        lat.append((time.perf_counter() - t0 - ta) * 1000.0)
        answers.append((st, res.size if st == 0 else 0))
    return lat, answers, time.perf_counter() - t0


def _spread(xs):
    xs = [x for x in xs if x is not None]
    if not xs:
        return None
    return {"min": min(xs), "median": statistics.median(xs), "max": max(xs)}


def run_served(args):
    import torch
    world, rank, local = _dist()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    from paper_2504_18943_gb300 import build
    build.build()
    from paper_2504_18943_gb300 import lsyn as L
    from paper_2504_18943_gb300 import workloads as W
    packed = _batched_problems(L, W)
    plain = _plain_service_times(L, packed, BATCH_MAX_SIZE, BATCH_CACHE)
    cfg = L.make_config(cache_bytes=BATCH_CACHE, device=local)
    rates = [float(r) for r in args.rates.split(",")]
    out = []
    for rate in rates:
        runs = []
        for rep in range(args.repeats):
            # every repeat draws its own arrival times (seed = repeat)
            arrivals = W.poisson_arrivals(rep, rate, args.duration)
            order = [i % BATCH_N for i in range(len(arrivals))]
            torch.cuda.synchronize()
            torch.cuda.empty_cache()  # the server's pool takes its share of what is free now
            with L.Server(cfg) as sv:
                for q in packed[:8]:  # warm the pool and the launch paths
                    sv.wait(sv.submit(q, BATCH_MAX_SIZE))
                tickets = [None] * len(arrivals)
                t0 = time.perf_counter()
                for i, (ta, pi) in enumerate(zip(arrivals, order)):
                    d = t0 + ta - time.perf_counter()
                    if d > 0:
                        time.sleep(d)
                    tickets[i] = sv.submit(packed[pi], BATCH_MAX_SIZE)
                res = [sv.wait(t) for t in tickets]
                t_end = time.perf_counter()
                stats = sv.stats()
            lat = [r[1].ms for r in res]
            wrong = sum(1 for (st, r, f), pi in zip(res, order) if (st, r.size if st == 0 else 0) !=
                        (plain[pi][0], plain[pi][1] if plain[pi][0] == 0 else 0))
            # The plain path as one serial FIFO server, replayed: each arrival
            # waits for the previous problems, then takes its measured
            # one-problem time.
            free_at, plat = 0.0, []
            for ta, pi in zip(arrivals, order):
                start = max(ta, free_at)
                free_at = start + plain[pi][2]
                plat.append((free_at - ta) * 1000.0)
            run = {"repeat": rep, "submitted": len(arrivals), "problems_per_s": len(arrivals) / (t_end - t0),
                   "p50_ms": _percentile(lat, 0.5), "p99_ms": _percentile(lat, 0.99), "answers_differ": wrong,
                   "plain_replayed": {"problems_per_s": len(arrivals) / max(free_at, arrivals[-1]),
                                      "p50_ms": _percentile(plat, 0.5), "p99_ms": _percentile(plat, 0.99)},
                   "sched": {k: stats[k] for k in ("steps", "large_levels", "evictions", "redos", "pool_peak")}}
            if args.plain_live:
                torch.cuda.synchronize()
                plive, answers, t_last = _plain_fifo_live(L, packed, arrivals, order, BATCH_MAX_SIZE, BATCH_CACHE)
                torch.cuda.empty_cache()
                run["plain_live"] = {"problems_per_s": len(arrivals) / t_last, "p50_ms": _percentile(plive, 0.5),
                                     "p99_ms": _percentile(plive, 0.99),
                                     "answers_differ": sum(1 for a, (st, r, f) in zip(answers, res)
                                                           if a != (st, r.size if st == 0 else 0))}
            runs.append(run)
        summary = {"rate": rate, "repeats": args.repeats, "runs": runs,
                   "problems_per_s": _spread([r["problems_per_s"] for r in runs]),
                   "p50_ms": _spread([r["p50_ms"] for r in runs]), "p99_ms": _spread([r["p99_ms"] for r in runs]),
                   "answers_differ": sum(r["answers_differ"] for r in runs),
                   "plain_replayed": {k: _spread([r["plain_replayed"][k] for r in runs])
                                      for k in ("problems_per_s", "p50_ms", "p99_ms")}}
        if args.plain_live:
            summary["plain_live"] = {k: _spread([r["plain_live"][k] for r in runs])
                                     for k in ("problems_per_s", "p50_ms", "p99_ms")}
        out.append(summary)
    if rank == 0:
        top = out[-1]
        line = {
            "metric": "problems/sec, p50/p99 time-to-formula", "value": top["problems_per_s"]["median"],
            "unit": "problems/s", "n_gpus": world, "steps": len(rates) * args.repeats, "warmup": 8,
            "ms_per_step": 1000.0 * args.duration, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "served: open-loop Poisson arrivals (seeded per repeat) of the 256 batched "
                                   "problems in turn, max size 13, 8 GiB cap each", "rates": rates,
                       "duration_s": args.duration, "repeats": args.repeats},
            "per_rate": out,
            "plain_how": "replayed: a FIFO queue served by the one-problem path, each problem taking its measured "
                         "lsyn_create + lsyn_solve + lsyn_destroy time; live (with --plain-live): the same FIFO "
                         "run for real under the same arrivals",
            "roofline": None, "roofline_note": "the level kernels' roofline is reported by the default (mid) workload",
            "e2e": {"value": top["problems_per_s"]["median"], "unit": "problems/s",
                    "h2d_bytes_per_step": None, "d2h_bytes_per_step": None},
            "gpu_launches": None,
        }
        print(json.dumps(line), flush=True)
    return 0


def _kernel_sha() -> str:
    import hashlib
    h = hashlib.sha256()
    for name in ("lsyn_device.cuh", "lsyn_api.cu", "lsyn_internal.h"):
        with open(os.path.join(ROOT, "paper_2504_18943_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 30 solves for the mid workload, about half a second on the GPU, "
                         "so that the clock sampler sees it; 3 for the large workload, the reference arm and the "
                         "batched workload; 5 for the paper's example)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lsyn", choices=["lsyn", "reference"])
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--large-seed", type=int, default=0)
    ap.add_argument("--ref-levels", type=int, default=7,
                    help="reference arm: levels of the mid problem the oracle builds per step (on all host cores)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="mid", choices=["mid", "large", "e3", "batched", "served"],
                    help="mid (default): the one-problem headline; large: 16 KiB matrices, 150 GB cache; "
                         "e3: the paper's worked example; batched: 256 problems per step; "
                         "served: Poisson arrivals through the server")
    ap.add_argument("--autotune", action="store_true", help="batched: run the autotuner before timing")
    ap.add_argument("--no-plain", action="store_true", help="batched: skip the plain-path comparison")
    ap.add_argument("--rates", default="50,200,1000", help="served: arrival rates (problems/s)")
    ap.add_argument("--duration", type=float, default=60.0, help="served: seconds of arrivals per rate")
    ap.add_argument("--repeats", type=int, default=1, help="served: runs per rate (each with its own arrival seed)")
    ap.add_argument("--plain-live", action="store_true",
                    help="served: also run the plain path as a real FIFO server under the same arrivals")
    args = ap.parse_args()
    if args.steps is None:
        one = _one_problem_workloads()
        args.steps = one[args.workload]["steps"] if (args.impl == "lsyn" and args.workload in one) else 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "served":
        return run_served(args)
    return run_lsyn(args)


if __name__ == "__main__":
    sys.exit(main())
