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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "mid-scale plain solve: 5 props, 64+64 traces, len U[8,32], Bernoulli(0.5), hidden size 11, " \
           "128 x uint32 words (512 B) per CM, 64 GiB cache, until first solution (seed 2: minimal size 11)"
METRIC = "unique formulas/sec"
CACHE_BYTES = 64 << 30
MAX_SIZE = 16


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


def cpu_baseline(problem, max_level: int = 6):
    """The oracle, as it stands, on a bounded sample: levels 1..max_level of the
    same problem, single-threaded on a host core."""
    import oracle
    spec = oracle.Spec.from_problem(problem)
    t0 = time.perf_counter()
    run = spec.enumerate(max_level)
    dt = time.perf_counter() - t0
    uniq = sum(run.size(k) for k in range(1, max_level + 1))
    return {"value": uniq / dt, "unit": METRIC, "cores": 1, "kind": "oracle",
            "sample": f"levels 1..{max_level} of the timed problem ({uniq} unique formulas, {dt:.1f} s)",
            "seconds": dt}


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    from paper_2504_18943_gb300 import workloads as W
    import oracle
    problem = W.mid_problem(args.seed, oracle.labeller)
    for _ in range(args.warmup):
        cpu_baseline(problem, args.ref_levels)
    total_u, total_t = 0.0, 0.0
    for _ in range(args.steps):
        b = cpu_baseline(problem, args.ref_levels)
        total_u += b["value"] * b["seconds"]
        total_t += b["seconds"]
    value = total_u / total_t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "unique formulas/sec",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * total_t / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "seed": args.seed, "sample_levels": args.ref_levels},
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": 1, "kind": "oracle",
                             "sample": f"levels 1..{args.ref_levels} of the mid-scale problem per step"},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


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

    seed = args.seed  # every rank solves the same problem: replicas, fixed work per GPU
    problem = W.mid_problem(seed, L.labeller)
    packed = L.pack_problem(problem)
    stream = torch.cuda.current_stream(dev)
    cfg = L.torch_config(cache_bytes=CACHE_BYTES, timing=True, stream=stream, device=local)
    ctx = L.lsyn_create(packed, cfg)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)  # > L2 (129 MB)

    def step():
        L.lsyn_reset(ctx)
        return L.lsyn_solve(ctx, MAX_SIZE)

    for _ in range(max(args.warmup, 0)):
        st, res, formula, levels = step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()

    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    uniques, launches, all_levels = 0, 0, []
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

    # End to end through the public API from pinned host buffers: create
    # (host->device copy of the traces), solve, read the formula back, destroy.
    pinned_atoms = torch.from_numpy(packed.atom_words.view(np.int32)).pin_memory()
    pinned_len = torch.from_numpy(packed.lengths).pin_memory()
    host_problem = L.PackedProblem(packed.n_props, packed.n_pos, packed.n_neg, packed.word_bits,
                                   pinned_len.numpy(), pinned_atoms.numpy().view(packed.word_dtype))
    e2e_uniques, e2e_ms = 0, 0.0
    e2e_steps = max(1, min(args.steps, 5))
    for i in range(e2e_steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c2 = L.lsyn_create(host_problem, L.torch_config(cache_bytes=CACHE_BYTES, stream=stream, device=local))
        st2, r2, f2, _ = L.lsyn_solve(c2, MAX_SIZE)
        L.lsyn_destroy(c2)
        dt = (time.perf_counter() - t0) * 1000.0
        if i > 0:  # the first call warms the allocator cache
            e2e_uniques += r2.unique
            e2e_ms += dt
    e2e_ms = _reduce_max(e2e_ms, world, dev)
    e2e_total = _reduce_sum(float(e2e_uniques), world, dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle  # the CPU-baseline leg only
        cpu = cpu_baseline(problem, args.ref_levels)
        cpu.pop("seconds", None)

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
            tj = json.load(f).get(dom, {})
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
                  "unique_per_s": round(lv.unique / (max(lv.ms, 1e-6) / 1e3), 1)} for lv in all_levels]
    if rank == 0:
        st, size, formula = results[-1]
        line = {
            "metric": METRIC, "value": value, "unit": "unique formulas/sec", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": max_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "seed": args.seed, "min_size": size, "l2_flush": True,
                       "parallelism": f"replicas{world}" if world > 1 else "single",
                       "formula": formula, "status": st},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak if peak else None, "traffic": traffic,
                         "kernel": {"unary": "k_unary_c (not/X/F/G level kernel)",
                                    "binary": "k_binary_c (and/or/U level kernel)"}[dom],
                         "peak_source": peak_kind, "alg_bytes_per_launch": alg_per_launch,
                         "launches": klaunch[dom],
                         "other": {n: {"achieved": (kbytes[n] / 1e9) / (kms[n] / 1e3) if kms[n] else None,
                                       "ms": kms[n]} for n in kms if n != dom}},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_total / (e2e_ms / 1000.0) if e2e_ms > 0 else None, "unit": "unique formulas/sec",
                    "h2d_bytes_per_step": packed.h2d_bytes, "d2h_bytes_per_step": 1 << 16,
                    "steps": e2e_steps},
            "gpu_launches": launches,
            "clocks": clocks.summary(),
            "levels": per_level,
        }
        print(json.dumps(line))
    L.lsyn_destroy(ctx)
    if world > 1:
        torch.distributed.destroy_process_group()
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
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lsyn", choices=["lsyn", "reference"])
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--ref-levels", type=int, default=7)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_lsyn(args)


if __name__ == "__main__":
    sys.exit(main())
