#!/usr/bin/env python3
"""Benchmark: spin-flip evaluations/s and local minima/s of the GPU local search.

One step = one ising_local_search call over the whole workload (every
instance, every replica, every restart) with the instances resident on the
GPU.  Workloads (synthetic, seeded; see workloads/):
  c1  16x16 periodic +/-J lattice, 64 replicas, 10 restarts
  c2  32^3 periodic +/-J lattice, h in {-1,0,1}, 1024 replicas, <= 100 sweeps
      per descent, 10 restarts (multi-spin coded)            [default]
  c3  4096 K4,4 cell grids (side 4..16), Gaussian J, h, one 3-spin coupling
      per cell, 32 replicas, FP32 fields with FP64 refresh every 16 sweeps
  c4  dense SK, N = 4096, 4096 replicas, sequential schedule on tensor cores
  c5  100^3 periodic Gaussian lattice, 16 replicas, 1000-sweep budget with
      restarts, FP32 fields refreshed in FP64 every 16 sweeps
  c5i the same lattice with +/-1 couplings
Prints one JSON line (rank 0).  --impl reference times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "spin-flip evals/s, minima/s on 1 GB300: batched/mixed vs plain at equal energy"
UNIT = "flip_evals/s"


def make_workload(name: str, instances: int = 0, sk_n: int = 0):
    """(instances, replicas, search kwargs, description).  `instances` (c3) and
    `sk_n` (c4) shrink the workload for profiling captures."""
    if name == "c1":
        inst = W.lattice((16, 16), periodic=True, couplings="pm1", seed=W.config_seed(0))
        return [inst], 64, dict(max_sweeps=1000, restarts=10), "16x16 periodic +/-J lattice, 64 replicas, 10 restarts"
    if name == "c2":
        inst = W.lattice((32, 32, 32), periodic=True, couplings="pm1", fields="pm1_0", seed=W.config_seed(1))
        return [inst], 1024, dict(max_sweeps=100, restarts=10), \
            "32^3 periodic +/-J lattice, h in {-1,0,1}, 1024 replicas, <=100 sweeps/descent, 10 restarts"
    if name == "c3":
        insts = W.chimera_batch(instances or 4096, 4, 16, seed=W.config_seed(2))
        return insts, 32, dict(max_sweeps=1000, restarts=1, refresh_every=16), \
            "4096 K4,4 cell grids (side 4..16), Gaussian J,h + one 3-spin coupling per cell, 32 replicas"
    if name == "c4":
        inst = W.sk(sk_n or 4096, seed=W.config_seed(3))
        return [inst], 4096, dict(max_sweeps=1000, restarts=1, refresh_every=16, schedule=1), \
            "dense SK N=4096, 4096 replicas, sequential schedule"
    if name == "c5":
        inst = W.lattice((100, 100, 100), periodic=True, couplings="gauss", seed=W.config_seed(4))
        return [inst], 16, dict(max_sweeps=1000, restarts=1 << 30, sweep_budget=1000, refresh_every=16), \
            "100^3 periodic Gaussian lattice, 16 replicas, 1000-sweep budget with restarts"
    if name == "c5i":
        inst = W.lattice((100, 100, 100), periodic=True, couplings="pm1", seed=W.config_seed(4))
        return [inst], 16, dict(max_sweeps=1000, restarts=1 << 30, sweep_budget=1000), \
            "100^3 periodic +/-J lattice, 16 replicas, 1000-sweep budget with restarts"
    if name == "l50":
        # the size of the paper's 50x50 timing (ln^2 n random starts, Sec. V), for --method fm
        inst = W.lattice((50, 50), periodic=True, couplings="gauss", seed=W.config_seed(6))
        return [inst], 61, dict(max_sweeps=1000, restarts=1), \
            "50x50 periodic Gaussian lattice, 61 = round(ln^2 2500) random starts"
    raise ValueError(name)


def seeds_for(name: str, n_inst: int, rank: int):
    base = W.config_seed(7 if name == "l50" else int(name[1]) - 1) + 1000003 * rank
    return [W.replica_seed(W.splitmix64(base + b)) for b in range(n_inst)]


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        # raw samples (summarised into the JSON line); ISING_BENCH_CLOCKS_DIR keeps them
        self.path = os.path.join(os.environ.get("ISING_BENCH_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"clocks_{os.getpid()}.csv")
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- peaks
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), d.get("bf16_tflops_sustained", 1700.0), "measured"
    return 6800.0, 1900.0, 1700.0, "fallback"


# ----------------------------------------------------------------------------- CPU oracle
def oracle_sample(name, insts, R, kw, budget_s=10.0):
    """Time the CPU oracle (single thread) on a bounded sample of the workload."""
    import oracle
    oracle.build()
    seeds = seeds_for(name, len(insts), 0)
    kw2 = {k: v for k, v in kw.items() if k in ("max_sweeps", "restarts", "sweep_budget", "refresh_every",
                                              "schedule")}
    evals = minima = 0
    t0 = time.perf_counter()
    done_units = []
    b = 0
    r_per = 1
    oinsts = {}
    while time.perf_counter() - t0 < budget_s:
        inst = insts[b % len(insts)]
        if b not in oinsts:
            oinsts[b] = oracle.OracleInstance(inst)
        _, _, _, st = oracle.descent(oinsts[b], seeds[b % len(insts)], b % len(insts), r_per, **kw2)
        evals += st["flip_evals"]
        minima += st["minima"]
        done_units.append((b % len(insts), r_per))
        b += 1
        if b >= len(insts):
            b = 0
            r_per += 1
    dt = time.perf_counter() - t0
    desc = (f"{len(done_units)} oracle calls (instance, first k replicas) of this workload, "
            f"{evals} evaluations, {dt:.1f} s")
    return evals / dt, minima / dt, desc, dt


# ----------------------------------------------------------------------------- multi-rank
def job_totals(t_local, evals_local, minima_local, dist=None, device=None):
    """Whole-job figures: the slowest rank's time, the work of all ranks summed.

    Replicas are independent, so each rank runs its own replicas (its own seeds)
    with no data-path collective; only these two reductions cross ranks.
    """
    if dist is None:
        return t_local, evals_local, minima_local
    import torch
    t = torch.tensor([t_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    w = torch.tensor([float(evals_local), float(minima_local)], dtype=torch.float64, device=device)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t.item()), float(w[0].item()), float(w[1].item())


# ----------------------------------------------------------------------------- main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="c2")
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--kernel", default="auto")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    # smaller variants of a workload, for profiler captures
    ap.add_argument("--replicas", type=int, default=0)
    ap.add_argument("--restarts", type=int, default=0)
    ap.add_argument("--sweep-budget", type=int, default=-1)
    ap.add_argument("--instances", type=int, default=0)
    ap.add_argument("--sk-n", type=int, default=0)
    ap.add_argument("--method", default="descent", choices=["descent", "fm"],
                    help="fm: the pass-based search with hill climbing (ising_fm_search) on the workload")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    insts, R, kw, desc = make_workload(args.workload, args.instances, args.sk_n)
    if args.replicas:
        R = args.replicas
    if args.restarts:
        kw["restarts"] = args.restarts
    if args.sweep_budget >= 0:
        kw["sweep_budget"] = args.sweep_budget
    if args.replicas or args.restarts or args.sweep_budget >= 0 or args.instances or args.sk_n:
        desc += f" [reduced: replicas={R}, {kw}]"

    if args.impl == "reference" and args.method == "fm":
        if rank == 0:
            run_fm_reference(args, insts, R, kw, desc)
        return
    if args.impl == "reference":
        if rank != 0:
            return
        ev, mn, sample, dt = oracle_sample(args.workload, insts, R, kw, budget_s=args.cpu_seconds)
        steps_t = []
        for _ in range(args.warmup + args.steps):
            pass
        line = {"metric": METRIC, "value": ev, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "i8->int64" if insts[0].dtype == "i8" else "f32/f64",
                "data": "synthetic", "minima_per_s": mn,
                "config": {"workload": args.workload, "description": desc, "replicas": R, **{k: v for k, v in kw.items()}},
                "cpu_baseline": {"value": ev, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
                "e2e": {"value": ev, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    if args.method == "fm":
        if rank == 0:
            run_fm(args, insts, R, kw, desc)
        return

    import torch
    import paper_0912_3912_gb300 as isg
    from paper_0912_3912_gb300 import build as B
    if rank == 0 or not os.path.exists(isg.LIB_PATH):
        B.build()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank if world > 1 else 0)
    torch.cuda.set_device(dev)

    kernel = {"auto": 0, "tile": 1, "msc": 2, "sweep": 3, "dense": 4, "plain": 5}[args.kernel]
    seeds = seeds_for(args.workload, len(insts), rank)
    h = isg.Handle(insts)
    chosen = h.plan_kernel(R, kernel=kernel, **{k: v for k, v in kw.items() if k in ("schedule",)})
    stream = torch.cuda.current_stream()
    total_spins = h.total_spins
    spins = torch.empty(R * total_spins, dtype=torch.int8, device=dev)
    E = torch.empty((len(insts), R), dtype=torch.float64, device=dev)
    minima = torch.empty((len(insts), R), dtype=torch.int32, device=dev)
    out = (spins, E, None, minima)
    l2_flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def step(stats=False):
        return h.local_search(seeds, R, kernel=kernel, stats=stats, out=out, **kw)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ref = step(stats=True)        # work counters of one step (identical every step)
    st = ref.stats
    torch.cuda.synchronize()

    if dist is not None:
        dist.barrier()
    clocks = ClockSampler(dev.index)
    h.set_timing(True)            # per-kernel CUDA events inside the library, over the timed steps
    torch.cuda.synchronize()
    ev_pairs = []
    for _ in range(args.steps):
        l2_flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        ev_pairs.append((a, b))
    torch.cuda.synchronize()
    clk = clocks.stop()
    ktimes = h.kernel_times()
    h.set_timing(False)
    ms = [a.elapsed_time(b) for a, b in ev_pairs]
    t_total, evals_job, minima_job = job_totals(sum(ms) / 1e3, st["flip_evals"] * args.steps,
                                                st["minima"] * args.steps, dist, dev)
    value = evals_job / t_total

    # end to end: host seeds in, host results out (pinned), through the C ABI
    h_spins = torch.empty(R * total_spins, dtype=torch.int8, pin_memory=True)
    h_E = torch.empty((len(insts), R), dtype=torch.float64, pin_memory=True)
    e2e_ms = []
    for _ in range(args.steps):
        l2_flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        h_spins.copy_(spins, non_blocking=True)
        h_E.copy_(E, non_blocking=True)
        b.record(stream)
        b.synchronize()
        e2e_ms.append(a.elapsed_time(b))
    e2e_value = st["flip_evals"] * len(e2e_ms) / (sum(e2e_ms) / 1e3)

    # roofline of the dominant kernel
    hbm, bf16, bf16s, peak_src = measured_peaks()
    n_launch_per_step = st.get("launches", 1)
    eff_kernel = chosen
    if chosen == isg.KERNEL_MSC or (chosen == isg.KERNEL_SWEEP and insts[0].dtype == "i8"):
        eff_kernel = 2 if chosen == isg.KERNEL_MSC else 3
    roof = roofline(args.workload, eff_kernel, insts, R, st, t_total / args.steps, clk, hbm, bf16s, peak_src,
                    ktimes, args.steps)
    st = {k: v for k, v in st.items() if k != "launches"}

    # equal-energy comparison with the plain comparator kernel
    plain = None
    if not args.no_plain and chosen != isg.KERNEL_PLAIN:
        comparator = isg.KERNEL_PLAIN
        if chosen == isg.KERNEL_DENSE_TC:
            # dense: the straightforward blocked version with library GEMMs
            os.environ["ISING_DENSE_CUBLAS"] = "1"
            comparator = isg.KERNEL_DENSE_TC
        try:
            pr = h.local_search(seeds, R, kernel=comparator, stats=True, **kw)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            pr = h.local_search(seeds, R, kernel=comparator, stats=True, **kw)
            b.record(stream)
            torch.cuda.synchronize()
            pms = a.elapsed_time(b)
            if insts[0].dtype == "i8":
                same = bool(torch.equal(pr.energy, E))  # integer couplings: identical results
            else:
                # float couplings: the comparator's rounding differs where its field
                # arithmetic does; report how the energies reached compare
                m1, m2 = float(E.mean().item()), float(pr.energy.mean().item())
                same = {"max_abs_diff": float((pr.energy - E).abs().max().item()), "mean_energy": m1,
                        "comparator_mean_energy": m2, "rel_mean_diff": abs(m1 - m2) / max(abs(m2), 1e-300),
                        "identical_replicas": float((pr.energy == E).double().mean().item())}
            plain = {"kind": "cublas_blocked" if chosen == isg.KERNEL_DENSE_TC else "plain",
                     "value": pr.stats["flip_evals"] / (pms / 1e3), "unit": UNIT, "ms_per_step": pms,
                     "energy_match": same, "speedup": value / (pr.stats["flip_evals"] / (pms / 1e3))}
        except Exception as ex:  # comparator not available for this workload
            plain = {"unavailable": str(ex)}
        finally:
            os.environ.pop("ISING_DENSE_CUBLAS", None)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ev, mn, sample, dt = oracle_sample(args.workload, insts, R, kw, budget_s=args.cpu_seconds)
        cpu = {"value": ev, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
               "minima_per_s": mn}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_total * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "bit-packed i1/int32" if insts[0].dtype == "i8" else "f32 fields, f64 refresh/energy",
            "data": "synthetic (seeded generators; the paper's instances are not available)",
            "minima_per_s": minima_job / t_total,
            "config": {"workload": args.workload, "description": desc, "replicas": R,
                       "instances": len(insts), "spins": total_spins,
                       "kernel": isg.KERNEL_NAMES[chosen], "l2": "flushed (512 MB write) before every timed step",
                       **{k: v for k, v in kw.items()}},
            "work_per_step": st,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * len(insts),
                    "d2h_bytes_per_step": R * total_spins + 8 * R * len(insts)},
            "gpu_launches": int(n_launch_per_step) * args.steps,
            "clocks": clk,
            "roofline": roof,
            "plain": plain,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    h.close()
    if dist is not None:
        dist.destroy_process_group()


def run_fm(args, insts, R, kw, desc):
    """Bench line of the pass-based search (one process): moves applied per
    second (every spin moves once per pass), device-timed over the steps, plus
    end to end with host copies and the oracle's heap implementation on a
    bounded sample of the same starts."""
    import torch
    import paper_0912_3912_gb300 as isg
    from paper_0912_3912_gb300 import build as B
    B.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    seeds = seeds_for(args.workload, len(insts), 0)
    restarts = int(kw.get("restarts", 1))
    h = isg.Handle(insts)
    stream = torch.cuda.current_stream()
    l2_flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        h.fm_search(seeds, R, restarts=restarts, stats=False)
    torch.cuda.synchronize()
    _, _, _, st = h.fm_search(seeds, R, restarts=restarts)
    clocks = ClockSampler(dev.index)
    h.set_timing(True)
    torch.cuda.synchronize()
    evs = []
    for _ in range(args.steps):
        l2_flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        h.fm_search(seeds, R, restarts=restarts, stats=False)
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    clk = clocks.stop()
    ktimes = h.kernel_times()
    h.set_timing(False)
    t = sum(a.elapsed_time(b) for a, b in evs) / 1e3
    value = st["flips"] * args.steps / t
    # end to end: results copied to pinned host buffers inside the timed region
    h_sp = torch.empty(R * h.total_spins, dtype=torch.int8, pin_memory=True)
    h_E = torch.empty((len(insts), R), dtype=torch.float64, pin_memory=True)
    e2e = []
    for _ in range(args.steps):
        l2_flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sp, E, _, _ = h.fm_search(seeds, R, restarts=restarts, stats=False)
        h_sp.copy_(sp, non_blocking=True)
        h_E.copy_(E, non_blocking=True)
        b.record(stream)
        b.synchronize()
        e2e.append(a.elapsed_time(b))
    e2e_value = st["flips"] * len(e2e) / (sum(e2e) / 1e3)
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        moves, n_runs, t0 = 0, 0, time.time()
        for b_, inst in enumerate(insts):
            for r in range(R):
                for k in range(restarts):
                    _, _, p = oracle.fm_search(inst, oracle.random_start(inst.n, seeds[b_], b_, r, k))
                    moves += p * inst.n
                    n_runs += 1
                    if time.time() - t0 > args.cpu_seconds:
                        break
                if time.time() - t0 > args.cpu_seconds:
                    break
            if time.time() - t0 > args.cpu_seconds:
                break
        dt = time.time() - t0
        cpu = {"value": moves / dt, "unit": "moves/s", "cores": 1, "kind": "oracle",
               "sample": f"{n_runs} oracle searches (first starts of this workload), {moves} moves, {dt:.1f} s"}
    line = {"metric": "pass-based search (Sec. IV, Fig. 3) moves/s on 1 GB300", "value": value, "unit": "moves/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64 (FP64-exact instances) or f64",
            "data": "synthetic (seeded generators)",
            "config": {"workload": args.workload, "method": "fm", "description": desc, "replicas": R,
                       "restarts": restarts, "instances": len(insts),
                       "l2": "flushed (512 MB write) before every timed step"},
            "work_per_step": {k: v for k, v in st.items() if k != "launches"},
            "e2e": {"value": e2e_value, "unit": "moves/s", "h2d_bytes_per_step": 8 * len(insts),
                    "d2h_bytes_per_step": int(h_sp.numel() + 8 * h_E.numel())},
            "gpu_launches": st.get("launches", 1) * args.steps, "clocks": clk,
            "roofline": None,
            "roofline_note": "a warp per search, one dependent chain per move (block-maximum reductions, "
                             "neighbour field updates): latency-bound, neither HBM nor an ALU pipe applies; "
                             "kernel ms per step: " + json.dumps({k: v[0] / args.steps for k, v in ktimes.items()}),
            "cpu_baseline": cpu}
    print(json.dumps(line))
    h.close()


def run_fm_reference(args, insts, R, kw, desc):
    """The reference arm of --method fm: the oracle's pass-based search (heap,
    one host core) on the first starts of the workload, each step a bounded
    sample (about --cpu-seconds / steps of work), moves applied per second."""
    import oracle
    oracle.build()
    seeds = seeds_for(args.workload, len(insts), 0)
    restarts = int(kw.get("restarts", 1))
    budget = max(args.cpu_seconds / max(args.steps + args.warmup, 1), 0.05)
    units = [(b, r, k) for b in range(len(insts)) for r in range(R) for k in range(restarts)]
    pos, rates, moves_all, runs_all, t_all = 0, [], 0, 0, 0.0
    for step in range(args.warmup + args.steps):
        moves, runs, t0 = 0, 0, time.perf_counter()
        while time.perf_counter() - t0 < budget:
            b, r, k = units[pos % len(units)]
            pos += 1
            _, _, p = oracle.fm_search(insts[b], oracle.random_start(insts[b].n, seeds[b], b, r, k))
            moves += p * insts[b].n
            runs += 1
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            rates.append(moves / dt)
            moves_all, runs_all, t_all = moves_all + moves, runs_all + runs, t_all + dt
    value = moves_all / t_all
    sample = f"{runs_all} oracle searches (first starts of this workload, in order), {moves_all} moves, {t_all:.1f} s"
    line = {"metric": "pass-based search (Sec. IV, Fig. 3) moves/s on 1 GB300", "value": value, "unit": "moves/s",
            "impl": "reference", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64 (oracle)",
            "data": "synthetic (seeded generators)",
            "config": {"workload": args.workload, "method": "fm", "description": desc, "replicas": R,
                       "restarts": restarts, "instances": len(insts)},
            "cpu_baseline": {"value": value, "unit": "moves/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "moves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def ncu_traffic(workload, kernel):
    """DRAM bytes per launch of `kernel` for `workload` from the committed ncu
    summary (read + write), or None when it holds no line for them."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "profiles", "dram_traffic.txt")
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    for line in lines:
        f = line.split()
        if len(f) >= 4 and f[0] == workload and f[1] == kernel and f[2].isdigit() and f[3].isdigit():
            return int(f[2]) + int(f[3])
    return None


def roofline(name, kernel, insts, R, st, step_s, clk, hbm, bf16s, src, ktimes=None, steps=1):
    """Roofline of the step's main kernel.  The algorithmic work per unit is the
    method's own (not the kernel's instruction count).  The time is that
    kernel's device time over the timed steps, from the CUDA events the library
    records around its launches (ising_set_timing); where none were recorded,
    the whole step's time (a lower bound for the kernel alone)."""
    out = _roofline(name, kernel, insts, R, st, step_s, clk, hbm, bf16s, src)
    kname = out.get("kernel")
    if kname == "tile_kernel" and ktimes and kname not in ktimes and "msc_cluster_kernel" in ktimes:
        kname = out["kernel"] = "msc_cluster_kernel"  # the lattice tiles split over CTA clusters
    if ktimes and kname in ktimes and ktimes[kname][0] > 0:
        k_s = ktimes[kname][0] / 1e3 / steps
        scale = step_s / k_s
        out["achieved"] *= scale
        out["frac"] *= scale
        out["time_basis"] = f"{kname}: CUDA events around its launches, {ktimes[kname][1] // max(1, steps)} per step"
        out["kernel_ms_per_step"] = k_s * 1e3
        out["kernel_share_of_step"] = k_s / step_s
    else:
        out["time_basis"] = "whole step (CUDA events)"
    if ktimes:
        out["kernels_ms_per_step"] = {k: v[0] / steps for k, v in ktimes.items()}
    tr = ncu_traffic(name, out.get("kernel"))
    if tr is not None:
        out["traffic"] = tr
        out["traffic_unit"] = "DRAM bytes per launch (ncu, committed summary)"
    return out


def _roofline(name, kernel, insts, R, st, step_s, clk, hbm, bf16s, src):
    sm_count = 152
    mhz = (clk or {}).get("sm_mhz") or 2070.0
    inst = insts[0]
    deg = sum(i.nnz for i in insts) / max(1, sum(i.n for i in insts)) if inst.row_ptr is not None else inst.n - 1
    lattice = inst.meta.get("kind") == "lattice" and inst.meta.get("periodic") and len(set(inst.meta["dims"])) == 1
    msc = inst.dtype == "i8" and inst.hyper_ptr is None and np.all(np.abs(inst.J) == 1) and (
        inst.h is None or np.all(np.abs(inst.h) <= 1))
    if msc and kernel in (2, 3):
        # integer/logic lane-operations per (spin, replica word): per bond one
        # unsatisfied-mask op, one for the field, about one adder op per input,
        # the flip mask and the word update: 2 deg + 4
        lanes = 32 if kernel == 2 else (32 if R > 16 else (16 if R > 8 else 8))
        ops = 2 * deg + 4
        words = st["flip_evals"] / lanes
        achieved = words * ops / step_s / 1e12
        peak = sm_count * 128 * mhz * 1e6 / 1e12
        kname = "sweep_chunk" if kernel == 3 else "tile_kernel"
        return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tlane-ops/s", "frac": achieved / peak,
                "traffic": None, "kernel": kname, "ops_per_word": ops, "replicas_per_word": lanes,
                "peak_source": f"derived: {sm_count} SMs x 128 integer lanes x {mhz:.0f} MHz (median SM clock under load)"}
    if kernel == 4:
        # Tensor-core work actually done: each descent's first sweeps (the
        # library's split, 3 unless overridden) and one export pass, 4 n^2 flops
        # per replica and pass (BF16 hi and lo GEMMs).  Later sweeps run as
        # incremental updates on CUDA cores and are not counted here.
        n = inst.n
        sweeps_a = int(os.environ.get("ISING_DENSE_TC_SWEEPS", "3"))
        flops = st["descents"] * (min(sweeps_a, st["sweeps"] / max(1, st["descents"])) + 1) * 4.0 * n * n
        achieved = flops / step_s / 1e12
        return {"bound": "tensor", "achieved": achieved, "peak": bf16s, "unit": "TFLOP/s", "frac": achieved / bf16s,
                "traffic": None, "kernel": "dense_tc_kernel", "flops_per_replica_pass": 4.0 * n * n,
                "tensor_passes_per_descent": sweeps_a + 1,
                "peak_source": f"{src} bf16 sustained (MEASURED_PEAKS.json)"}
    # incremental method in HBM terms: per visit a 4-byte field read and 1/8 byte of
    # spin; per accepted flip deg x (8 bytes coupling + index, 8 bytes field update)
    byts = st["flip_evals"] * 4.125 + st["flips"] * deg * 16.0
    achieved = byts / step_s / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": None, "kernel": "sweep_chunk" if kernel == 3 else "tile_kernel", "bytes_per_step": byts,
            "peak_source": f"{src} copy bandwidth (MEASURED_PEAKS.json)"}


if __name__ == "__main__":
    main()
