#!/usr/bin/env python3
"""Benchmark: spin-flip evaluations/s and local minima/s of the GPU local search.

One step = one ising_local_search call over a whole workload (every instance,
every replica, every restart) with the instances resident on the GPU.
Workloads (synthetic, seeded; see workloads/):
  c1  16x16 periodic +/-J lattice, 64 replicas, 10 restarts
  c2  32^3 periodic +/-J lattice, h in {-1,0,1}, 1024 replicas, <= 100 sweeps
      per descent, 10 restarts (multi-spin coded)
  c3  4096 K4,4 cell grids (side 4..16), Gaussian J, h, one 3-spin coupling
      per cell, 32 replicas, FP32 fields with FP64 refresh every 16 sweeps
  c4  dense SK, N = 4096, 4096 replicas, sequential schedule on tensor cores
  c5  100^3 periodic Gaussian lattice (10^6 spins), 16 replicas, 1000-sweep
      budget with restarts, FP32 fields refreshed in FP64 every 16 sweeps
      [headline: the largest single-GPU workload, bound by HBM]
  c5i the same lattice with +/-1 couplings

Default run: the headline workload timed for exactly --steps steps, then every
other workload as a sub-record under "per_workload" (each timed for at least
--min-seconds), one JSON line on rank 0.  --impl reference times the CPU
oracle on the headline workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "spin-flip evals/s, minima/s on 1 GB300: batched/mixed vs plain at equal energy"
UNIT = "flip_evals/s"
HEADLINE = "c5"
ALL_WORKLOADS = ("c1", "c2", "c3", "c4", "c5", "c5i")
DENSE_TENSOR_SWEEPS = 3   # the library's default split of a dense descent (tensor-core sweeps first)


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
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons while a
    timed region runs; start() returns once the first sample has arrived, so
    that the samples cover the region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.path = os.path.join(os.environ.get("ISING_BENCH_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"clocks_{os.getpid()}_{id(self)}.csv")
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        t0 = time.time()
        while time.time() - t0 < 3.0:
            self.fh.flush()
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.02)
        self.first_lines = self._count()

    def _count(self):
        try:
            with open(self.path) as f:
                return sum(1 for _ in f)
        except OSError:
            return 0

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


# ----------------------------------------------------------------------------- peaks
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), d.get("bf16_tflops_sustained", 1700.0), "measured"
    return 6800.0, 1900.0, 1700.0, "fallback"


# ----------------------------------------------------------------------------- CPU oracle
def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def oracle_units(name, insts, R, kw):
    """The CPU sample's work units and the oracle parameters they run with.

    A unit is (instance, first replica, replica count); units go instance by
    instance, replica by replica, in the workload's own order.  The 100^3
    lattices run only the first 40 sweeps of each replica's 1000-sweep budget
    (a full budget is about 9 s of one core per replica)."""
    okw = {k: v for k, v in kw.items() if k in ("max_sweeps", "restarts", "sweep_budget", "refresh_every",
                                                "schedule")}
    note = "the workload's own parameters"
    if name in ("c5", "c5i"):
        okw["sweep_budget"] = 40
        note = "the first 40 sweeps of each replica's 1000-sweep budget"
    per = 8 if (max(i.n for i in insts) <= 4096 and R >= 8 and name != "c4") else 1
    units = [(b, r0, min(per, R - r0)) for b in range(len(insts)) for r0 in range(0, R, per)]
    return units, okw, note


def oracle_sample(name, insts, R, kw, seconds, threads, seeds=None, start=0):
    """Time the CPU oracle on a bounded sample of the workload: `threads` host
    threads take units in order from a shared counter until `seconds` have
    passed (units in flight finish).  The oracle's C calls release the GIL, so
    the threads run in parallel; the oracle itself is unchanged.  Returns a
    dict with rates, the wall time and a description of the sample."""
    import oracle
    oracle.build()
    if seeds is None:
        seeds = seeds_for(name, len(insts), 0)
    units, okw, note = oracle_units(name, insts, R, kw)
    lock = threading.Lock()
    cache = {}
    state = {"next": start, "evals": 0, "flips": 0, "minima": 0, "units": 0, "replicas": 0}
    t0 = time.perf_counter()
    deadline = t0 + seconds

    def oinst(b):
        with lock:
            o = cache.get(b)
        if o is None:
            o = oracle.OracleInstance(insts[b])
            with lock:
                cache[b] = o
        return o

    def worker():
        while True:
            with lock:
                if time.perf_counter() >= deadline:
                    return
                k = state["next"]
                state["next"] += 1
            b, r0, cnt = units[k % len(units)]
            _, _, _, st = oracle.descent(oinst(b), seeds[b], b, cnt, first_replica=r0, **okw)
            with lock:
                state["evals"] += st["flip_evals"]
                state["flips"] += st["flips"]
                state["minima"] += st["minima"]
                state["units"] += 1
                state["replicas"] += cnt

    ths = [threading.Thread(target=worker) for _ in range(threads)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    dt = time.perf_counter() - t0
    desc = (f"{state['replicas']} replica searches of this workload ({note}; units of "
            f"(instance, replica range) taken in order by {threads} host thread(s)), "
            f"{state['evals']} evaluations in {dt:.2f} s")
    return {"value": state["evals"] / dt, "minima_per_s": state["minima"] / dt, "wall_s": dt,
            "evals": state["evals"], "threads": threads, "sample": desc, "next": state["next"]}


def cpu_baseline(name, insts, R, kw, seconds):
    """The oracle on one host thread and on every host core (half the time each)."""
    cores = os.cpu_count() or 1
    one = oracle_sample(name, insts, R, kw, seconds / 2, 1)
    allc = oracle_sample(name, insts, R, kw, seconds / 2, cores)
    return {"value": allc["value"], "unit": UNIT, "cores": cores, "kind": "oracle", "sample": allc["sample"],
            "minima_per_s": allc["minima_per_s"], "cpu_model": cpu_model(), "nproc": cores,
            "single_thread": {"value": one["value"], "unit": UNIT, "cores": 1, "sample": one["sample"],
                              "minima_per_s": one["minima_per_s"]}}


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


# ----------------------------------------------------------------------------- one workload on the GPU
def gpu_record(name, args, dev, rank=0, dist=None, steps=None, min_seconds=0.0, plain=True, cpu_seconds=0.0):
    """Measure one workload: `steps` timed steps (at least `min_seconds` of
    device time when steps is None), end to end with host copies, the
    roofline of its main kernel, the plain comparator at equal energy and the
    CPU oracle.  Returns (record dict, per-step work counters)."""
    import torch
    import paper_0912_3912_gb300 as isg

    insts, R, kw, desc = make_workload(name, args.instances if name == args.workload else 0,
                                       args.sk_n if name == args.workload else 0)
    if name == args.workload:
        if args.replicas:
            R = args.replicas
        if args.restarts:
            kw["restarts"] = args.restarts
        if args.sweep_budget >= 0:
            kw["sweep_budget"] = args.sweep_budget
        if args.replicas or args.restarts or args.sweep_budget >= 0 or args.instances or args.sk_n:
            desc += f" [reduced: replicas={R}, {kw}]"
    kernel = {"auto": 0, "tile": 1, "msc": 2, "sweep": 3, "dense": 4, "plain": 5}[args.kernel]
    seeds = seeds_for(name, len(insts), rank)
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

    wms = []
    for _ in range(args.warmup):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        wms.append((a, b))
    torch.cuda.synchronize()
    ref = step(stats=True)        # work counters of one step (identical every step)
    st = ref.stats
    torch.cuda.synchronize()
    if steps is None:
        est = min(a.elapsed_time(b) for a, b in wms) if wms else 1.0
        steps = max(args.steps, int(math.ceil(min_seconds * 1e3 / max(est, 1e-3))))

    if dist is not None:
        dist.barrier()
    clocks = ClockSampler(dev.index)
    h.set_timing(True)            # per-kernel CUDA events inside the library, over the timed steps
    torch.cuda.synchronize()
    ev_pairs = []
    for _ in range(steps):
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
    t_total, evals_job, minima_job = job_totals(sum(ms) / 1e3, st["flip_evals"] * steps,
                                                st["minima"] * steps, dist, dev)
    value = evals_job / t_total

    # end to end: host seeds in, host results out (pinned), through the C ABI
    h_spins = torch.empty(R * total_spins, dtype=torch.int8, pin_memory=True)
    h_E = torch.empty((len(insts), R), dtype=torch.float64, pin_memory=True)
    e2e_ms = []
    for _ in range(steps):
        l2_flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        h_spins.copy_(spins, non_blocking=True)
        h_E.copy_(E, non_blocking=True)
        b.record(stream)
        b.synchronize()
        e2e_ms.append(a.elapsed_time(b))
    t_e2e, ev_e2e, _ = job_totals(sum(e2e_ms) / 1e3, st["flip_evals"] * steps, 0, dist, dev)
    e2e_value = ev_e2e / t_e2e

    hbm, bf16, bf16s, peak_src = measured_peaks()
    n_launch_per_step = st.get("launches", 1)
    eff_kernel = chosen
    if chosen == isg.KERNEL_MSC or (chosen == isg.KERNEL_SWEEP and insts[0].dtype == "i8"):
        eff_kernel = 2 if chosen == isg.KERNEL_MSC else 3
    roof = roofline(name, eff_kernel, insts, R, st, t_total / steps, clk, hbm, bf16s, peak_src, ktimes, steps)
    work = {k: v for k, v in st.items() if k != "launches"}

    # equal-energy comparison with the plain comparator
    pl = None
    if plain and chosen != isg.KERNEL_PLAIN:
        comparator, ckw = isg.KERNEL_PLAIN, {}
        if chosen == isg.KERNEL_DENSE_TC:
            # dense: the straightforward blocked version with library GEMMs
            comparator, ckw = isg.KERNEL_DENSE_TC, {"dense_variant": isg.DENSE_LIBRARY}
        try:
            h.local_search(seeds, R, kernel=comparator, stats=True, **ckw, **kw)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            pr = h.local_search(seeds, R, kernel=comparator, stats=True, **ckw, **kw)
            b.record(stream)
            torch.cuda.synchronize()
            pms = a.elapsed_time(b)
            m1, m2 = float(E.mean().item()), float(pr.energy.mean().item())
            energies = {"mean_energy": m1, "comparator_mean_energy": m2,
                        "max_abs_diff": float((pr.energy - E).abs().max().item()),
                        "identical_replicas": float((pr.energy == E).double().mean().item())}
            if insts[0].dtype == "i8":
                same = bool(torch.equal(pr.energy, E))  # integer couplings: identical results
            else:
                # float couplings: the comparator's field arithmetic differs only
                # in rounding where noted (dense); equal energies up to FP64
                same = energies["max_abs_diff"] <= 1e-9 * max(1.0, abs(m1)) if chosen != isg.KERNEL_DENSE_TC \
                    else energies["identical_replicas"]
            pv = pr.stats["flip_evals"] / (pms / 1e3)
            pl = {"kind": "cublas_blocked" if chosen == isg.KERNEL_DENSE_TC else "plain",
                  "value": pv, "unit": UNIT, "ms_per_step": pms, "energy_match": same, "energies": energies,
                  "speedup": value / pv}
        except Exception as ex:  # comparator not available for this workload
            pl = {"unavailable": str(ex)}

    cpu = None
    if cpu_seconds > 0 and rank == 0 and dist is None:
        cpu = cpu_baseline(name, insts, R, kw, cpu_seconds)

    rec = {
        "workload": name, "description": desc, "value": value, "unit": UNIT,
        "minima_per_s": minima_job / t_total, "steps": steps, "ms_per_step": t_total * 1e3 / steps,
        "evaluated_per_s": value * st.get("evaluated", st["flip_evals"]) / max(1, st["flip_evals"]),
        "replicas": R, "instances": len(insts), "spins": total_spins, "kernel": isg.KERNEL_NAMES[chosen],
        "params": dict(kw), "work_per_step": work,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * len(insts),
                "d2h_bytes_per_step": R * total_spins + 8 * R * len(insts)},
        "gpu_launches_per_step": int(n_launch_per_step),
        "clocks": clk, "roofline": roof, "plain": pl, "cpu_baseline": cpu,
        "dtype": "bit-packed i1/int32" if insts[0].dtype == "i8" and chosen in (isg.KERNEL_MSC, isg.KERNEL_TILE,
                                                                               isg.KERNEL_SWEEP)
        else ("int32" if insts[0].dtype == "i8" else
              ("bf16 hi+lo tensor GEMMs, f32 fields, f64 energies" if chosen == isg.KERNEL_DENSE_TC
               else "f32 fields, f64 refresh/energy")),
    }
    h.close()
    del l2_flush
    torch.cuda.empty_cache()
    return rec


# ----------------------------------------------------------------------------- main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default=HEADLINE)
    ap.add_argument("--per-workload", default=",".join(w for w in ALL_WORKLOADS if w != HEADLINE),
                    help="comma-separated workloads measured as sub-records after the headline ('' for none)")
    ap.add_argument("--headline-only", action="store_true", help="no sub-records (profiling captures)")
    ap.add_argument("--min-seconds", type=float, default=1.5,
                    help="minimum timed device time of each sub-record")
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--kernel", default="auto")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="CPU oracle time of the headline's baseline (half on one thread, half on all cores)")
    ap.add_argument("--sub-cpu-seconds", type=float, default=4.0, help="the same for each sub-record")
    ap.add_argument("--ref-seconds", type=float, default=60.0,
                    help="--impl reference: oracle time over all warm-up and timed steps")
    # smaller variants of the headline workload, for profiler captures
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

    if args.impl == "reference":
        if rank != 0:
            return            # the oracle runs once, on rank 0; other ranks exit without work
        insts, R, kw, desc = make_workload(args.workload, args.instances, args.sk_n)
        if args.method == "fm":
            run_fm_reference(args, insts, R, kw, desc)
        else:
            run_reference(args, insts, R, kw, desc)
        return

    if args.method == "fm":
        if rank == 0:
            insts, R, kw, desc = make_workload(args.workload, args.instances, args.sk_n)
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

    head = gpu_record(args.workload, args, dev, rank, dist, steps=args.steps, plain=not args.no_plain,
                      cpu_seconds=0.0 if args.no_cpu_baseline else args.cpu_seconds)
    subs = {}
    if world == 1 and not args.headline_only:
        for w in [x for x in args.per_workload.split(",") if x and x != args.workload]:
            try:
                subs[w] = gpu_record(w, args, dev, 0, None, steps=None, min_seconds=args.min_seconds,
                                     plain=not args.no_plain,
                                     cpu_seconds=0.0 if args.no_cpu_baseline else args.sub_cpu_seconds)
            except Exception as ex:
                subs[w] = {"workload": w, "unavailable": f"{type(ex).__name__}: {ex}"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": head["dtype"],
            "data": "synthetic (seeded generators; the paper's instances are not available)",
            "minima_per_s": head["minima_per_s"], "evaluated_per_s": head["evaluated_per_s"],
            "config": {"workload": args.workload, "description": head["description"], "replicas": head["replicas"],
                       "instances": head["instances"], "spins": head["spins"], "kernel": head["kernel"],
                       "l2": "flushed (512 MB write) before every timed step",
                       "parallelism": f"replicas sharded over {world} GPU(s), no data-path collective",
                       **head["params"]},
            "work_per_step": head["work_per_step"],
            "e2e": head["e2e"],
            "gpu_launches": head["gpu_launches_per_step"] * args.steps,
            "clocks": head["clocks"],
            "roofline": head["roofline"],
            "plain": head["plain"],
            "cpu_baseline": head["cpu_baseline"],
            "per_workload": subs,
        }
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def run_reference(args, insts, R, kw, desc):
    """The reference arm: the CPU oracle as it stands on every host core, each
    step a bounded sample of the workload (units continue where the previous
    step stopped), flip evaluations per second over the timed steps."""
    cores = os.cpu_count() or 1
    seeds = seeds_for(args.workload, len(insts), 0)
    per_step = max(0.25, args.ref_seconds / max(1, args.steps + args.warmup))
    pos, evals, minima, t_all, walls, samples = 0, 0, 0.0, 0.0, [], []
    for k in range(args.warmup + args.steps):
        r = oracle_sample(args.workload, insts, R, kw, per_step, cores, seeds=seeds, start=pos)
        pos = r["next"]
        if k >= args.warmup:
            evals += r["evals"]
            minima += r["minima_per_s"] * r["wall_s"]
            t_all += r["wall_s"]
            walls.append(r["wall_s"])
            samples.append(r["sample"])
    value = evals / t_all
    sample = (f"{args.steps} timed steps of about {per_step:.2f} s each on {cores} threads; last: {samples[-1]}"
              if samples else "")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_all / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int64 (oracle)" if insts[0].dtype == "i8" else "f64/f32 mirror (oracle)",
            "data": "synthetic", "minima_per_s": minima / t_all,
            "config": {"workload": args.workload, "description": desc, "replicas": R, **kw},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                             "cpu_model": cpu_model(), "nproc": cores},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


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
        cpu = {"value": moves / dt, "unit": "moves/s", "cores": 1, "kind": "oracle", "cpu_model": cpu_model(),
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
    pos, moves_all, runs_all, t_all = 0, 0, 0, 0.0
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
            moves_all, runs_all, t_all = moves_all + moves, runs_all + runs, t_all + dt
    value = moves_all / t_all
    sample = f"{runs_all} oracle searches (first starts of this workload, in order), {moves_all} moves, {t_all:.1f} s"
    line = {"metric": "pass-based search (Sec. IV, Fig. 3) moves/s on 1 GB300", "value": value, "unit": "moves/s",
            "impl": "reference", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t_all / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64 (oracle)",
            "data": "synthetic (seeded generators)",
            "config": {"workload": args.workload, "method": "fm", "description": desc, "replicas": R,
                       "restarts": restarts, "instances": len(insts)},
            "cpu_baseline": {"value": value, "unit": "moves/s", "cores": 1, "kind": "oracle", "sample": sample,
                             "cpu_model": cpu_model()},
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


_LOGIC_PEAK = None


def logic_peak_tops(sm_count, mhz):
    """Peak of the multi-spin-coded kernels in T lane-ops/s: the lop3 issue rate
    measured on this GPU in this run (ising_logic_peak, best of three ~10 ms
    launches), else the derived 128 lanes per SM per clock."""
    global _LOGIC_PEAK
    if _LOGIC_PEAK is None:
        try:
            import paper_0912_3912_gb300 as isg
            _LOGIC_PEAK = (isg.logic_peak() / 1e12, "")
        except Exception as ex:
            _LOGIC_PEAK = (0.0, f" (measurement failed: {ex})")
    if _LOGIC_PEAK[0] > 0:
        return _LOGIC_PEAK[0], "measured: lop3.b32 issue rate of this GPU in this run (ising_logic_peak)"
    return sm_count * 128 * mhz * 1e6 / 1e12, \
        f"derived: {sm_count} SMs x 128 integer lanes x {mhz:.0f} MHz (median SM clock under load)" + _LOGIC_PEAK[1]


def _roofline(name, kernel, insts, R, st, step_s, clk, hbm, bf16s, src):
    sm_count = 152
    mhz = (clk or {}).get("sm_mhz") or 2070.0
    inst = insts[0]
    deg = sum(i.nnz for i in insts) / max(1, sum(i.n for i in insts)) if inst.row_ptr is not None else inst.n - 1
    msc = inst.dtype == "i8" and inst.hyper_ptr is None and np.all(np.abs(inst.J) == 1) and (
        inst.h is None or np.all(np.abs(inst.h) <= 1))
    if msc and kernel in (2, 3):
        # integer/logic lane-operations per (spin, replica word): per bond one
        # unsatisfied-mask op, one for the field, about one adder op per input,
        # the flip mask and the word update: 2 deg + 4.  Words counted are the
        # evaluated ones (visits skipped by the pending masks do no logic).
        lanes = 32 if kernel == 2 else (32 if R > 16 else (16 if R > 8 else 8))
        ops = 2 * deg + 4
        evaluated = st.get("evaluated", st["flip_evals"])
        words = evaluated / lanes
        achieved = words * ops / step_s / 1e12
        peak, psrc = logic_peak_tops(sm_count, mhz)
        kname = "sweep_chunk" if kernel == 3 else "tile_kernel"
        return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tlane-ops/s", "frac": achieved / peak,
                "traffic": None, "kernel": kname, "ops_per_word": ops, "replicas_per_word": lanes,
                "evaluated_share_of_visits": evaluated / max(1, st["flip_evals"]), "peak_source": psrc}
    if kernel == 4:
        # Tensor-core work actually done: each descent's first sweeps (the
        # library's default split) and one export pass, 4 n^2 flops per
        # replica and pass (BF16 hi and lo GEMMs).  Later sweeps run as
        # incremental updates on CUDA cores and are not counted here.
        n = inst.n
        sweeps_a = DENSE_TENSOR_SWEEPS
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
            "bytes_model": "4.125 B per (spin, replica) visit + 16 B x degree per accepted flip",
            "peak_source": f"{src} copy bandwidth (MEASURED_PEAKS.json)"}


if __name__ == "__main__":
    main()
