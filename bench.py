#!/usr/bin/env python
"""Benchmark of the REWL hot path: Wang-Landau flip attempts per second.

Workload (default): 2D q=10 Potts L=80, periodic, 64 windows at 75% overlap x 16 walkers per
window (1024 walkers), flatness 0.8, ln f from 1 halving towards 1e-8, 10^4 moves per walker
between flatness checks / replica exchanges; lattices from seeded uniform states 0..9.  A round
is one pass of the whole hot path: 10^4 WL moves per walker (+ ln g / H updates), the flatness
test and window advance, the replica exchange and the end-of-round test; one step is
--rounds-per-step rounds (default 256, about 0.2 s, so that the clock sampler sees the GPU
under load).

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA events on the stream
the kernels run on, with the 129 MB L2 flushed (256 MB write) before every timed step.  The
move kernel is additionally timed on its own (events inside the library) for the roofline.
`e2e` repeats the K steps through the blocking public call (rewl_run) and reads the window
ln g back to the host after every step.  The CPU baseline is the C oracle on the host cores.

Multi-GPU (torchrun): every rank runs an independent replica (weak scaling, no collective on
the data path); value = attempts of all ranks / max rank time.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    "ising_L64_h32_m16": dict(model=0, L=64, windows=32, walkers=16, overlap=0.75,
                              lnf_final=1e-8, flatness=0.8, interval=10_000, config_id=2),
    "potts10_L40_h64_m16": dict(model=10, L=40, windows=64, walkers=16, overlap=0.75,
                                lnf_final=1e-8, flatness=0.8, interval=10_000, config_id=3),
    "potts10_L80_h64_m16": dict(model=10, L=80, windows=64, walkers=16, overlap=0.75,
                                lnf_final=1e-8, flatness=0.8, interval=10_000, config_id=5),
    "ising_L8_h4_m1": dict(model=0, L=8, windows=4, walkers=1, overlap=0.75,
                           lnf_final=1e-6, flatness=0.8, interval=10_000, config_id=1),
    # accuracy against the exact g(E) with more walkers per window (--full-run)
    "ising_L8_h4_m128": dict(model=0, L=8, windows=4, walkers=128, overlap=0.75, lnf_final=1e-8,
                             flatness=0.8, interval=10_000, config_id=1, seed_instance=108),
    "ising_L16_h8_m64": dict(model=0, L=16, windows=8, walkers=64, overlap=0.75, lnf_final=1e-8,
                             flatness=0.8, interval=10_000, config_id=1, seed_instance=116),
    "ising_L32_h32_m16": dict(model=0, L=32, windows=32, walkers=16, overlap=0.75, lnf_final=1e-8,
                              flatness=0.8, interval=10_000, config_id=1, seed_instance=132),
    # 24 uneven instances in one launch per round: (model, L) cycles Ising 16/32/64 and
    # q=10 Potts 20/40; windows [8,16,32,64][i%4]; walkers [4,8,16][(i//4)%3]; 6720 walkers
    "batch24_uneven": dict(batch=True, interval=10_000, config_id=4, lnf_final=1e-8,
                           flatness=0.8, overlap=0.75),
}


def batch24_descs(wl, rank=0):
    out = []
    for i in range(24):
        model, L = [(0, 16), (0, 32), (0, 64), (10, 20), (10, 40)][i % 5]
        out.append(dict(model=model, L=L, windows=[8, 16, 32, 64][i % 4],
                        walkers=[4, 8, 16][(i // 4) % 3], lnf_final=wl["lnf_final"],
                        flatness=wl["flatness"], overlap=wl["overlap"],
                        seed=seed_for(wl["config_id"], 100 * rank + i), instance=i))
    return out
METRIC = "WL flip attempts/s"
UNIT = "attempts/s"
# Algorithmic integer work of one WL attempt (Philox4x32-10 call, site and neighbour index
# arithmetic, energy change, window test, accept test, ln g / H update), in thread
# instructions; the issue roofline is SMs x 128 lanes x SM clock.
ALG_INSTR_PER_ATTEMPT = 85
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
# side files (nvidia-smi clock samples, predicted ln g): $REWL_BENCH_OUT, else the temp folder
OUT_DIR = os.environ.get("REWL_BENCH_OUT") or __import__("tempfile").gettempdir()
THROTTLE_BITS = {0x8: "hw_slowdown", 0x40: "hw_thermal_slowdown", 0x20: "sw_thermal_slowdown",
                 0x4: "sw_power_cap", 0x80: "hw_power_brake_slowdown", 0x1: "gpu_idle",
                 0x2: "applications_clocks_setting", 0x100: "display_clock_setting"}


def seed_for(config_id: int, instance: int = 0) -> int:
    return 0x5EED201400000000 + config_id * 1000 + instance


# ----------------------------------------------------------------------------- CPU oracle leg
def _oracle_worker(args):
    wl, inst, rounds, warm = args
    import oracle as O
    o = O.REWL(wl["model"], wl["L"], wl["windows"], wl["overlap"], wl["walkers"], wl["lnf_final"],
               wl["flatness"], seed=seed_for(wl["config_id"], inst), instance=inst,
               interval=wl["interval"])
    assert o.init() == 0
    if warm:
        o.run(warm)
    t0 = time.perf_counter()
    o.run(rounds)
    return time.perf_counter() - t0


def oracle_throughput(wl, procs: int, rounds: int, warm: int = 0):
    """Independent oracle instances on `procs` host cores (spawned processes)."""
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        times = pool.map(_oracle_worker, [(wl, i, rounds, warm) for i in range(procs)])
    attempts = procs * rounds * wl["windows"] * wl["walkers"] * wl["interval"]
    return attempts / max(times), max(times), attempts


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self, index: int):
        self.index, self.proc, self.path = index, None, None

    def __enter__(self):
        try:
            self.path = os.path.join(OUT_DIR, f"clocks_bench_{os.getpid()}.csv")
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=clocks.sm,clocks.max.sm,"
                 "power.draw,clocks_event_reasons.active", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if not self.proc or not self.path or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], [], set()
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 4:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
                bits = int(parts[3], 16)
            except ValueError:
                continue
            for b, name in THROTTLE_BITS.items():
                if bits & b and name != "gpu_idle":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- ranks
def max_over_ranks(values, device=None):
    """Element-wise max of per-rank timings (all_reduce MAX); identity on one process."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def whole_job_rate(per_rank_units, world, rank_ms):
    """Weak scaling: units of all ranks divided by the slowest rank's time."""
    return per_rank_units * world / (rank_ms / 1e3)


# ----------------------------------------------------------------------------- main arms
def workload_config(args, wl, world):
    """The `config` object of a single-lattice workload (both arms print the same one)."""
    per_round = wl["windows"] * wl["walkers"] * wl["interval"]
    return {"workload": args.workload,
            "model": "ising" if wl["model"] == 0 else f"potts{wl['model']}",
            "L": wl["L"], "windows": wl["windows"], "walkers_per_window": wl["walkers"],
            "walkers": wl["windows"] * wl["walkers"], "interval": wl["interval"],
            "overlap": wl["overlap"], "flatness": wl["flatness"], "lnf_final": wl["lnf_final"],
            "lnf_init": args.lnf_init,
            "parallelism": f"replicas{world}" if world > 1 else "1gpu",
            "l2": "flushed (256 MB write) before every timed step"}


KERNEL_SOURCES = ["paper_1402_2328_gb300/csrc/rewl_kernels.cu",
                  "paper_1402_2328_gb300/csrc/rewl_kernels.cuh",
                  "paper_1402_2328_gb300/csrc/rewl_device.cuh"]


def kernel_source_digest():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


RECORDED_KEYS = ("traffic_bytes_per_launch", "issue_slots_frac_of_sm_peak",
                 "smem_wavefronts_frac_of_sm_peak", "kernel_source_digest")


def recorded_profile(workload):
    """Figures of the committed ncu summary of this workload's move kernel (DRAM bytes per
    launch, issue-slot and shared-memory-wavefront fractions of the SM peaks), when it was
    captured from the current kernel source; else {}."""
    path = os.path.join(ROOT, "profiles", f"k_move_{workload}.md")
    if not os.path.exists(path):
        return {}
    vals = {}
    for line in open(path):
        t = line.strip().lstrip("-* ").replace("`", "")
        for key in RECORDED_KEYS:
            if t.startswith(key + ":"):
                vals[key] = t.split(":", 1)[1].strip()
    if vals.pop("kernel_source_digest", None) != kernel_source_digest():
        return {}
    out = {}
    for key, v in vals.items():
        try:
            out[key] = float(v)
        except ValueError:
            pass
    return out


def recorded_traffic(workload):
    """DRAM bytes (read + write) per move launch from the committed ncu summary, or None."""
    v = recorded_profile(workload).get("traffic_bytes_per_launch")
    return int(v) if v is not None else None


def _roofline(per_launch_attempts, move_ms, move_launches, sms, step_ms, workload=None):
    peaks = json.load(open(MEASURED_PEAKS)) if os.path.exists(MEASURED_PEAKS) else {}
    sm_max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak_tinst = sms * 128 * sm_max_mhz * 1e6 / 1e12
    move_avg_s = (move_ms / max(move_launches, 1)) / 1e3
    achieved = ALG_INSTR_PER_ATTEMPT * per_launch_attempts / move_avg_s / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak_tinst, "unit": "Tinst/s",
            "frac": achieved / peak_tinst,
            "traffic": recorded_traffic(workload) if workload else None, "kernel": "k_move",
            "ncu": ({k: v for k, v in recorded_profile(workload).items()
                     if k != "traffic_bytes_per_launch"} or None) if workload else None,
            "kernel_ms_avg": move_avg_s * 1e3,
            "kernel_share_of_step": move_ms / step_ms if step_ms else None,
            "alg_inst_per_attempt": ALG_INSTR_PER_ATTEMPT,
            "peak_basis": f"{sms} SMs x 128 lanes x {sm_max_mhz:.0f} MHz (max SM clock), of measured"}


def run_gpu_batch(args, wl, rank, world):
    """Config-4 batch: aggregate attempts/s of 24 uneven instances advanced by one move launch
    per round (autotuned walkers per CTA), against the same instances run one at a time."""
    import torch
    import paper_1402_2328_gb300.rewl as R

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    descs = batch24_descs(wl, rank)
    b = R.REWLBatch(descs, interval=wl["interval"], stream=stream)
    b.init()
    best, trial = b.autotune(rounds=1)  # trial rounds of the simulation itself, untimed
    info = b.info()
    per_round = info["walkers"] * wl["interval"]
    RPS = args.rounds_per_step
    per_step = per_round * RPS
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    b.step(args.warmup * RPS)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    b.set_param("profile", 1)
    b.kernel_time(reset=True)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    with ClockSampler(dev) as clk:
        for a, z in evs:
            flush.zero_()
            a.record(stream)
            b.step(RPS)
            z.record(stream)
        torch.cuda.synchronize()
    step_ms = sum(a.elapsed_time(z) for a, z in evs)
    move_ms, move_launches = b.kernel_time(reset=True)
    b.set_param("profile", 0)
    # e2e: the blocking public call per round + window ln g of every instance back to host
    d2h = 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        b.run(max_rounds=RPS)
        for i in range(len(descs)):
            x = b.instance(i).get_state("lng_mean")
            d2h += x.nbytes
    e2e_s = time.perf_counter() - t0
    b.close()
    # the same instances one at a time (each with its own launches), same number of rounds
    solo_ms = 0.0
    for d in descs:
        g = R.REWL(d["model"], d["L"], d["windows"], d["overlap"], d["walkers"], d["lnf_final"],
                   d["flatness"], seed=d["seed"], instance=d["instance"],
                   interval=wl["interval"], stream=stream)
        g.init()
        g.step(args.warmup * RPS)
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        g.step(args.steps * RPS)
        z.record(stream)
        torch.cuda.synchronize()
        solo_ms += a.elapsed_time(z)
        g.close()
    t_max, e2e_s = max_over_ranks([step_ms, e2e_s], device="cuda")
    attempts = per_step * args.steps * world
    return {
        "metric": METRIC, "value": whole_job_rate(per_step * args.steps, world, t_max), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32+f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "instances": len(descs), "walkers": info["walkers"],
                   "interval": wl["interval"],
                   "ctas_per_launch": info["ctas"], "autotuned": best,
                   "autotune_ms_per_round": trial,
                   "parallelism": f"replicas{world}" if world > 1 else "1gpu",
                   "l2": "flushed (256 MB write) before every timed step"},
        "roofline": _roofline(per_round, move_ms, move_launches, sms, step_ms, args.workload),
        "step_work": {"rounds": RPS, "attempts": per_step * world},
        "one_at_a_time": {"value": per_step * args.steps / (solo_ms / 1e3), "unit": UNIT,
                          "ms_per_step": solo_ms / args.steps},
        "e2e": {"value": attempts / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": d2h // max(args.steps, 1),
                "call": f"rewl_batch_run({RPS} rounds) + rewl_get_state(lng_mean) of each instance"},
        "gpu_launches": 4 * RPS * args.steps, "clocks": clk.summary(),
    }


def exact_lng_golden(model, L):
    """Exact ln g from the committed golden files (Ising only), or None."""
    if model != 0:
        return None
    g = os.path.join(ROOT, "tests", "golden")
    for name in (f"ising_L{L}_lng.txt", f"ising_L{L}_counts.txt"):
        path = os.path.join(g, name)
        if os.path.exists(path):
            vals = []
            for line in open(path):
                if line.startswith("#"):
                    continue
                v = line.split()[1]
                if name.endswith("counts.txt"):
                    c = int(v)
                    vals.append(math.log(c) if c > 0 else -math.inf)
                else:
                    vals.append(float(v))
            return vals
    return None


def run_full(args, wl):
    """Time to solution: init, then rounds until every window has ln f < ln f_final."""
    import numpy as np
    import torch
    import paper_1402_2328_gb300.rewl as R

    torch.cuda.set_device(0)
    lnf_final = args.lnf_final if args.lnf_final else wl["lnf_final"]
    r = R.REWL(wl["model"], wl["L"], wl["windows"], wl["overlap"], wl["walkers"], lnf_final,
               wl["flatness"], seed=seed_for(wl["config_id"], wl.get("seed_instance", 0)),
               interval=wl["interval"], lnf_init=args.lnf_init, schedule=args.schedule)
    t0 = time.perf_counter()
    r.init()
    t_init = time.perf_counter() - t0
    with ClockSampler(0) as clk:
        status = r.run(max_seconds=args.max_seconds)
    t_run = time.perf_counter() - t0 - t_init
    st = r.stats()
    out = {"workload": args.workload, "lnf_final": lnf_final,
           "schedule": "1/t" if args.schedule else "halving", "status": status,
           "seconds_init": t_init,
           "seconds_run": t_run, "rounds": st["rounds"], "attempts": st["attempts"],
           "attempts_per_s": st["attempts"] / max(t_run, 1e-9),
           "windows_finished": st["windows_finished"], "windows": r.h,
           "min_iteration": st["min_iteration"], "max_lnf": st["max_lnf"],
           "swap_acceptance": st["swap_accepted"] / max(st["swap_attempts"], 1),
           "exact_fraction": st["exact_decisions"] / max(st["attempts"], 1),
           "clocks": clk.summary()}
    if status == "done":
        lng, joins = r.stitch(0)
        ex = exact_lng_golden(wl["model"], wl["L"])
        if ex is not None:
            ex = np.array(ex)
            fin = np.isfinite(ex)
            mx = ex[fin].max()
            ex = ex - (mx + math.log(np.exp(ex[fin] - mx).sum()) - r.N * math.log(2))
            out["max_abs_dlng_vs_exact"] = float(np.max(np.abs(lng[fin] - ex[fin])))
            out["rms_dlng_vs_exact"] = float(np.sqrt(np.mean((lng[fin] - ex[fin]) ** 2)))
        if r.m >= 2:
            # jackknife error bars over the m walkers' fragments (Sec. 3); the paper finds the
            # deviation from the exact result of the order of the statistical error
            err = r.jackknife(0)
            ok = np.isfinite(err) & np.isfinite(lng)
            out["jackknife_max"] = float(err[ok].max())
            out["jackknife_rms"] = float(np.sqrt(np.mean(err[ok] ** 2)))
            if ex is not None:
                okx = ok & np.isfinite(ex)
                out["rms_dlng_over_jackknife_rms"] = float(
                    np.sqrt(np.mean((lng[okx] - ex[okx]) ** 2)) / np.sqrt(np.mean(err[okx] ** 2)))
    r.close()
    return out


def run_warm(args):
    """Learned warm start: plain REWL on Ising and q=10 Potts, L = 8..32 (one batched launch
    per round) -> joined ln g -> MLP trained on the GPU -> predicted ln g of the target lattice;
    then the target run cold (ln f0 = 1) and warm (predicted ln g, small ln f0), timed."""
    import numpy as np
    import torch
    import paper_1402_2328_gb300.rewl as R
    from paper_1402_2328_gb300 import warm as WM

    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    descs = []
    for i, (model, L) in enumerate(WM.TRAIN_LATTICES):
        B = L * L if model == 0 else 2 * L * L
        h = max(2, min(16, B // 128))
        descs.append(dict(model=model, L=L, windows=h, walkers=4, lnf_final=args.train_lnf_final,
                          seed=seed_for(5, 500 + i), instance=i))
    b = R.REWLBatch(descs, interval=10_000)
    st = b.run(max_seconds=args.max_seconds)
    t_train_runs = time.perf_counter() - t0
    runs, train_stats = [], []
    # learned window boundaries: the first-iteration cost profile of the largest training
    # lattice of the target model, carried to the target lattice by energy per site
    big = max((i for i, d in enumerate(descs) if d["model"] == args.warm_model),
              key=lambda i: descs[i]["L"])
    lw_lo, lw_hi = b.instance(big).balanced_windows_for(args.warm_L, args.warm_windows, 0.75)
    for i, d in enumerate(descs):
        inst = b.instance(i)
        s_i = inst.stats()
        if s_i["windows_finished"] == inst.h:
            lng, _ = inst.stitch(0)
            runs.append((d["model"], d["L"], lng))
        train_stats.append(dict(model=d["model"], L=d["L"], windows=d["windows"],
                                rounds=s_i["rounds"], finished=s_i["windows_finished"] == inst.h))
    b.close()
    X, T = WM.training_set(runs)
    t1 = time.perf_counter()
    P, hist = WM.train(X, T, steps=args.train_steps, lr=3e-3, seed=seed_for(5, 999))
    torch.cuda.synchronize()
    t_fit = time.perf_counter() - t1
    lng_pred = WM.predict_lng(P, args.warm_model, args.warm_L)

    # run-time balanced windows of the target lattice itself (Fig. 1b): a pre-run with equal
    # windows until every window finished its first iteration, then the balanced layout
    bal = None
    if any(v.partition("@")[0].endswith("_bal") for v in args.warm_variants.split(",")):
        pre = R.REWL(args.warm_model, args.warm_L, args.warm_windows, 0.75, args.warm_walkers,
                     args.warm_lnf_final, 0.8, seed=seed_for(5, 900), interval=10_000)
        pre.init()
        tp = time.perf_counter()
        while time.perf_counter() - tp < args.max_seconds:
            pre.run(max_rounds=500)
            if np.all(pre.get_state("first_iter_round") > 0):
                break
        t1 = pre.get_state("first_iter_round")
        bal = dict(seconds=time.perf_counter() - tp, rounds=int(pre.get_state("round")[0]),
                   complete=bool(np.all(t1 > 0)))
        bal["lo"], bal["hi"] = pre.balanced_windows(args.warm_windows, 0.75)
        pre.close()

    # windows balanced by the cost of later iterations (rounds per iteration over iterations
    # 3..6 of an equal-window pre-run on the target lattice)
    late = None
    if any(v.partition("@")[0].endswith("_late") for v in args.warm_variants.split(",")):
        from paper_1402_2328_gb300 import balance as BL
        pre = R.REWL(args.warm_model, args.warm_L, args.warm_windows, 0.75, args.warm_walkers,
                     args.warm_lnf_final, 0.8, seed=seed_for(5, 900), interval=10_000)
        llo, lhi, late = BL.late_balanced_windows(pre, args.warm_windows, 3, 6,
                                                  max_seconds=args.max_seconds)
        late.update(lo=llo, hi=lhi)
        pre.close()

    def target(seed, variant):
        # variant: kind[@ln f0], kind in warm (learned windows), warm_eq, cold, cold_lw,
        # cold_bal / warm_bal (windows balanced by the pre-run's first iterations) and
        # cold_late / warm_late (balanced by its later iterations)
        kind, _, lnf0 = variant.partition("@")
        if kind.startswith("warm"):
            r = WM.warm_handle(args.warm_model, args.warm_L, args.warm_windows, args.warm_walkers,
                               args.warm_lnf_final, seed, lng_pred,
                               lnf_init=float(lnf0) if lnf0 else args.warm_lnf_init)
        else:
            r = R.REWL(args.warm_model, args.warm_L, args.warm_windows, 0.75, args.warm_walkers,
                       args.warm_lnf_final, 0.8, seed=seed, interval=10_000)
        if kind in ("warm", "cold_lw"):
            r.set_windows(lw_lo, lw_hi)
        if kind.endswith("_bal"):
            r.set_windows(bal["lo"], bal["hi"])
        if kind.endswith("_late"):
            r.set_windows(late["lo"], late["hi"])
        ts = time.perf_counter()
        status = r.run(max_seconds=args.max_seconds)
        dt = time.perf_counter() - ts
        s_r = r.stats()
        out = dict(status=status, seconds=dt, rounds=s_r["rounds"], attempts=s_r["attempts"],
                   windows_finished=s_r["windows_finished"], max_lnf=s_r["max_lnf"])
        lng = r.stitch(0)[0] if status == "done" else None
        if status == "done" and r.m >= 2:
            err = r.jackknife(0)
            ok = np.isfinite(err) & np.isfinite(lng)
            out["jackknife_max"] = float(err[ok].max())
            out["jackknife_rms"] = float(np.sqrt(np.mean(err[ok] ** 2)))
        r.close()
        return out, lng

    results, lngs = {}, {}
    per_seed = {}
    for si in range(args.warm_seeds):
        for kind in args.warm_variants.split(","):
            res, lng = target(seed_for(args.warm_seed_config, args.warm_seed_offset + si), kind)
            per_seed.setdefault(kind, []).append((res, lng))
    for kind, lst in per_seed.items():
        results[kind], lngs[kind] = lst[0]
    cold = results.get("cold")
    warm = results.get("warm")
    for v, res in results.items():
        if cold and res.get("status") == "done" and cold["status"] == "done":
            res["time_vs_cold"] = res["seconds"] / cold["seconds"]
        if lngs.get(v) is not None and lngs.get("cold") is not None and v != "cold":
            a, c_ = lngs[v], lngs["cold"]
            fin = np.isfinite(a) & np.isfinite(c_)
            res["max_abs_dlng_vs_cold"] = float(np.max(np.abs(a[fin] - c_[fin])))
        ex_g = exact_lng_golden(args.warm_model, args.warm_L)
        if lngs.get(v) is not None and ex_g is not None:
            ex_a = np.array(ex_g)
            f2 = np.isfinite(ex_a)
            ex_a = ex_a - (ex_a[f2].max() + math.log(np.exp(ex_a[f2] - ex_a[f2].max()).sum())
                           - args.warm_L ** 2 * math.log(2))
            res["max_abs_dlng_vs_exact"] = float(np.max(np.abs(lngs[v][f2] - ex_a[f2])))
    lng_cold, lng_warm = lngs.get("cold"), lngs.get("warm")

    # mean over seeds: seconds, rounds, error against the exact result where it exists
    ex_all = exact_lng_golden(args.warm_model, args.warm_L)
    summary = {}
    for kind, lst in per_seed.items():
        secs = [r_["seconds"] for r_, _ in lst if r_["status"] == "done"]
        errs = []
        if ex_all is not None:
            ex_a = np.array(ex_all)
            f2 = np.isfinite(ex_a)
            ex_a = ex_a - (ex_a[f2].max() + math.log(np.exp(ex_a[f2] - ex_a[f2].max()).sum())
                           - args.warm_L ** 2 * math.log(2))
            errs = [float(np.max(np.abs(l_[f2] - ex_a[f2]))) for _, l_ in lst if l_ is not None]
        summary[kind] = {"seeds": len(lst), "done": len(secs),
                         "seconds": [r_["seconds"] for r_, _ in lst],
                         "mean_seconds": float(np.mean(secs)) if secs else None,
                         "max_abs_dlng_vs_exact": errs,
                         "mean_max_abs_dlng_vs_exact": float(np.mean(errs)) if errs else None}
    if "cold" in summary and summary["cold"]["mean_seconds"]:
        for kind, v in summary.items():
            if v["mean_seconds"]:
                v["mean_time_vs_cold"] = v["mean_seconds"] / summary["cold"]["mean_seconds"]

    def maxdiff(a, b_):
        if a is None or b_ is None:
            return None
        fin = np.isfinite(a) & np.isfinite(b_)
        return float(np.max(np.abs(a[fin] - b_[fin])))

    N = args.warm_L ** 2
    q = 2 if args.warm_model == 0 else args.warm_model
    pred = np.array(lng_pred, np.float64)
    mx = pred.max()
    pred_n = pred - (mx + math.log(np.exp(pred - mx).sum()) - N * math.log(q))
    if lng_cold is not None:
        pred_n = np.where(np.isfinite(lng_cold), pred_n, -np.inf)
    if os.environ.get("REWL_BENCH_OUT"):
        np.save(os.path.join(OUT_DIR, "warm_lng_pred.npy"), pred)
    return {"warm_start": {
        "target": dict(model=args.warm_model, L=args.warm_L, windows=args.warm_windows,
                       walkers_per_window=args.warm_walkers, lnf_final=args.warm_lnf_final,
                       lnf_init_warm=args.warm_lnf_init),
        "training_runs": train_stats, "training_status": st,
        "training_runs_seconds": t_train_runs, "training_samples": int(X.shape[0]),
        "fit_seconds": t_fit, "fit_loss": hist[-1][1],
        "runs": results, "over_seeds": summary,
        "learned_windows": {"lo": lw_lo.tolist(), "hi": lw_hi.tolist()},
        "balanced_prerun": ({k: (v.tolist() if hasattr(v, "tolist") else v) for k, v in bal.items()}
                            if bal else None),
        "late_balanced_prerun": ({k: (v.tolist() if hasattr(v, "tolist") else v)
                                  for k, v in late.items()} if late else None),
        "speedup_time": (cold["seconds"] / warm["seconds"])
        if cold and warm and warm["status"] == "done" and cold["status"] == "done" else None,
        "max_abs_dlng_warm_vs_cold": maxdiff(lng_warm, lng_cold),
        # every pair of finished variants of the first seed, and of two seeds of one variant
        "pairwise_max_abs_dlng": {
            **{f"{a}|{b}": maxdiff(lngs[a], lngs[b]) for a in lngs for b in lngs
               if a < b and lngs[a] is not None and lngs[b] is not None},
            **{f"{k}|seed0-seed1": maxdiff(lst[0][1], lst[1][1]) for k, lst in per_seed.items()
               if len(lst) > 1 and lst[0][1] is not None and lst[1][1] is not None}},
        "max_abs_dlng_prediction_vs_cold": maxdiff(pred_n, lng_cold),
    }}


def run_em(args):
    """Joint g(E, M) of the Ising model (Sec. 3, Eqs. 3-4): REWL to ln f_final, then production
    rounds (frozen ln g, multicanonical per window) with and without the (E, M) measurement, and
    the normal-vector join; for L = 6 the error against the exact g(E, M) (golden file)."""
    import numpy as np
    import torch
    import paper_1402_2328_gb300.rewl as R

    torch.cuda.set_device(0)
    L, h, m, K = args.em_L, args.em_windows, args.em_walkers, args.em_rounds
    r = R.REWL(0, L, h, 0.75, m, args.em_lnf_final, 0.8, seed=seed_for(7), interval=10_000)
    t0 = time.perf_counter()
    status = r.run(max_seconds=args.max_seconds)
    t_conv = time.perf_counter() - t0
    r.set_param("production", 1)
    t0 = time.perf_counter()
    r.run(max_rounds=K)
    t_plain = time.perf_counter() - t0
    r.set_param("measure_em", 1)
    t0 = time.perf_counter()
    r.run(max_rounds=K)
    t_meas = time.perf_counter() - t0
    t0 = time.perf_counter()
    out, joins = r.stitch_em()
    t_join = time.perf_counter() - t0
    res = {"workload": f"ising_L{L}_h{h}_m{m}", "lnf_final": args.em_lnf_final, "status": status,
           "seconds_to_lnf_final": t_conv, "production_rounds": K,
           "ms_per_round_plain": t_plain * 1e3 / K, "ms_per_round_measured": t_meas * 1e3 / K,
           "seconds_join": t_join, "points_present": int(np.isfinite(out).sum()),
           "joins": joins.tolist()}
    path = os.path.join(ROOT, "tests", "golden", f"ising_L{L}_em_counts.txt")
    if os.path.exists(path):
        N = L * L
        ex = np.full((N + 1, N + 1), -np.inf)
        for line in open(path):
            if not line.startswith("#"):
                k, j, v = line.split()
                ex[int(k), int(j)] = math.log(int(v))
        fin = np.isfinite(ex) & np.isfinite(out)
        d = np.abs(out[fin] - ex[fin])
        res.update(max_abs_dlng_vs_exact=float(d.max()), mean_abs_dlng_vs_exact=float(d.mean()),
                   points_exact=int(np.isfinite(ex).sum()))
    r.close()
    return {"em": res}


def run_speedup(args):
    """Eq. (5): s_o(h, m) = N_single / N_o(h, m), N = MC moves of the slowest walker until the
    first WL iteration is complete ((rounds until the last window's first halving) x interval).
    Equal windows (Fig. 1a) for h in --speedup-h, then run-time balanced windows (Fig. 1b) built
    from each equal-window run's first-iteration times, run with new seeds.  Every (h, seed)
    instance of a phase advances in one batched launch per round; ln f_final = 0.75 stops each
    window at its first halving."""
    import numpy as np
    import torch
    import paper_1402_2328_gb300.rewl as R

    torch.cuda.set_device(0)
    model, L, m = args.speedup_model, args.speedup_L, args.speedup_walkers
    hs = [int(x) for x in args.speedup_h.split(",")]
    S, interval = args.speedup_seeds, args.speedup_interval

    def phase(layouts, seed_base):
        descs, keys = [], []
        for (h, s) in sorted(layouts):
            descs.append(dict(model=model, L=L, windows=h, walkers=m, lnf_final=0.75,
                              seed=seed_for(6, seed_base + 100 * h + s), instance=len(descs)))
            keys.append((h, s))
        b = R.REWLBatch(descs, interval=interval)
        for i, k in enumerate(keys):
            if layouts[k] is not None:
                b.instance(i).set_windows(*layouts[k])
        b.init()
        t0 = time.perf_counter()
        status = b.run(max_seconds=args.max_seconds)
        sec = time.perf_counter() - t0
        res = {}
        for i, k in enumerate(keys):
            inst = b.instance(i)
            t1 = inst.get_state("first_iter_round").astype(np.int64)
            res[k] = dict(t1=t1, lohi=inst.balanced_windows(k[0], 0.75) if k[0] > 1 else None,
                          width=(inst.get_state("hi") - inst.get_state("lo") + 1))
        b.close()
        return res, status, sec

    eq, st_eq, sec_eq = phase({(h, s): None for h in hs for s in range(S)}, 0)
    bal_layouts = {(h, s): eq[(h, s)]["lohi"] for h in hs if h > 1 for s in range(S)}
    bal, st_bal, sec_bal = phase(bal_layouts, 50_000)

    def summary(res, h):
        n = [res[(h, s)]["t1"].max() * interval for s in range(S) if res[(h, s)]["t1"].min() > 0]
        spread = [res[(h, s)]["t1"].max() / res[(h, s)]["t1"].min() for s in range(S)
                  if res[(h, s)]["t1"].min() > 0]
        return (float(np.mean(n)) if n else None, float(np.mean(spread)) if spread else None,
                len(n))

    n_single, _, _ = summary(eq, 1) if 1 in hs else (None, None, 0)
    rows = []
    for h in hs:
        ne, sp_e, ok_e = summary(eq, h)
        nb, sp_b, ok_b = summary(bal, h) if h > 1 else (ne, sp_e, ok_e)
        rows.append({"h": h, "m": m,
                     "N_equal": ne, "s_equal": n_single / ne if n_single and ne else None,
                     "t1_spread_equal": sp_e,
                     "N_balanced": nb, "s_balanced": n_single / nb if n_single and nb else None,
                     "t1_spread_balanced": sp_b, "seeds_done": [ok_e, ok_b]})
    return {"speedup": {"model": model, "L": L, "overlap": 0.75, "walkers_per_window": m,
                        "interval": interval, "seeds": S, "status": [st_eq, st_bal],
                        "seconds": [sec_eq, sec_bal], "rows": rows}}


def run_gpu(args, wl, rank, world):
    import torch
    import paper_1402_2328_gb300.rewl as R

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    r = R.REWL(wl["model"], wl["L"], wl["windows"], wl["overlap"], wl["walkers"], wl["lnf_final"],
               wl["flatness"], seed=seed_for(wl["config_id"], rank), instance=rank,
               interval=wl["interval"], stream=stream,
               lnf_init=args.lnf_init)
    r.init()
    per_round = r.nw * wl["interval"]
    RPS = args.rounds_per_step
    per_step = per_round * RPS
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        r.step(RPS)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    r.set_param("profile", 1)
    r.kernel_time(reset=True)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        for a, b in evs:
            flush.zero_()  # L2 flush, outside the timed events
            a.record(stream)
            r.step(RPS)
            b.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    step_ms = sum(a.elapsed_time(b) for a, b in evs)
    move_ms, move_launches = r.kernel_time(reset=True)
    r.set_param("profile", 0)
    st = r.stats()
    if st["exact_decisions"] < 0:
        raise RuntimeError("bad stats")
    # e2e through the blocking public call, reading window ln g back each round
    lng_bytes = r.h * r.W * 8
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r.run(max_rounds=RPS)
        _ = r.get_state("lng_mean")
    e2e_s = time.perf_counter() - t0
    t_max, e2e_s = max_over_ranks([step_ms, e2e_s], device="cuda")
    attempts = per_step * args.steps * world
    value = whole_job_rate(per_step * args.steps, world, t_max)
    clocks = clk.summary()
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32+f64", "data": "synthetic",
        "config": workload_config(args, wl, world),
        "step_work": {"rounds": RPS, "attempts": per_step * world},
        "roofline": _roofline(per_round, move_ms, move_launches, sms, step_ms, args.workload),
        "e2e": {"value": attempts / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": lng_bytes + 48,
                "call": f"rewl_run({RPS} rounds) + rewl_get_state(lng_mean) per step"},
        "gpu_launches": 4 * RPS * args.steps,
        "clocks": clocks,
        "exact_fraction": st["exact_decisions"] / max(st["attempts"], 1),
    }
    r.close()
    return out


def run_gpu_sharded(args, wl, rank, world):
    """One run of the workload with its windows split over the ranks (consecutive ranges, one
    shard per GPU; Sec. 2 exchange across shard boundaries by point-to-point transfers after
    every round).  Strong scaling: the total work is fixed as N grows."""
    import torch
    import torch.distributed as dist
    from paper_1402_2328_gb300 import shard as S
    import paper_1402_2328_gb300.rewl as RW

    ndev = torch.cuda.device_count()
    dev = int(os.environ.get("LOCAL_RANK", "0")) % max(ndev, 1)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    seed = seed_for(wl["config_id"])
    glo, ghi = RW.windows_layout(RW.num_bins(wl["model"], wl["L"]), wl["windows"], wl["overlap"])
    wb, n = S.split_windows(wl["windows"], world)[rank]
    h = S.make_shard(wl["model"], wl["L"], glo, ghi, wb, n, wl["walkers"], wl["lnf_final"],
                     wl["flatness"], seed, interval=wl["interval"], lnf_init=args.lnf_init,
                     stream=stream)
    h.init()
    d = S.DistShard(h, rank, world, torch.device("cuda", dev))
    per_round = wl["windows"] * wl["walkers"] * wl["interval"]   # the whole run, all ranks
    RPS = args.rounds_per_step
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    d.step(args.warmup * RPS)
    torch.cuda.synchronize()
    dist.barrier()
    h.set_param("profile", 1)
    h.kernel_time(reset=True)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    with ClockSampler(dev) as clk:
        for a, b in evs:
            flush.zero_()
            a.record(stream)
            d.step(RPS)
            b.record(stream)
        torch.cuda.synchronize()
    dist.barrier()
    step_ms = sum(a.elapsed_time(b) for a, b in evs)
    move_ms, move_launches = h.kernel_time(reset=True)
    h.set_param("profile", 0)
    t_max = max_over_ranks([step_ms], device="cuda" if dist.get_backend() == "nccl" else "cpu")[0]
    nb = len(d.bounds)
    out = {
        "metric": METRIC, "value": per_round * RPS * args.steps / (t_max / 1e3), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "int32+f64", "data": "synthetic",
        "config": dict(workload_config(args, wl, 1), parallelism=f"windows{world}"),
        "step_work": {"rounds": RPS, "attempts": per_round * RPS},
        "roofline": _roofline(h.nw * wl["interval"], move_ms, move_launches, sms, step_ms, args.workload),
        "gpu_launches": (4 + 4 * nb) * RPS * args.steps,
        "shards": S.split_windows(wl["windows"], world),
        "transport": dist.get_backend(), "clocks": clk.summary(),
    }
    h.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--sharded", action="store_true",
                    help="N > 1: split the workload's windows over the ranks (one run, strong "
                         "scaling) instead of N independent replicas")
    ap.add_argument("--backend", default="nccl", choices=["nccl", "gloo"],
                    help="torch.distributed backend for N > 1 (gloo: transfers through the host)")
    ap.add_argument("--workload", default="potts10_L80_h64_m16", choices=sorted(WORKLOADS))
    ap.add_argument("--rounds-per-step", type=int, default=256,
                    help="rounds of the hot path in one timed step")
    ap.add_argument("--cpu-rounds", type=int, default=2, help="oracle rounds per core (baseline)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--lnf-init", type=float, default=1.0, help="ln f of the first iteration")
    ap.add_argument("--full-run", action="store_true",
                    help="run the workload to ln f < ln f_final and report the time to solution")
    ap.add_argument("--max-seconds", type=float, default=1800.0, help="cap of --full-run")
    ap.add_argument("--lnf-final", type=float, default=0.0,
                    help="--full-run: ln f_final instead of the workload's")
    ap.add_argument("--schedule", type=int, default=0, choices=[0, 1],
                    help="--full-run: 0 = ln f halving, 1 = switch to the 1/t schedule")
    ap.add_argument("--warm-start", action="store_true",
                    help="learned warm start experiment: train on small lattices, compare "
                         "warm vs cold on the target lattice")
    ap.add_argument("--warm-model", type=int, default=10)
    ap.add_argument("--warm-L", type=int, default=80)
    ap.add_argument("--warm-windows", type=int, default=64)
    ap.add_argument("--warm-walkers", type=int, default=16)
    ap.add_argument("--warm-lnf-final", type=float, default=1e-8)
    ap.add_argument("--warm-lnf-init", type=float, default=1e-3)
    ap.add_argument("--train-lnf-final", type=float, default=1e-6)
    ap.add_argument("--train-steps", type=int, default=6000)
    ap.add_argument("--em", action="store_true",
                    help="joint g(E, M): production rounds with the (E, M) measurement + join")
    ap.add_argument("--em-L", type=int, default=32)
    ap.add_argument("--em-windows", type=int, default=16)
    ap.add_argument("--em-walkers", type=int, default=8)
    ap.add_argument("--em-lnf-final", type=float, default=1e-6)
    ap.add_argument("--em-rounds", type=int, default=2000)
    ap.add_argument("--speedup", action="store_true",
                    help="speed-up s_o(h, m) of Eq. (5) with equal and run-time balanced windows")
    ap.add_argument("--speedup-model", type=int, default=0)
    ap.add_argument("--speedup-L", type=int, default=32)
    ap.add_argument("--speedup-walkers", type=int, default=1)
    ap.add_argument("--speedup-h", default="1,2,4,8,16,32")
    ap.add_argument("--speedup-seeds", type=int, default=8)
    ap.add_argument("--speedup-interval", type=int, default=10_000)
    ap.add_argument("--warm-seeds", type=int, default=1, help="target runs per variant")
    ap.add_argument("--warm-seed-config", type=int, default=5,
                    help="target seeds: seed_for(config, offset + i), i < --warm-seeds")
    ap.add_argument("--warm-seed-offset", type=int, default=1)
    ap.add_argument("--warm-variants", default="cold,warm",
                    help="comma list of cold | warm | cold_lw | warm_eq (lw: learned windows) | "
                         "cold_bal | warm_bal (first-iteration balanced) | cold_late | warm_late "
                         "(later-iteration balanced), each optionally @ln_f0, e.g. warm_eq@0.01")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    wl = WORKLOADS[args.workload]
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    procs = os.cpu_count() or 1

    if args.full_run:
        print(json.dumps({"full_run": run_full(args, wl)}))
        return
    if args.warm_start:
        print(json.dumps(run_warm(args)))
        return
    if args.speedup:
        print(json.dumps(run_speedup(args)))
        return
    if args.em:
        print(json.dumps(run_em(args)))
        return

    if args.impl == "reference":
        # the oracle is the reference arm: rank 0 only, host cores only
        if rank != 0:
            return
        # a step of this arm is one round of the workload on one core; the cores run
        # `procs` independent instances in parallel, so the steps taken are procs x rounds and
        # ms_per_step x steps equals the timed wall time
        rounds = max(1, math.ceil(args.steps / procs))
        val, tmax, attempts = oracle_throughput(wl, procs, rounds, warm=0)
        steps = procs * rounds
        out = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world,
               "steps": steps, "warmup": args.warmup,
               "ms_per_step": tmax * 1e3 / steps, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "int32+f64", "data": "synthetic",
               "config": workload_config(args, wl, world),
               "step_work": {"rounds": 1, "attempts": wl["windows"] * wl["walkers"] * wl["interval"]},
               "cpu_baseline": {"value": val, "unit": UNIT, "cores": procs, "kind": "oracle",
                                "sample": f"{procs} independent oracle instances of the workload, "
                                          f"{rounds} rounds each ({attempts:.3g} attempts, "
                                          f"{tmax:.1f} s)"},
               "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0,
                       "d2h_bytes_per_step": 0}}
        print(json.dumps(out))
        return

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not wl.get("batch"):
        # spawn the oracle pool before the first CUDA call
        val, tmax, attempts = oracle_throughput(wl, procs, args.cpu_rounds)
        cpu = {"value": val, "unit": UNIT, "cores": procs, "kind": "oracle",
               "sample": f"{procs} independent single-threaded oracle instances of the workload, "
                         f"{args.cpu_rounds} rounds each ({attempts:.3g} attempts, {tmax:.1f} s)"}
    if world > 1:
        import torch
        ndev = max(torch.cuda.device_count(), 1)
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")) % ndev)  # before NCCL binds a GPU
        torch.distributed.init_process_group(args.backend)
    if args.sharded and world > 1 and not wl.get("batch"):
        out = run_gpu_sharded(args, wl, rank, world)
    else:
        out = run_gpu_batch(args, wl, rank, world) if wl.get("batch") else run_gpu(args, wl, rank, world)
    if rank == 0:
        if cpu is not None:
            out["cpu_baseline"] = cpu
        print(json.dumps(out))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
