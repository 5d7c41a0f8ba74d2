"""Benchmark: IPC sim-steps per second summed over environments.

Workload (N=1, default): the uneven batch, 1024 grasp environments stepped as one batch through
the C ABI. Each env is, with equal odds, a soft star-shaped object of log-uniform 2k-60k
Neo-Hookean tets squeezed between kinematic rigid plates, or the same kind of object grasped by
two soft wedge finger pads (~5k tets each); a quarter of the envs have two gripper pairs. dt =
5 ms, FP64, objects' E log-uniform 1e4-1e6 Pa. Every run starts from the same synthetic
contact-phase state (grippers placed where their schedules put them at step 20, 0.7-0.8 mm from
the object), does W untimed steps and times K steps of every env. A "step" is one ipc_step over
the whole batch: every active env advances one time step (its full Newton loop).
`--workload pads` selects the 64-env pad grasp of a rigid hull instead.

Legs of the same JSON line:
  value        FP64 batched, device-timed (CUDA events on the scene's stream)
  e2e          the same K steps through the public API with host buffers (next targets up,
               all DOFs down, every step)
  plain_fp64   the same kernels one env at a time (a stated sample of the envs, from the same
               states): the plain GPU stepper, and the paper-style ratio of N envs batched
               over the same N envs run in sequence (Sec. IV-A)
  mixed_precision  the same K steps in mixed precision, and the error of both precisions
               against a converged FP64 solve of a sample
  cpu_baseline the CPU oracle on a bounded sample, one env per host core
  serving      grasp-evaluation requests served by continuous batching

Under torchrun every rank runs its own batch: the global pool of world x N envs is split by
greedy longest-processing-time bin-packing of their estimated costs (tets + surface size), so
the ranks get equal work (weak scaling, no collective on the data path); rank times combine by
max.

--impl reference times the CPU oracle (plain FP64, no GPU) on a bounded sample of the same
workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mpc
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2503_05020_b300 import scenes as S  # noqa: E402

METRIC = "IPC sim-steps/s summed over envs"
UNIT = "env-steps/s"
DT = 0.005


class Workload:
    def __init__(self, name: str):
        self.name = name
        if name == "uneven":
            self.build, self.state_at, self.start = S.uneven_batch_env, S.grasp_state_at, S.UNEVEN_START_STEP
            self.cost = S.uneven_batch_cost
        else:
            self.build, self.state_at, self.start = S.pad_grasp_env, S.pad_grasp_state_at, 20
            self.cost = lambda i: 1.0

    def config(self, n_env, tets, world):
        if self.name == "uneven":
            w = (f"uneven batch x{n_env} envs: soft star objects of log-uniform 2k-60k tets squeezed by rigid plates "
                 f"or grasped by two soft pads (~5k tets each), 25% with two gripper pairs, dt={DT}s, FP64, "
                 f"from schedule step {self.start}")
            sched = "plates: close 75 steps, lift; pads: close 100 steps (gravity off), then lift (gravity on)"
        else:
            w = (f"pad-grasp x{n_env} envs (2 soft pads ~5k tets each + rigid hull 1584 tris), dt={DT}s, FP64, "
                 f"from schedule step {self.start}")
            sched = "close 100 steps (gravity off) then lift 0.1 m (gravity on)"
        return {"workload": w, "envs_per_gpu": n_env, "tets_per_env_avg": tets, "start_step": self.start,
                "schedule": sched, "l2": "inputs larger than L2 (BSR + element buffers of the batch exceed 126 MB)",
                "parallelism": "replicas" if world == 1 else f"env-sharded x{world} (LPT by estimated cost)"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="uneven", choices=["uneven", "pads"])
    ap.add_argument("--envs", type=int, default=None, help="envs per GPU (default 1024 uneven, 64 pads)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--pcg-cluster", type=int, default=0,
                    help="PCG launch shape: 0 automatic, 1/2/4/8/16 CTAs per env cluster, -1 tiled multi-launch")
    ap.add_argument("--plain-envs", type=int, default=16, help="envs of the one-env-at-a-time leg (0: none)")
    ap.add_argument("--ref-envs", type=int, default=16, help="envs of the converged FP64 reference (0: none)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=12, help="requests per arrival rate of the serving leg (0: none)")
    ap.add_argument("--serve-rates", default="0.2,20", help="Poisson arrival rates of the serving leg (1/s)")
    ap.add_argument("--serve-ref", type=int, default=3, help="requests of the serving leg's converged FP64 reference")
    ap.add_argument("--no-mixed-leg", action="store_true",
                    help="skip the mixed-precision run of the same steps that the FP64 line reports beside it")
    ap.add_argument("--cpu-budget", type=float, default=150.0, help="seconds of oracle time for --impl reference")
    ap.add_argument("--leg-budget", type=float, default=1100.0,
                    help="seconds since the start of the run after which secondary legs not yet begun are skipped "
                         "(the headline line is always printed)")
    a = ap.parse_args()
    if a.envs is None:
        a.envs = 1024 if a.workload == "uneven" else 64
    return a


def shard_env_ids(rank, world, n_env, cost=None):
    """Env ids of one rank. The global pool holds world * n_env envs; it is split by greedy
    longest-processing-time bin-packing of the envs' estimated costs, so each rank gets an equal
    share of the work (the counts may differ by a few envs). Disjoint, and the same on every
    rank without communication."""
    ids = list(range(world * n_env))
    if world == 1:
        return ids
    costs = [cost(i) if cost else 1.0 for i in ids]
    return S.lpt_shards(costs, world)[rank]


def _build_one(args):
    name, i = args
    return Workload(name).build(i)


def make_envs(wl: Workload, ids):
    """Build the envs (a spawned process pool: no CUDA context is ever forked)."""
    n_proc = min(len(ids), os.cpu_count() or 1, 16)
    if len(ids) < 64 or n_proc <= 1:
        return [wl.build(i) for i in ids]
    with mpc.get_context("spawn").Pool(n_proc) as pool:
        return pool.map(_build_one, [(wl.name, i) for i in ids], chunksize=8)


# The oracle's cost grows faster than linearly with an env's size (all-pairs broad phase, CG to
# 1e-12): its timed sample takes envs of at most this many tets (the small end of the batch), so
# that one step of the sample takes seconds, not hours.
CPU_SAMPLE_MAX_TETS = 6000


def cpu_sample(tets, n):
    """Envs of the CPU oracle sample: n envs at evenly spaced size quantiles among the envs of at
    most CPU_SAMPLE_MAX_TETS tets (all envs when none is that small)."""
    small = [i for i, t in enumerate(tets) if t <= CPU_SAMPLE_MAX_TETS] or list(range(len(tets)))
    return [small[j] for j in stratified([tets[i] for i in small], n)]


def stratified(values, n):
    """Indices of n items at evenly spaced quantiles (i + 0.5) / n of the given values (ties by
    index): a sample that keeps the batch's size mix."""
    order = sorted(range(len(values)), key=lambda i: (values[i], i))
    n = min(n, len(order))
    return sorted({order[int((k + 0.5) * len(order) / n)] for k in range(n)})


def max_over_ranks(v, world, device):
    """The largest value over the ranks: a run's time is its slowest rank's."""
    if world <= 1:
        return float(v)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(v, world, device):
    if world <= 1:
        return float(v)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_throughput(env_steps, seconds):
    """Whole-job env-steps/s: the env-steps of every rank over the slowest rank's time."""
    return env_steps / seconds


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def host_info() -> dict:
    model = platform.processor() or ""
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model}


# FP64 peak of one B300 from its unit counts and clock: 148 SMs x 4 FP64 flop/clk (2 DFMA) x
# 2.032 GHz (1.25 TFLOP/s nominal at the boost clock; 1.11 measured by an FMA loop at 2032 MHz).
FP64_PEAK_TFLOPS = 148 * 4 * 2.032e9 / 1e12


# DRAM bytes per launch of k_pcg_cluster measured by ncu (dram__bytes_read.sum +
# dram__bytes_write.sum over every launch of `bench.py --steps 2 --warmup 3 --plain-envs 0
# --no-mixed-leg --no-cpu-baseline --serve-requests 0`, averaged per launch). Keyed by (workload,
# envs, precision); a workload without a capture of the current kernel reports null.
PCG_DRAM_BYTES_PER_LAUNCH = {("uneven", 1024, "fp64"): 21.154e9}


def roofline(prof, precision, traffic=None):
    kern = {"pcg_solve": "k_pcg_cluster (persistent per-environment PCG, whole solve per launch)",
            "spmv": "k_spmv (PCG matrix-vector product)"}
    solve = "pcg_solve" if prof["pcg_solve"]["launches"] > 0 else "spmv"
    sp = prof[solve]
    if not (sp["ms"] > 0 and sp["launches"] > 0):
        return None
    hbm, hbm_kind = peaks()
    sec = sp["ms"] / 1000.0
    gbs = sp["work"] / sec / 1e9
    flops = prof["pcg_flops"]["work"] if solve == "pcg_solve" else 0.0
    tflops = flops / sec / 1e12
    fp64 = precision == "fp64"
    # ridge point: intensity (flop/B) above peak_flops / peak_bandwidth is arithmetic-bound
    intensity = flops / sp["work"] if sp["work"] > 0 else 0.0
    alu_bound = fp64 and flops > 0 and intensity > FP64_PEAK_TFLOPS * 1e12 / (hbm * 1e9)
    base = {"kernel": kern[solve], "traffic": traffic if solve == "pcg_solve" else None,
            "bytes_per_launch": sp["work"] / sp["launches"],
            "flops_per_launch": flops / sp["launches"], "intensity_flop_per_byte": round(intensity, 4),
            "avg_launch_us": 1000.0 * sp["ms"] / sp["launches"], "launches": sp["launches"],
            "hbm_gbs": round(gbs, 1), "hbm_frac": round(gbs / hbm, 4), "hbm_peak_source": f"{hbm_kind} hbm_gbs"}
    if alu_bound:
        base.update({"bound": "alu", "achieved": round(tflops, 4), "peak": round(FP64_PEAK_TFLOPS, 4),
                     "unit": "TFLOP/s (FP64)", "frac": round(tflops / FP64_PEAK_TFLOPS, 4),
                     "note": "FP64 FMA pipe: peak from 148 SMs x 4 flop/clk x 2.032 GHz"})
    else:
        base.update({"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s", "frac": round(gbs / hbm, 4),
                     "note": "fraction of measured HBM copy bandwidth"})
    return base


# Algorithmic bytes per tet of a Neo-Hookean Hessian evaluation: the tet (int4), its 12
# parameters, env id and 4 gathered nodes in; energy, 12 gradient and 78 Hessian entries out
# (the Hessian in FP32 under mixed precision).
ELASTIC_BYTES_PER_TET = {"fp64": 16 + 96 + 4 + 96 + 8 + 96 + 78 * 8, "mixed": 16 + 96 + 4 + 96 + 8 + 96 + 78 * 4}

# kernels of each profiled family, as the library groups them
FAMILY_KERNELS = {
    "pcg_solve": "k_pcg_cluster (persistent per-environment PCG)",
    "elastic": "k_elastic<HESS> (Neo-Hookean energy, gradient, projected Hessian)",
    "contact": "k_barrier_local + k_barrier_hess + k_friction + k_joint (Hessian evaluations; side stream)",
    "assembly": "stencil incidence sort, k_assemble_grad, k_assemble_bsr, k_precond_soft, k_precond_body",
    "ccd": "step filter: swept-box cover test or collect traversals, k_accd_pairs",
    "broad": "constraint-set collect traversals (k_trav_pt, k_trav_ee)",
}


def kernel_fractions(prof, precision):
    """Achieved algorithmic HBM bandwidth of every profiled kernel family over the timed region:
    the family's algorithmic bytes (counted by the library from each launch's sizes, or on the
    device; elastic: tets x bytes per tet) over the summed CUDA-event time of its launches, and
    that as a fraction of the measured HBM copy rate."""
    hbm, kind = peaks()
    out = {}
    for fam, what in FAMILY_KERNELS.items():
        p = prof.get(fam)
        if not p or p["ms"] <= 0 or p["work"] <= 0:
            continue
        work = p["work"] * (ELASTIC_BYTES_PER_TET[precision] if fam == "elastic" else 1.0)
        gbs = work / (p["ms"] / 1000.0) / 1e9
        out[fam] = {"kernels": what, "launches": int(p["launches"]), "ms": round(p["ms"], 2),
                    "bytes": float(f"{work:.4g}"), "gb_s": round(gbs, 1), "hbm_frac": round(gbs / hbm, 4)}
    out["peak"] = {"hbm_gbs": hbm, "source": f"{kind} hbm_gbs"}
    return out


def cpu_oracle_sample(envs, states, params, n_threads):
    """Time the oracle on n_threads envs x 1 step from the given states (bounded CPU sample)."""
    from oracle import oracle as O

    oe = []
    for env, (x, v, step) in zip(envs, states):
        o = O.OracleEnv(params, env)
        o.set_state(x, v, step)
        oe.append(o)
    t0 = time.perf_counter()
    O.run_batch(oe, 1, n_threads)
    dt = time.perf_counter() - t0
    return len(oe) / dt, len(oe), dt


def timed_steps(sc, stream, k):
    """Device time (ms) of one ipc_step(k) call: CUDA events on the scene's stream."""
    import torch

    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    sc.step(k)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def guarded(leg, *a):
    """Run one secondary leg of the line; an error in it is recorded in its place (the headline
    measurement already taken stays valid and is still printed)."""
    try:
        return leg(*a)
    except Exception as ex:  # noqa: BLE001 - reported in the line, not swallowed
        import traceback

        traceback.print_exc()
        return {"error": f"{type(ex).__name__}: {ex}"}


def budgeted(t_run0, budget, leg, *a):
    """A secondary leg, run through `guarded` unless the run has already spent `budget` seconds
    since `t_run0`; a leg that is not started is recorded as skipped with the time spent."""
    spent = time.perf_counter() - t_run0
    if spent > budget:
        return {"skipped": f"not started: {spent:.0f} s of the run's {budget:.0f} s leg budget spent"}
    return guarded(leg, *a)


def run_ours(args):
    import torch

    t_run0 = time.perf_counter()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    wl = Workload(args.workload)
    ids_global = shard_env_ids(rank, world, args.envs, wl.cost)
    envs = make_envs(wl, ids_global)  # before the first CUDA call
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2503_05020_b300 import ipc

    params = S.scene_params(DT)
    stream = torch.cuda.Stream()  # a non-default stream: the library's kernels and the timing events share it
    torch.cuda.set_stream(stream)
    prec = ipc.MIXED if args.precision == "mixed" else ipc.FP64
    sc = ipc.Scene(params, precision=prec, device=local, stream=stream.cuda_stream, pcg_cluster=args.pcg_cluster)
    ids = [sc.add_env(e) for e in envs]
    for eid, env in zip(ids, envs):
        x, v = wl.state_at(env, wl.start)
        sc.set_state(eid, x, v, wl.start)
    sc.step(args.warmup)
    snap = [(sc.dofs(e), sc.velocities(e), sc.status(e)["step"]) for e in ids]
    # envs that stopped during the warm-up (Newton cap, or their schedule's end) take no part in the
    # later legs: restoring their state would make them active again and repeat their last step
    live = [i for i, e in enumerate(ids) if sc.status(e)["status"] == "ACTIVE"]
    p_start = [sc.points(e) for e in ids]

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    # ---- device-timed region
    clocks = ClockSampler(local)
    sc.profile(True)
    l0 = sc.launch_count()
    st_before = [sc.status(e) for e in ids]
    st0 = [s["steps"] for s in st_before]
    torch.cuda.synchronize()
    barrier()
    clocks.start()
    ms = timed_steps(sc, stream, args.steps)  # one call: every env runs its K steps at its own pace
    barrier()
    clk = clocks.stop()
    launches = sc.launch_count() - l0
    prof = sc.profile_read()
    sc.profile(False)
    stats = [sc.status(e) for e in ids]
    steps_done = sum(s["steps"] for s in stats) - sum(st0)
    failed = sum(s["status"] == "FAILED" for s in stats)
    x_end = [sc.points(e) for e in ids]
    t_max = max_over_ranks(ms, world, "cuda")
    all_steps = sum_over_ranks(steps_done, world, "cuda")
    value = job_throughput(all_steps, t_max / 1000.0)

    # ---- end to end through the public API with host buffers: per step, the next kinematic
    # targets of every env go host -> device and the DOFs of every env come back.
    for i in live:
        x, v, st = snap[i]
        sc.set_state(ids[i], x, v, st)
    n_all = sc.all_dofs_size()
    h_out = torch.empty(n_all, dtype=torch.float64, pin_memory=True).numpy()
    # the next targets of every env for each step (the API takes those of the envs still active)
    rows = [[env["targets"][min(st + k, len(env["targets"]) - 1)].reshape(-1) for env, (_, _, st) in zip(envs, snap)]
            for k in range(args.steps)]
    h_tg = torch.empty(sum(len(r) for r in rows[0]), dtype=torch.float64, pin_memory=True).numpy()
    h2d = 0
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for k in range(args.steps):
        st = sc.all_status()
        act_rows = [r for eid, r in zip(ids, rows[k]) if st[eid][0] == "ACTIVE"]
        n = sum(len(r) for r in act_rows)
        if n:
            h_tg[:n] = np.concatenate(act_rows)
            sc.set_next_targets(h_tg[:n])
        h2d += 8 * n
        sc.step(1)
        sc.all_dofs(h_out)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, "cuda")
    e2e_value = job_throughput(all_steps, e2e_s)
    counters = sc.scene_counters(ids[0])
    # iteration counts of the timed region only (the status counters are cumulative)
    newton = sum(s["newton_iters"] for s in stats) - sum(s["newton_iters"] for s in st_before)
    pcg_its = sum(s["pcg_iters"] for s in stats) - sum(s["pcg_iters"] for s in st_before)
    sc.close()
    del sc

    tets = [sum(len(s["tets"]) for s in e["soft"]) for e in envs]
    plain = mixed = None
    if world == 1 and args.plain_envs > 0:
        plain = budgeted(t_run0, args.leg_budget, plain_leg, args, params, envs, snap, tets, stream, local, value, live)
    if world == 1 and args.precision == "fp64" and not args.no_mixed_leg:
        mixed = budgeted(t_run0, args.leg_budget, mixed_leg, args, params, envs, snap, p_start, x_end, tets, stream,
                         local, t_max / args.steps, {i for i, s_ in enumerate(stats) if s_["status"] == "FAILED"}, live)
        if plain and "value" in plain and "value" in mixed:
            plain["mixed_batched_over_plain"] = round(mixed["value"] / plain["value"], 2)

    if rank != 0:
        if world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()
        return

    # ---- roofline of the dominant kernel: the persistent per-env PCG when it runs, else the
    # tiled SpMV. Its bound is the roof its arithmetic intensity reaches first: FP64 arithmetic
    # (B300 runs FP64 at 1/58 of FP32) or HBM bandwidth.
    roof = roofline(prof, args.precision,
                    PCG_DRAM_BYTES_PER_LAUNCH.get((args.workload, args.envs, args.precision)) if world == 1 else None)

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = budgeted(t_run0, args.leg_budget, cpu_leg, envs, snap, tets, live, params)
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(t_max / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f64+f32",
        "data": "synthetic", "config": wl.config(len(envs), int(np.mean(tets)), world),
        "roofline": roof, "cpu_baseline": cpu,
        "e2e": {"value": round(e2e_value, 2), "unit": UNIT, "h2d_bytes_per_step": int(h2d // max(args.steps, 1)),
                "d2h_bytes_per_step": int(h_out.nbytes)},
        "gpu_launches": int(launches), "clocks": clk, "plain_fp64": plain, "mixed_precision": mixed, "serving": None,
        "env_steps_done": int(steps_done), "envs_failed": int(failed),
        "failed_envs": [{"env": int(ids_global[i]), "tets": int(tets[i]), "reason": stats[i]["reason"],
                         "step": int(stats[i]["step"])} for i in range(len(ids)) if stats[i]["status"] == "FAILED"],
        "profile_ms": {k: round(v["ms"], 2) for k, v in prof.items() if k not in ("pcg_flops", "host_idle")},
        "kernel_roofline": kernel_fractions(prof, args.precision),
        "host_round_trips": {"count": int(prof["host_idle"]["launches"]), "gpu_idle_ms": round(prof["host_idle"]["ms"], 2),
                             "gpu_idle_frac": round(prof["host_idle"]["ms"] / t_max, 4) if t_max > 0 else None,
                             "note": "GPU idle time behind the host reads inside the timed ipc_step call: events "
                                     "before each wait and at the next kernel launch, on the scene's stream"},
        "counters_last_iteration": counters,
        "newton_iters_per_env_step": round(newton / max(steps_done, 1), 2),
        "pcg_iters_per_newton": round(pcg_its / max(newton, 1), 1),
    }
    if world == 1 and args.serve_requests > 0:
        line["serving"] = budgeted(t_run0, args.leg_budget, serving_leg, args, params, local)
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def cpu_leg(envs, snap, tets, live, params):
    """The CPU oracle on the host cores: one env per thread, 1 step each from the timed region's
    start state, on envs of the batch's small end (CPU_SAMPLE_MAX_TETS)."""
    threads = min(os.cpu_count() or 1, 64)
    sel = [live[j] for j in cpu_sample([tets[i] for i in live], threads)]
    v_cpu, n_cpu, dt_cpu = cpu_oracle_sample([envs[i] for i in sel], [snap[i] for i in sel], params, threads)
    return {"value": round(v_cpu, 4), "unit": UNIT, "cores": min(threads, n_cpu), "kind": "oracle",
            "sample": f"{n_cpu} envs at evenly spaced size quantiles among the envs of at most "
                      f"{CPU_SAMPLE_MAX_TETS} tets (tets {min(tets[i] for i in sel)}-{max(tets[i] for i in sel)}; "
                      f"the batch's envs average {int(np.mean(tets))}), 1 step each from the timed region's start "
                      f"state, one env per thread, {dt_cpu:.1f} s wall", **host_info()}


def plain_leg(args, params, envs, snap, tets, stream, device, batched_value, live=None):
    """The plain FP64 GPU stepper: the same kernels, one env at a time (its own scene, automatic
    PCG shape, which for a single env has one candidate and is never tuned), on a sample of the
    envs at evenly spaced size quantiles, each from the timed region's start state for the same
    K steps. Also the paper's comparison (Sec. IV-A): the sample's envs batched in one scene over
    the same envs run one after another."""
    from paper_2503_05020_b300 import ipc

    live = list(range(len(envs))) if live is None else live
    sel = [live[j] for j in stratified([tets[i] for i in live], args.plain_envs)]
    seq_ms, steps = 0.0, 0
    for i in sel:
        sc = ipc.Scene(params, precision=ipc.FP64, device=device, stream=stream.cuda_stream)
        eid = sc.add_env(envs[i])
        x, v, st = snap[i]
        sc.set_state(eid, x, v, st)
        sc.step(0)  # layout outside the timed call
        s0 = sc.status(eid)["steps"]
        seq_ms += timed_steps(sc, stream, args.steps)
        steps += sc.status(eid)["steps"] - s0
        sc.close()
    value = steps / (seq_ms / 1000.0)
    sc = ipc.Scene(params, precision=ipc.FP64, device=device, stream=stream.cuda_stream)
    ids = [sc.add_env(envs[i]) for i in sel]
    for eid, i in zip(ids, sel):
        x, v, st = snap[i]
        sc.set_state(eid, x, v, st)
    sc.step(0)
    s0 = sum(sc.status(e)["steps"] for e in ids)
    b_ms = timed_steps(sc, stream, args.steps)
    b_steps = sum(sc.status(e)["steps"] for e in ids) - s0
    sc.close()
    return {"value": round(value, 2), "unit": UNIT, "envs": len(sel),
            "sample": f"{len(sel)} envs at evenly spaced size quantiles (tets {min(tets[i] for i in sel)}-"
                      f"{max(tets[i] for i in sel)}), {args.steps} steps each from the timed region's start state",
            "batched_over_plain": round(batched_value / value, 2),
            "paper_style_ratio": {"n_envs": len(sel), "batched_ms": round(b_ms, 1), "sequential_ms": round(seq_ms, 1),
                                  "ratio": round((b_steps / b_ms) / (steps / seq_ms), 2),
                                  "paper": "16x (512 envs, LEAP hand), 40x / 48x (400 envs, UMI gripper); "
                                           "1x H100, FP64 (Sec. I, IV-A)"}}


def mixed_leg(args, params, envs, snap, p_start, x_end, tets, stream, device, ms_fp64, failed_fp64=(), live=None):
    """The same K timed steps from the same state with FP32 Hessians and PCG (FP64 energies,
    gradients, barrier, CCD and line search): throughput and speedup over the FP64 run. Accuracy:
    the largest difference of a point's world position from the FP64 run (all points, and the
    grasped objects' points) relative to the largest FP64 point displacement of the run; and on
    a sample of envs, both precisions against a converged FP64 solve of the same steps (PCG to
    1e-10, Newton tolerance x1e-2)."""
    from paper_2503_05020_b300 import ipc

    sc = ipc.Scene(params, precision=ipc.MIXED, device=device, stream=stream.cuda_stream,
                   pcg_cluster=args.pcg_cluster)
    live = list(range(len(envs))) if live is None else live
    ids = [sc.add_env(envs[i]) for i in live]
    for eid, i in zip(ids, live):
        sc.set_state(eid, *snap[i])
    sc.step(1)  # warm-up (tuner, first-call costs), then back to the snapshot
    for eid, i in zip(ids, live):
        sc.set_state(eid, *snap[i])
    sc.profile(True)
    sts0 = [sc.status(e) for e in ids]
    s0 = sum(st["steps"] for st in sts0)
    ms = timed_steps(sc, stream, args.steps)
    prof = sc.profile_read()
    sc.profile(False)
    sts = [sc.status(e) for e in ids]
    steps = sum(st["steps"] for st in sts) - s0
    x_mixed = [None] * len(envs)
    for eid, i in zip(ids, live):
        x_mixed[i] = sc.points(eid)
    failed_m = {i for i, st in zip(live, sts) if st["status"] == "FAILED"}
    failed = len(failed_m)
    newton = sum(st["newton_iters"] for st in sts) - sum(st["newton_iters"] for st in sts0)
    pcg_its = sum(st["pcg_iters"] for st in sts) - sum(st["pcg_iters"] for st in sts0)
    sc.close()

    def errors(xa, xb, rows):
        disp = max(float(np.abs(xb[i] - p_start[i]).max()) for i in rows)
        d_all = max(float(np.abs(xa[i] - xb[i]).max()) for i in rows)
        d_obj = 0.0
        for i in rows:
            o = object_points(envs[i])
            d_obj = max(d_obj, float(np.abs(xa[i][o] - xb[i][o]).max()))
        return {"max_diff_m": d_all, "rel_all_points": d_all / disp if disp > 0 else None,
                "rel_object_points": d_obj / disp if disp > 0 else None, "max_displacement_m": disp}

    # envs that failed in either precision stop at different points: compared only where both ran
    rows = [i for i in live if i not in failed_m and i not in failed_fp64]
    out = {"value": round(steps / (ms / 1000.0), 2), "unit": UNIT, "ms_per_step": round(ms / args.steps, 3),
           "speedup_vs_fp64": round((ms_fp64 * args.steps) / ms, 3), "envs_failed": int(failed),
           "pcg_iters_per_newton": round(pcg_its / max(newton, 1), 1),
           "vs_fp64": dict(errors(x_mixed, x_end, rows), envs_compared=len(rows)),
           "dtype": "f32 Hessians + PCG, f64 energies/gradients/barrier/CCD/line search",
           "roofline": roofline(prof, "mixed"),
           "profile_ms": {k: round(v["ms"], 2) for k, v in prof.items() if k not in ("pcg_flops", "host_idle")}}
    if args.ref_envs > 0:
        sel = [i for i in stratified(tets, args.ref_envs) if i in rows]
        pr = dict(params, pcg_rel_tol=1e-10, newton_tol=params["newton_tol"] * 1e-2, max_pcg=20000)
        sc = ipc.Scene(pr, precision=ipc.FP64, device=device, stream=stream.cuda_stream)
        rid = [sc.add_env(envs[i]) for i in sel]
        for eid, i in zip(rid, sel):
            x, v, st = snap[i]
            sc.set_state(eid, x, v, st)
        sc.step(args.steps)
        x_ref = {i: sc.points(e) for e, i in zip(rid, sel) if sc.status(e)["status"] != "FAILED"}
        sc.close()
        sel = sorted(x_ref)
        xr = [x_ref.get(i) for i in range(len(envs))]
        out["vs_converged_fp64"] = {"envs": len(sel), "mixed": errors(x_mixed, xr, sel),
                                    "fp64": errors(x_end, xr, sel)}
    return out


def object_points(env):
    """Indices of the grasped object's points among an env's points (soft vertices in body order,
    then the affine bodies' rest vertices)."""
    kind, k = env.get("object", ("soft", len(env["soft"]) - 1))
    if kind == "soft":
        o = sum(len(s["verts"]) for s in env["soft"][:k])
        return np.arange(o, o + len(env["soft"][k]["verts"]))
    o = sum(len(s["verts"]) for s in env["soft"]) + sum(len(a["verts"]) for a in env["affine"][:k])
    return np.arange(o, o + len(env["affine"][k]["verts"]))


SERVE_BUDGET = 180 * 10 ** 9  # HBM admission budget of the serving configuration (bytes)


def serving_leg(args, params, device):
    """Grasp-evaluation serving (the serving configuration): seeded Poisson streams of requests,
    each the plate squeeze or the soft-pad grasp of a soft object of log-uniform 1k-100k tets
    (close, lift 5 cm, shake +/-15 deg at 2 Hz, hold still; 200 steps), served by continuous
    batching on one device-resident scene admitted under a 180 GB HBM budget, at several arrival
    rates, in FP64 and in mixed precision. Per rate: throughput, p50/p99 latency and queue wait.
    Per request: the stability label of Sec. III-D at its last step, in both precisions; and, on a
    subset, the final object points of both precisions against a converged FP64 run of the same
    requests. A request's result does not depend on the rate (each env does exactly the work it
    does alone), so labels and points are taken from the first rate."""
    from paper_2503_05020_b300 import ipc
    from paper_2503_05020_b300.serve import GraspServer, Request, object_points, poisson_arrivals

    n = args.serve_requests
    rates = [float(r) for r in args.serve_rates.split(",")]
    envs = [S.serving_request_env(i) for i in range(n)]
    tets = [sum(len(s["tets"]) for s in e["soft"]) for e in envs]
    out = {"requests_per_rate": n, "rates_req_s": rates, "steps_per_request": len(envs[0]["targets"]),
           "hbm_budget_bytes": SERVE_BUDGET, "object_tets": [min(tets), max(tets)],
           "request": "plate squeeze or soft-pad grasp of a soft object (log-uniform 1k-100k tets): close 70 "
                      "steps, lift 5 cm in 50, shake +/-15 deg at 2 Hz for 60, hold 20; dt 5 ms",
           "per_rate": {}}
    results = {}
    for name, prec in (("fp64", ipc.FP64), ("mixed", ipc.MIXED)):
        for k, rate in enumerate(rates):
            reqs = [Request(i, e, t) for i, (e, t) in enumerate(zip(envs, poisson_arrivals(rate, n, 20250306)))]
            srv = GraspServer(params, precision=prec, device=device, hbm_budget_bytes=SERVE_BUDGET, max_envs=1024,
                              admit_period=8, steps_per_call=8)
            rep = srv.run(reqs)
            rec = {kk: (round(v, 4) if isinstance(v, float) else v) for kk, v in rep.items()}
            rec["stable"] = int(sum(bool(r.result.get("stable")) for r in reqs))
            out["per_rate"].setdefault(str(rate), {})[name] = rec
            if k == 0:
                results[name] = {r.rid: dict(r.result, status=r.status) for r in reqs}
            srv.scene.close()
    lab = {nm: [bool(results[nm][i].get("stable")) for i in range(n)] for nm in results}
    out["stable_labels"] = lab
    out["request_status"] = {nm: [results[nm][i].get("status") for i in range(n)] for nm in results}
    out["labels_agree"] = lab["fp64"] == lab["mixed"]
    hi = str(rates[-1])
    out["mixed_over_fp64_throughput"] = round(out["per_rate"][hi]["mixed"]["env_steps_s"]
                                              / out["per_rate"][hi]["fp64"]["env_steps_s"], 3)
    # converged FP64 reference of a subset: its final object points against both precisions,
    # relative to the object's largest point displacement over the request
    sub = stratified(tets, min(args.serve_ref, n))
    pr = dict(params, pcg_rel_tol=1e-10, newton_tol=params["newton_tol"] * 1e-2, max_pcg=20000)
    sc = ipc.Scene(pr, precision=ipc.FP64, device=device)
    ids = [sc.add_env(envs[i]) for i in sub]
    sc.step(len(envs[0]["targets"]))
    from paper_2503_05020_b300.serve import initial_points

    per_req = []
    for eid, i in zip(ids, sub):
        st = sc.status(eid)["status"]
        rec = {"request": i, "tets": tets[i], "converged_status": st,
               "status": {nm: results[nm][i].get("status") for nm in results}}
        if st == "DONE" and all(v == "DONE" for v in rec["status"].values()):
            ref = sc.points(eid)
            sl = object_points(envs[i])
            p0 = initial_points(envs[i])
            disp = float(np.abs(ref[sl] - p0[sl]).max())
            disp_all = float(np.abs(ref - p0).max())
            for nm in results:
                pts = results[nm][i]["points"]
                rec[nm] = {"rel_object_points": float(np.abs(pts[sl] - ref[sl]).max()) / disp,
                           "rel_all_points": float(np.abs(pts - ref).max()) / disp_all}
        per_req.append(rec)
    sc.close()
    out["vs_converged_fp64"] = {"per_request": per_req,
                                "note": "largest point difference at the request's end over the largest point "
                                        "displacement of the converged run (PCG 1e-10, Newton tolerance x1e-2); "
                                        "requests that failed in any run are not compared"}
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", 0))
    if rank != 0:
        return
    from oracle import oracle as O

    wl = Workload(args.workload)
    params = S.scene_params(DT)
    threads = min(os.cpu_count() or 1, 64)
    # the workload's config is the GPU arm's (all its envs); the timed sample is one env per core
    # at evenly spaced size quantiles among the batch's small envs
    all_envs = make_envs(wl, list(range(args.envs)))
    all_tets = [sum(len(s["tets"]) for s in e["soft"]) for e in all_envs]
    sel = cpu_sample(all_tets, threads)
    envs = [all_envs[i] for i in sel]
    oe = []
    for env in envs:
        o = O.OracleEnv(params, env)
        x, v = wl.state_at(env, wl.start)
        o.set_state(x, v, wl.start)
        oe.append(o)
    t_start = time.perf_counter()
    for _ in range(min(args.warmup, 1)):
        O.run_batch(oe, 1, threads)
    done, t_timed = 0, 0.0
    for _ in range(args.steps):
        if time.perf_counter() - t_start > args.cpu_budget and done > 0:
            break
        t0 = time.perf_counter()
        O.run_batch(oe, 1, threads)
        t_timed += time.perf_counter() - t0
        done += 1
    value = len(oe) * done / t_timed
    tets = [sum(len(s["tets"]) for s in e["soft"]) for e in envs]
    line = {"metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": 0, "steps": done,
            "warmup": min(args.warmup, 1), "ms_per_step": round(1000 * t_timed / max(done, 1), 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": wl.config(args.envs, int(np.mean(all_tets)), 1), "impl": "reference",
            "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": min(threads, len(oe)), "kind": "oracle",
                             "sample": f"{len(oe)} of the {args.envs} envs at evenly spaced size quantiles among the "
                                       f"envs of at most {CPU_SAMPLE_MAX_TETS} tets (tets {min(tets)}-{max(tets)}; the "
                                       f"batch's envs average {int(np.mean(all_tets))}), {done} of {args.steps} steps "
                                       f"(budget {args.cpu_budget:.0f} s), one env per thread", **host_info()},
            "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
