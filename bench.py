"""Benchmark: IPC sim-steps per second summed over environments.

Workload (N=1): 64 pad-grasp environments (two soft wedge finger pads of ~5k Neo-Hookean tets
each squeezing a rigid affine-body convex hull of 1584 triangles, dt = 5 ms, FP64), stepped as
one batch through the C ABI. Every run starts from the same synthetic contact-phase state
(pads placed where the closing schedule puts them at step 20, 0.8 mm from the object), does W
untimed steps and times K steps of every env. A "step" is one ipc_step over the whole batch:
every active env advances one time step (its full Newton loop).

Under torchrun every rank runs its own 64 envs (seeds offset by rank): independent replicas,
weak scaling, no collective on the data path; the rank times are combined by max.

--impl reference times the CPU oracle (plain FP64, no GPU) on a bounded sample of the same
workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2503_05020_b300 import scenes as S  # noqa: E402

METRIC = "IPC sim-steps/s summed over envs"
UNIT = "env-steps/s"
START_STEP = 20
DT = 0.005


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--envs", type=int, default=64)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--pcg-cluster", type=int, default=0,
                    help="PCG launch shape: 0 automatic, 1/2/4/8 CTAs per env cluster, -1 tiled multi-launch")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=24, help="requests of the serving leg (0: none)")
    ap.add_argument("--serve-rate", type=float, default=1.5, help="Poisson arrival rate of the serving leg (1/s)")
    ap.add_argument("--no-mixed-leg", action="store_true",
                    help="skip the mixed-precision run of the same steps that the FP64 line reports beside it")
    ap.add_argument("--cpu-budget", type=float, default=150.0, help="seconds of oracle time for --impl reference")
    return ap.parse_args()


def workload_config(n_env, tets, start):
    return {"workload": f"pad-grasp x{n_env} envs (2 soft pads ~5k tets each + rigid hull 1584 tris), "
                        f"dt={DT}s, FP64, from schedule step {start}",
            "envs_per_gpu": n_env, "tets_per_env_avg": tets, "start_step": start,
            "schedule": "close 100 steps (gravity off) then lift 0.1 m (gravity on)",
            "l2": "inputs larger than L2 (BSR + element buffers of the batch exceed 126 MB)",
            "parallelism": "replicas"}


def shard_env_ids(rank, n_env):
    """Env seeds of one rank: rank r steps envs r*n .. r*n + n - 1 (independent replicas with
    disjoint envs; the batch shards across ranks with no data-path collective)."""
    return [rank * n_env + i for i in range(n_env)]


def make_envs(rank, n_env):
    return [S.pad_grasp_env(i) for i in shard_env_ids(rank, n_env)]


def max_over_ranks(v, world, device):
    """The largest value over the ranks: a run's time is its slowest rank's."""
    if world <= 1:
        return float(v)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, n_env, steps, seconds):
    """Whole-job env-steps/s: the envs and steps of every rank over the slowest rank's time."""
    return world * n_env * steps / seconds


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


# FP64 peak of one B300 from its unit counts and clock: 148 SMs x 4 FP64 flop/clk (2 DFMA) x
# 2.032 GHz (1.25 TFLOP/s nominal at the boost clock; 1.11 measured by an FMA loop at 2032 MHz).
FP64_PEAK_TFLOPS = 148 * 4 * 2.032e9 / 1e12


def roofline(prof, precision):
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
    base = {"kernel": kern[solve], "traffic": None, "bytes_per_launch": sp["work"] / sp["launches"],
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


def cpu_oracle_sample(envs, states, params, n_threads):
    """Time the oracle on n_threads envs x 1 step from the given states (bounded CPU sample)."""
    from oracle import oracle as O

    sel = list(range(min(n_threads, len(envs))))
    oe = []
    for i in sel:
        o = O.OracleEnv(params, envs[i])
        x, v, step = states[i]
        o.set_state(x, v, step)
        oe.append(o)
    t0 = time.perf_counter()
    O.run_batch(oe, 1, len(oe))
    dt = time.perf_counter() - t0
    return len(oe) / dt, len(oe), dt


def run_ours(args):
    import torch

    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2503_05020_b300 import ipc

    params = S.scene_params(DT)
    envs = make_envs(rank, args.envs)
    stream = torch.cuda.Stream()  # a non-default stream: the library's kernels and the timing events share it
    torch.cuda.set_stream(stream)
    prec = ipc.MIXED if args.precision == "mixed" else ipc.FP64
    sc = ipc.Scene(params, precision=prec, device=local, stream=stream.cuda_stream, pcg_cluster=args.pcg_cluster)
    ids = [sc.add_env(e) for e in envs]
    for eid, env in zip(ids, envs):
        x, v = S.pad_grasp_state_at(env, START_STEP)
        sc.set_state(eid, x, v, START_STEP)
    sc.step(args.warmup)
    snap = [(sc.dofs(e), sc.velocities(e), sc.status(e)["step"]) for e in ids]
    p_start = [sc.points(e) for e in ids]

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    # ---- device-timed region
    clocks = ClockSampler(local)
    sc.profile(True)
    l0 = sc.launch_count()
    torch.cuda.synchronize()
    barrier()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sc.step(args.steps)  # one call: every env runs its K steps at its own pace
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    launches = sc.launch_count() - l0
    ms = e0.elapsed_time(e1)
    prof = sc.profile_read()
    sc.profile(False)
    steps_done = sum(sc.status(e)["steps"] for e in ids)
    failed = sum(sc.status(e)["status"] == "FAILED" for e in ids)
    x_end = [sc.points(e) for e in ids]
    t_max = max_over_ranks(ms, world, "cuda")
    value = job_throughput(world, args.envs, args.steps, t_max / 1000.0)

    # ---- end to end through the public API with host buffers: per step, the next kinematic
    # targets of every env go host -> device and the DOFs of every env come back.
    for eid, (x, v, st) in zip(ids, snap):
        sc.set_state(eid, x, v, st)
    n_all = sc.all_dofs_size()
    h_out = torch.empty(n_all, dtype=torch.float64, pin_memory=True).numpy()
    tg_all = []
    for k in range(args.steps):
        tg_all.append(np.concatenate([env["targets"][min(st + k, len(env["targets"]) - 1)].reshape(-1)
                                      for env, (_, _, st) in zip(envs, snap)]))
    h_tg = torch.empty(len(tg_all[0]), dtype=torch.float64, pin_memory=True).numpy()
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for k in range(args.steps):
        h_tg[:] = tg_all[k]
        sc.set_next_targets(h_tg)
        sc.step(1)
        sc.all_dofs(h_out)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, "cuda")
    e2e_value = job_throughput(world, args.envs, args.steps, e2e_s)

    mixed = None
    if world == 1 and args.precision == "fp64" and not args.no_mixed_leg:
        mixed = mixed_leg(args, params, envs, snap, p_start, x_end, stream, local, t_max / args.steps)

    if rank != 0:
        if world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()
        return

    # ---- roofline of the dominant kernel: the persistent per-env PCG when it runs, else the
    # tiled SpMV. Its bound is the roof its arithmetic intensity reaches first: FP64 arithmetic
    # (B300 runs FP64 at 1/58 of FP32) or HBM bandwidth.
    fam = max(prof, key=lambda k: prof[k]["ms"])
    roof = roofline(prof, args.precision)
    tets = int(np.mean([sum(len(s["tets"]) for s in e["soft"]) for e in envs]))

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        threads = min(os.cpu_count() or 1, 8)
        v_cpu, n_cpu, dt_cpu = cpu_oracle_sample(envs, snap, params, threads)
        cpu = {"value": round(v_cpu, 4), "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{n_cpu} envs x 1 step from the timed region's start state, one env per thread, "
                         f"{dt_cpu:.1f} s wall"}
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(t_max / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f64+f32",
        "data": "synthetic", "config": workload_config(args.envs, tets, START_STEP),
        "roofline": roof, "cpu_baseline": cpu,
        "e2e": {"value": round(e2e_value, 2), "unit": UNIT, "h2d_bytes_per_step": int(h_tg.nbytes),
                "d2h_bytes_per_step": int(h_out.nbytes)},
        "gpu_launches": int(launches), "clocks": clk, "mixed_precision": mixed, "serving": None,
        "env_steps_done": int(steps_done), "envs_failed": int(failed),
        "profile_ms": {k: round(v["ms"], 2) for k, v in prof.items() if k != "pcg_flops"},
        "counters_last_iteration": sc.scene_counters(ids[0]),
        "newton_iters_per_env_step": round(sum(sc.status(e)["newton_iters"] for e in ids) / max(steps_done, 1), 2),
        "pcg_iters_per_newton": round(sum(sc.status(e)["pcg_iters"] for e in ids)
                                      / max(sum(sc.status(e)["newton_iters"] for e in ids), 1), 1),
    }
    if world == 1 and args.serve_requests > 0:
        line["serving"] = serving_leg(args, params, local)
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def mixed_leg(args, params, envs, snap, p_start, x_end, stream, device, ms_fp64):
    """The same K timed steps from the same state with FP32 Hessians and PCG (FP64 energies,
    gradients, barrier, CCD and line search): throughput, speedup over the FP64 run, and the
    largest difference of a point's world position from the FP64 run (all points, and the
    grasped objects' points) relative to the largest FP64 point displacement of the run."""
    import torch

    from paper_2503_05020_b300 import ipc

    sc = ipc.Scene(params, precision=ipc.MIXED, device=device, stream=stream.cuda_stream,
                   pcg_cluster=args.pcg_cluster)
    ids = [sc.add_env(e) for e in envs]
    for eid, env in zip(ids, envs):
        x, v = S.pad_grasp_state_at(env, START_STEP)
        sc.set_state(eid, x, v, START_STEP)
    sc.step(args.warmup)
    for eid, (x, v, st) in zip(ids, snap):
        sc.set_state(eid, x, v, st)
    sc.profile(True)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sc.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    prof = sc.profile_read()
    sc.profile(False)
    # world positions of every point (soft vertices, then the object's vertices)
    diff = max(float(np.abs(sc.points(e) - x).max()) for e, x in zip(ids, x_end))
    disp = max(float(np.abs(x - x0).max()) for x, x0 in zip(x_end, p_start))
    obj_diff = 0.0
    for e, x, env in zip(ids, x_end, envs):
        o = sum(len(s["verts"]) for s in env["soft"])
        obj_diff = max(obj_diff, float(np.abs(sc.points(e)[o:] - x[o:]).max()))
    failed = sum(sc.status(e)["status"] == "FAILED" for e in ids)
    value = args.envs * args.steps / (ms / 1000.0)
    return {"value": round(value, 2), "unit": UNIT, "ms_per_step": round(ms / args.steps, 3),
            "speedup_vs_fp64": round((ms_fp64 * args.steps) / ms, 3), "max_displacement_diff_m": diff,
            "rel_displacement_diff": diff / disp if disp > 0 else None,
            "rel_object_displacement_diff": obj_diff / disp if disp > 0 else None, "envs_failed": int(failed),
            "dtype": "f32 Hessians + PCG, f64 energies/gradients/barrier/CCD/line search",
            "roofline": roofline(prof, "mixed"),
            "profile_ms": {k: round(v["ms"], 2) for k, v in prof.items() if k != "pcg_flops"}}


def serving_leg(args, params, device):
    """Grasp-evaluation serving: a seeded Poisson stream of requests (one pad grasp each: close,
    lift 0.1 m, shake +/-15 deg at 2 Hz; 200 steps; seeded objects of uneven size) served by
    continuous batching on one device-resident scene, in FP64 and in mixed precision."""
    from paper_2503_05020_b300 import ipc
    from paper_2503_05020_b300.serve import GraspServer, Request, poisson_arrivals

    n = args.serve_requests
    envs = [S.grasp_request_env(5000 + i) for i in range(n)]
    arrivals = poisson_arrivals(args.serve_rate, n, 20250306)
    out = {"requests": n, "rate_req_s": args.serve_rate, "steps_per_request": len(envs[0]["targets"]),
           "request": "pad grasp: close 80 steps, lift 0.1 m in 60, shake +/-15 deg at 2 Hz for 60; dt 5 ms"}
    for name, prec in (("fp64", ipc.FP64), ("mixed", ipc.MIXED)):
        reqs = [Request(i, e, t) for i, (e, t) in enumerate(zip(envs, arrivals))]
        srv = GraspServer(params, precision=prec, device=device, max_envs=64, admit_period=8, steps_per_call=8)
        rep = srv.run(reqs)
        held = [bool(r.result.get("held")) for r in reqs]
        out[name] = {k: (round(v, 4) if isinstance(v, float) else v) for k, v in rep.items()}
        out[name]["held"] = int(sum(held))
        out.setdefault("held_labels", {})[name] = held
        del srv
    lab = out.pop("held_labels")
    out["grasp_labels_agree"] = lab["fp64"] == lab["mixed"]
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", 0))
    if rank != 0:
        return
    from oracle import oracle as O

    params = S.scene_params(DT)
    threads = min(os.cpu_count() or 1, 8)
    envs = make_envs(0, threads)
    oe = []
    for env in envs:
        o = O.OracleEnv(params, env)
        x, v = S.pad_grasp_state_at(env, START_STEP)
        o.set_state(x, v, START_STEP)
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
    # the workload's config is the GPU arm's (all its envs); the timed sample is its first envs
    tets = int(np.mean([sum(len(s["tets"]) for s in e["soft"]) for e in make_envs(0, args.envs)]))
    line = {"metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": 0, "steps": done,
            "warmup": min(args.warmup, 1), "ms_per_step": round(1000 * t_timed / max(done, 1), 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args.envs, tets, START_STEP), "impl": "reference",
            "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{len(oe)} of the {args.envs} envs, {done} of {args.steps} steps "
                                       f"(budget {args.cpu_budget:.0f} s), one env per thread"},
            "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
