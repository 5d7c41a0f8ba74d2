"""Serving form: grasp-evaluation requests stepped by continuous batching on one GPU.

A request is one environment with its whole schedule (Sec. III-D's evaluation protocol: close,
lift, optionally shake) and an arrival time. The server keeps one device-resident scene. At step
boundaries it admits requests that have arrived, in arrival order, while the scene's HBM budget
(checked by the library on ipc_env_add from each environment's estimated bytes) and the slot cap
allow; admitted environments join the running batch (Sec. III-A: every environment keeps its own
state, step size, stopping test and failure). Each call of ipc_step advances every running
environment `steps_per_call` time steps, each at its own pace: inside the call an environment
that has finished a step starts the next one while slower ones still iterate. A finished
environment (DONE or FAILED) is read back at the end of that call; it leaves the scene at the
next admission round, so one relayout of the batch serves both its departure and new arrivals.
Relayouts are spaced at least `admit_period` batch steps apart while environments are running.

Latency of a request = time its result was read back - its arrival time; the report gives p50
and p99 over requests, throughput in requests/s and environment-steps/s, and per-request queue
wait. The loop itself is thin host code over the C ABI: every step of the simulation runs in the
library's kernels.
"""
from __future__ import annotations

import math
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import ipc


@dataclass
class Request:
    rid: int
    env: dict
    arrival: float  # seconds after the start of the run
    # filled in by the server
    admitted: float | None = None
    finished: float | None = None
    status: str | None = None
    reason: str | None = None
    steps: int = 0
    result: dict = field(default_factory=dict)

    @property
    def latency(self) -> float | None:
        return None if self.finished is None else self.finished - self.arrival


def poisson_arrivals(rate: float, n: int, seed: int) -> list[float]:
    """n arrival times of a Poisson process of the given rate (1/s), from a SplitMix64 stream."""
    from .scenes import SplitMix64

    rng = SplitMix64(seed)
    t, out = 0.0, []
    for _ in range(n):
        u = rng.uniform(0.0, 1.0)
        t += -math.log(max(1.0 - u, 1e-300)) / rate
        out.append(t)
    return out


def percentile(values, q: float) -> float | None:
    v = sorted(values)
    if not v:
        return None
    k = min(len(v) - 1, max(0, int(math.ceil(q / 100.0 * len(v))) - 1))  # nearest rank
    return v[k]


def object_points(env: dict) -> slice | None:
    """Rows of the grasped object (env["object"] = ("soft" | "affine", index)) in the point list:
    soft bodies' vertices first, then each affine body's vertices."""
    if "object" not in env:
        return None
    kind, idx = env["object"]
    if kind == "soft":
        o = sum(len(s["verts"]) for s in env["soft"][:idx])
        return slice(o, o + len(env["soft"][idx]["verts"]))
    o = sum(len(s["verts"]) for s in env["soft"]) + sum(len(a["verts"]) for a in env["affine"][:idx])
    return slice(o, o + len(env["affine"][idx]["verts"]))


def initial_points(env: dict) -> np.ndarray:
    """World positions of every point at the env's initial state: soft vertices, then each
    affine body's rest vertices mapped by its q0 (x = p + A X, A's columns q0[3:6], [6:9], [9:12])."""
    parts = [np.asarray(s["verts"], dtype=np.float64) for s in env["soft"]]
    for a in env["affine"]:
        q = np.asarray(a["q0"], dtype=np.float64)
        A = np.stack([q[3:6], q[6:9], q[9:12]], axis=1)
        parts.append(q[:3] + np.asarray(a["verts"], dtype=np.float64) @ A.T)
    return np.concatenate(parts, axis=0)


def object_handle(env: dict) -> int | None:
    """Body handle of the grasped object (soft bodies first, then affine bodies)."""
    if "object" not in env:
        return None
    kind, idx = env["object"]
    return idx if kind == "soft" else len(env["soft"]) + idx


def com_velocity(env: dict, v: np.ndarray) -> np.ndarray:
    """Velocity of the grasped object's centre of mass (the mean of its points) from the env's DOF
    rates: a soft object's vertex rates, or for an affine object p' + A' xbar averaged over its
    rest vertices."""
    kind, idx = env["object"]
    if kind == "soft":
        o = sum(len(s["verts"]) for s in env["soft"][:idx])
        return v[3 * o: 3 * (o + len(env["soft"][idx]["verts"]))].reshape(-1, 3).mean(axis=0)
    o = 3 * sum(len(s["verts"]) for s in env["soft"]) + 12 * idx
    q = v[o: o + 12]
    xb = np.asarray(env["affine"][idx]["verts"], dtype=np.float64).mean(axis=0)
    return q[:3] + xb[0] * q[3:6] + xb[1] * q[6:9] + xb[2] * q[9:12]


def object_result(env: dict, points: np.ndarray, points0: np.ndarray, v: np.ndarray | None = None,
                  handles: np.ndarray | None = None, eps_v: float = 0.0, dt: float = 0.0,
                  stable_factor: float = 1.0) -> dict:
    """Grasp outcome: mean displacement of the grasped object's points, whether it rose by more
    than half the schedule's lift, and the stability label of Sec. III-D at the last step (the
    object touches another body, and its centre of mass moved less than stable_factor * eps_v * dt
    in that step; the motion is dt times the centre's velocity, v = (x - x^t) / dt)."""
    sl = object_points(env)
    if sl is None or points0 is None:
        return {}
    disp = (points[sl] - points0[sl]).mean(axis=0)
    lift = float(env.get("lift", 0.0))
    out = {"object_disp": disp.tolist(), "held": bool(lift > 0 and disp[2] > 0.5 * lift)}
    if v is not None and handles is not None:
        obj = object_handle(env)
        in_contact = any((int(a) == obj) != (int(b) == obj) for a, b in handles)
        com_step = float(np.linalg.norm(com_velocity(env, v))) * dt
        out.update({"in_contact": bool(in_contact), "com_step": com_step,
                    "stable": bool(in_contact and com_step < stable_factor * eps_v * dt)})
    return out


class GraspServer:
    def __init__(self, params: dict, precision: int = ipc.FP64, hbm_budget_bytes: int = 0, max_envs: int = 64,
                 admit_period: int = 8, steps_per_call: int = 1, device: int = 0, scene=None, clock=None, sleep=None):
        self.scene = scene if scene is not None else ipc.Scene(params, precision=precision, device=device,
                                                             hbm_budget_bytes=hbm_budget_bytes)
        self.max_envs = max_envs
        self.admit_period = max(1, admit_period)
        self.steps_per_call = max(1, steps_per_call)
        self.clock = clock or time.perf_counter
        self.sleep = sleep or time.sleep
        self.eps_v, self.dt = params.get("eps_v", 0.0), params.get("dt", 0.0)
        self.batch_steps = 0
        self.env_steps = 0
        self.relayouts = 0
        self.max_active = 0

    def run(self, requests: list[Request]) -> dict:
        sc = self.scene
        pending = deque(sorted(requests, key=lambda r: (r.arrival, r.rid)))
        active: dict[int, Request] = {}  # env id -> request, still stepping
        done_in_scene: list[int] = []  # finished env ids not yet removed
        start_pts: dict[int, np.ndarray] = {}
        last_step: dict[int, int] = {}  # env id -> its step count at the last read-back
        t0 = self.clock()
        since_relayout = self.admit_period
        while pending or active:
            now = self.clock() - t0
            arrived = bool(pending) and pending[0].arrival <= now
            if (not active) or (since_relayout >= self.admit_period and (arrived or done_in_scene)):
                changed = False
                for eid in done_in_scene:
                    sc.remove_env(eid)
                    changed = True
                done_in_scene.clear()
                while pending and pending[0].arrival <= now and len(active) < self.max_envs:
                    req = pending[0]
                    try:
                        eid = sc.add_env(req.env)
                    except ipc.IpcError as e:
                        if e.status == ipc.STATUS_CODES["ERR_BUDGET"] and active:
                            break  # waits for memory to free up
                        pending.popleft()
                        req.status, req.reason, req.finished = "REJECTED", str(e), now
                        continue
                    pending.popleft()
                    req.admitted = now
                    active[eid] = req
                    last_step[eid] = 0
                    # host-side (no relayout per admission); only what the grasp outcome needs
                    start_pts[eid] = initial_points(req.env) if "object" in req.env else None
                    changed = True
                if changed:
                    self.relayouts += 1
                    since_relayout = 0
            if not active:
                if pending:
                    self.sleep(max(0.0, pending[0].arrival - (self.clock() - t0)))
                continue
            self.max_active = max(self.max_active, len(active))
            n = self.steps_per_call
            sc.step(n)
            self.batch_steps += n
            since_relayout += n
            status = sc.all_status()
            t_now = self.clock() - t0
            for eid in list(active):
                st, reason, step = status[eid]
                self.env_steps += step - last_step[eid]
                last_step[eid] = step
                if st in ("DONE", "FAILED"):
                    req = active.pop(eid)
                    req.finished, req.status, req.reason, req.steps = t_now, st, reason, step
                    pts = sc.points(eid)
                    req.result = {"dofs": sc.dofs(eid), "points": pts,
                                  **object_result(req.env, pts, start_pts.pop(eid))}
                    if "object" in req.env and hasattr(sc, "grasp_result"):
                        req.result.update(sc.grasp_result(eid))  # the library's Sec. III-D label
                    done_in_scene.append(eid)
        for eid in done_in_scene:
            sc.remove_env(eid)
        wall = self.clock() - t0
        lat = [r.latency for r in requests if r.status in ("DONE", "FAILED")]
        wait = [r.admitted - r.arrival for r in requests if r.admitted is not None]
        return {"requests": len(requests), "completed": sum(r.status == "DONE" for r in requests),
                "failed": sum(r.status == "FAILED" for r in requests),
                "rejected": sum(r.status == "REJECTED" for r in requests), "wall_s": wall,
                "p50_latency_s": percentile(lat, 50), "p99_latency_s": percentile(lat, 99),
                "mean_latency_s": float(np.mean(lat)) if lat else None,
                "p50_wait_s": percentile(wait, 50), "p99_wait_s": percentile(wait, 99),
                "throughput_req_s": len(lat) / wall if wall > 0 else None,
                "env_steps_s": self.env_steps / wall if wall > 0 else None, "batch_steps": self.batch_steps,
                "relayouts": self.relayouts, "max_active": self.max_active}
