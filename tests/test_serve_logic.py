"""Host logic of the serving loop (no GPU): a fake scene with the library's admission contract
(ipc_env_add fails with ERR_BUDGET when the scene's HBM budget is exhausted) and a simulated
clock. Checks arrival-order admission, continuous batching (a request joins while others run),
budget waits, rejection of a request that can never fit, relayout spacing, and latency
accounting."""
import math

import numpy as np

from paper_2503_05020_b300 import ipc
from paper_2503_05020_b300.serve import GraspServer, Request, percentile, poisson_arrivals


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 0.0)


class FakeScene:
    """Each env finishes after env["steps"] batch steps; a batch step costs 0.1 s of fake time."""

    def __init__(self, clock, budget=math.inf):
        self.clock, self.budget, self.used = clock, budget, 0.0
        self.envs, self.next_id, self.log = {}, 0, []

    def add_env(self, env):
        if env["bytes"] > self.budget:
            raise ipc.IpcError(ipc.STATUS_CODES["ERR_BUDGET"], "larger than the budget")
        if self.used + env["bytes"] > self.budget:
            raise ipc.IpcError(ipc.STATUS_CODES["ERR_BUDGET"], "budget")
        eid = self.next_id
        self.next_id += 1
        self.used += env["bytes"]
        self.envs[eid] = {"env": env, "step": 0}
        self.log.append(("add", env["name"], self.clock()))
        return eid

    def remove_env(self, eid):
        self.used -= self.envs[eid]["env"]["bytes"]
        self.log.append(("remove", self.envs[eid]["env"]["name"], self.clock()))
        del self.envs[eid]

    def step(self, n=1):
        for _ in range(n):
            for e in self.envs.values():
                if e["step"] < e["env"]["steps"]:
                    e["step"] += 1
            self.clock.t += 0.1

    def all_status(self):
        return {k: ("DONE" if e["step"] >= e["env"]["steps"] else "ACTIVE", "none", e["step"])
                for k, e in self.envs.items()}

    def points(self, eid):
        return np.full((1, 3), float(self.envs[eid]["step"]))

    def dofs(self, eid):
        return np.full(3, float(self.envs[eid]["step"]))


def env(name, steps, nbytes=1.0):
    return {"name": name, "steps": steps, "bytes": nbytes, "soft": [], "affine": []}


def serve(reqs, budget=math.inf, max_envs=64, admit_period=1, steps_per_call=1):
    clk = FakeClock()
    sc = FakeScene(clk, budget)
    srv = GraspServer({}, scene=sc, clock=clk, sleep=clk.sleep, max_envs=max_envs, admit_period=admit_period,
                      steps_per_call=steps_per_call)
    return srv, sc, srv.run(reqs)


def test_continuous_batching_joins_running_batch_and_accounts_latency():
    reqs = [Request(0, env("a", 10), 0.0), Request(1, env("b", 5), 0.35), Request(2, env("c", 3), 5.0)]
    srv, sc, rep = serve(reqs)
    assert rep["completed"] == 3 and rep["rejected"] == 0
    a, b, c = reqs
    assert b.admitted < a.finished  # b joined while a was running
    assert abs(a.latency - 1.0) < 1e-9  # 10 steps of 0.1 s from t = 0
    assert b.steps == 5 and abs(b.finished - (b.admitted + 0.5)) < 0.11
    assert c.admitted >= 5.0  # the idle server waits for the late arrival
    assert rep["max_active"] == 2
    assert rep["p50_latency_s"] == percentile([r.latency for r in reqs], 50)


def test_budget_admits_in_arrival_order_and_waits_for_memory():
    reqs = [Request(i, env(f"r{i}", 4, nbytes=1.0), 0.0) for i in range(4)]
    big = Request(9, env("big", 4, nbytes=5.0), 0.0)
    srv, sc, rep = serve(reqs + [big], budget=2.0)
    assert rep["completed"] == 4 and rep["rejected"] == 1 and big.status == "REJECTED"
    assert rep["max_active"] == 2
    adds = [name for kind, name, _ in sc.log if kind == "add"]
    assert adds == ["r0", "r1", "r2", "r3"]
    assert reqs[2].admitted >= reqs[0].finished  # waited for a slot of memory


def test_relayouts_are_spaced_by_the_admission_period():
    reqs = [Request(i, env(f"r{i}", 20), 0.1 * i) for i in range(10)]
    srv, sc, rep = serve(reqs, admit_period=8)
    assert rep["completed"] == 10
    adds = sorted(t for kind, _, t in sc.log if kind == "add")
    rounds = sorted(set(round(t, 6) for t in adds))
    assert all(b - a >= 0.8 - 1e-9 for a, b in zip(rounds, rounds[1:]))  # >= 8 steps of 0.1 s apart
    assert rep["relayouts"] >= len(rounds)  # every admission round relayouts the batch once


def test_percentile_nearest_rank_and_poisson_arrivals():
    v = list(range(1, 101))
    assert percentile(v, 50) == 50 and percentile(v, 99) == 99 and percentile(v, 100) == 100
    assert percentile([], 50) is None
    t = poisson_arrivals(20.0, 4000, 7)
    assert all(b > a for a, b in zip(t, t[1:]))
    gaps = np.diff([0.0] + t)
    assert abs(gaps.mean() - 1 / 20.0) < 0.1 / 20.0
    assert abs(gaps.std() - 1 / 20.0) < 0.15 / 20.0  # exponential gaps: std = mean


def test_multi_step_calls_count_each_env_step_once():
    """With several time steps per call an env that finishes inside the call is read back at the
    call's end; env-steps count each env's own steps (not the call length)."""
    reqs = [Request(0, env("a", 10), 0.0), Request(1, env("b", 3), 0.0)]
    srv, sc, rep = serve(reqs, admit_period=4, steps_per_call=4)
    assert rep["completed"] == 2
    assert srv.env_steps == 13
    assert rep["batch_steps"] == 12  # three calls of four steps
    assert reqs[1].finished == 0.4 and reqs[0].finished == 1.2


def test_slots_bound_the_batch_and_latency_includes_the_wait():
    """At most max_envs requests are on the GPU at once; the next one is admitted when a slot
    frees up, and its latency runs from its arrival (queue wait included), not its admission."""
    reqs = [Request(i, env(f"r{i}", 5 + i), 0.0) for i in range(5)]
    srv, sc, rep = serve(reqs, max_envs=2)
    assert rep["completed"] == 5 and rep["max_active"] == 2
    third = reqs[2]
    assert third.admitted >= reqs[0].finished > 0.0
    assert third.latency == third.finished - third.arrival
    assert third.latency > third.finished - third.admitted


def test_admission_rounds_fall_exactly_every_admission_period():
    """Requests arriving every 0.1 s (one batch step) with an admission period of 8 steps are
    admitted in rounds at t = 0, 0.8 and 1.6 s: a round as soon as the period has passed."""
    reqs = [Request(i, env(f"r{i}", 20), 0.1 * i) for i in range(10)]
    srv, sc, rep = serve(reqs, admit_period=8)
    rounds = sorted(set(round(t, 6) for kind, _, t in sc.log if kind == "add"))
    assert rounds == [0.0, 0.8, 1.6]


def test_grasp_outcome_of_the_object_rows():
    """The grasped object's rows in the point list come after every soft vertex and every
    earlier affine body's vertices; its outcome is their mean displacement, and it counts as
    held when it rose by more than half the scheduled lift."""
    from paper_2503_05020_b300.serve import initial_points, object_points, object_result

    soft = [dict(verts=np.zeros((4, 3))), dict(verts=np.ones((3, 3)))]
    q = np.array([0.5, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0, 1], dtype=np.float64)
    aff = [dict(verts=np.zeros((6, 3)), q0=q), dict(verts=np.eye(3), q0=q), dict(verts=np.zeros((2, 3)), q0=q)]
    e = {"soft": soft, "affine": aff, "object": ("affine", 1), "lift": 0.1}
    assert object_points(e) == slice(13, 16)
    p0 = initial_points(e)
    assert p0.shape == (18, 3) and np.allclose(p0[13:16], np.eye(3) + [0.5, 0, 0])
    for rise, held in ((0.03, False), (0.06, True)):
        p = p0.copy()
        p[13:16] += [0.01, 0.0, rise]
        r = object_result(e, p, p0)
        assert np.allclose(r["object_disp"], [0.01, 0.0, rise]) and r["held"] is held
    assert object_points(dict(e, object=("soft", 1))) == slice(4, 7)


def test_stability_label_of_a_finished_request():
    """Sec. III-D's label at the last step: stable when the object touches another body and its
    centre of mass (the mean of its points) moved less than eps_v dt in that step, the motion being
    dt times the mean of the object's point velocities."""
    from paper_2503_05020_b300 import scenes as S
    from paper_2503_05020_b300.serve import object_result, initial_points

    env = S.serving_request_env(4)  # plates squeezing a soft object (handle 0, plates 1 and 2)
    assert env["object"] == ("soft", 0) and len(env["affine"]) == 2
    pts = initial_points(env)
    n = len(env["soft"][0]["verts"])
    eps_v, dt = 1e-3, 0.005
    v = np.zeros(3 * n + 24)
    slow = v.copy()
    slow[2:3 * n:3] = 0.5 * eps_v  # every object vertex at half the threshold speed
    fast = v.copy()
    fast[0:3 * n:3] = 2.0 * eps_v
    touching = np.array([[0, 1], [2, 0]])
    apart = np.array([[1, 2]])  # the plates touch each other, not the object
    r = object_result(env, pts, pts, slow, touching, eps_v, dt)
    assert r["stable"] and r["in_contact"] and abs(r["com_step"] - 0.5 * eps_v * dt) < 1e-18
    assert not object_result(env, pts, pts, fast, touching, eps_v, dt)["stable"]
    r = object_result(env, pts, pts, slow, apart, eps_v, dt)
    assert not r["in_contact"] and not r["stable"]


def test_binding_names_the_grasped_object_by_its_handle():
    """The env descriptor's grasped_object is 1 + the object's handle (soft bodies first, then
    affine bodies), 0 when the env names none."""
    from paper_2503_05020_b300 import scenes as S

    assert ipc._EnvMarshal(S.serving_request_env(4)).desc.grasped_object == 1  # soft body 0
    assert ipc._EnvMarshal(S.pad_grasp_env(0)).desc.grasped_object == 3  # after two soft pads: affine 0
    assert ipc._EnvMarshal(S.single_tet_env()).desc.grasped_object == 0
