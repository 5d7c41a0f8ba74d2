"""The grasp evaluation protocol on the GPU (needs a B300): a pad grasp closes with the
contact-force finger halt, settles, and goes through the six axis-aligned gravity phases; the
grasp that keeps its pads closed ends with the object between them, the one whose pads reopen
drops it and is labelled unstable. And the same protocol loop run on the oracle (through a
twin of the scene interface it uses) gives the same halt steps, the same label and the same
trajectory within 1e-6 m."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_05020_b300 import ipc
from paper_2503_05020_b300 import protocol as P
from paper_2503_05020_b300 import scenes as S
from paper_2503_05020_b300.serve import object_points

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

DT, CLOSE = 0.005, 60


def _run(env, p):
    sc = ipc.Scene(p)
    eid = sc.add_env(env)
    out = P.evaluate_grasp(sc, eid, env, fingers=[0, 1], obj=2, obj_points=object_points(env), close_steps=CLOSE,
                           eps_v=p["eps_v"], dt=DT)
    return out, sc.status(eid), sc.invariants(eid)


def test_pad_grasp_through_the_evaluation_protocol():
    p = S.scene_params(DT)
    held = P.evaluation_env(S.pad_grasp_env(0), close_steps=CLOSE, settle_steps=20, dt=DT)
    out, st, inv = _run(held, p)
    assert st["status"] == "DONE", st
    assert inv == {"intersections": 0, "inverted": 0}
    assert out.in_contact
    assert min(out.peak_force.values()) > 0.0  # both pads pressed the object
    for k, s in out.halted.items():  # a halted pad had passed the 50 N threshold
        assert out.peak_force[k] > P.HALT_FORCE_N and 0 <= s < CLOSE
    released = dict(held)
    T = np.array(held["targets"])
    T[CLOSE:] = T[0]  # the pads reopen after closing
    released["targets"] = T
    out_r, st_r, _ = _run(released, p)
    assert st_r["status"] == "DONE", st_r
    assert not out_r.stable and not out_r.in_contact


class OracleTwin:
    """The scene interface evaluate_grasp uses (step, contact forces and handles, schedule
    rewrite, points), over one oracle env: the protocol's host loop runs unchanged on it."""

    def __init__(self, params, env):
        self.o = O.OracleEnv(params, env)

    def _x(self):
        return self.o.state()[0]

    def step(self, n=1):
        self.o.step(n)

    def contact_forces(self, eid):
        return self.o.contact_forces(self._x())

    def contact_handles(self, eid):
        return self.o.contact_bodies(self._x())

    def set_env_targets(self, eid, first_step, targets):
        self.o.set_targets(first_step, targets)

    def points(self, eid):
        return self.o.points(self._x())


def test_protocol_on_the_gpu_matches_its_oracle_twin():
    """The single-env configuration's cube squeeze (plates as the fingers, handles 1 and 2; the
    cube is handle 0) through the whole protocol: 50 closing steps with the 50 N halt, 10
    settling steps, six 0.1 s gravity phases. Parity settings."""
    dt = 0.01
    p = S.parity_params(S.scene_params(dt))
    env = P.evaluation_env(S.cube_squeeze_env(0), close_steps=50, settle_steps=10, dt=dt)
    args = dict(fingers=[1, 2], obj=0, obj_points=slice(0, 125), close_steps=50, eps_v=p["eps_v"], dt=dt)
    sc = ipc.Scene(p)
    eid = sc.add_env(env)
    out_g = P.evaluate_grasp(sc, eid, env, **args)
    tw = OracleTwin(p, env)
    out_o = P.evaluate_grasp(tw, 0, env, **args)
    assert out_g.halted == out_o.halted and len(out_o.halted) == 2  # both plates halted, same step
    assert all(0 < s < 50 for s in out_o.halted.values())
    assert (out_g.stable, out_g.in_contact) == (out_o.stable, out_o.in_contact)
    assert out_o.in_contact
    for k in (1, 2):
        assert abs(out_g.peak_force[k] - out_o.peak_force[k]) <= 1e-6 * out_o.peak_force[k]
    assert abs(out_g.com_step - out_o.com_step) <= 1e-6
    assert np.abs(sc.dofs(eid) - tw.o.state()[0]).max() <= 1e-6
    assert sc.status(eid)["status"] == "DONE" and tw.o.status()["status"] == "DONE"
