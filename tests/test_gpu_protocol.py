"""The grasp evaluation protocol on the GPU (needs a B300): a pad grasp closes with the
contact-force finger halt, settles, and goes through the six axis-aligned gravity phases; the
grasp that keeps its pads closed ends with the object between them, the one whose pads reopen
drops it and is labelled unstable."""
import numpy as np
import pytest

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
