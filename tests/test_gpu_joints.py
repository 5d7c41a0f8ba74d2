"""Articulated affine bodies: point joints 1/2 h^2 k |x_a - x_b|^2 between affine bodies, as the
GPU path applies them (a joint is a two-anchor stencil in the contact and friction stencil
machinery), against the oracle (needs a B300).

* a cube hanging by a joint settles at the closed-form sag m g / k plus the affine body's own
  stretch (the oracle pins the same closed form);
* a jointed cube swinging into a fixed wall (joint, barrier and friction together): energy and
  gradient within 1e-10 and the trajectory within 1e-6 m of the oracle over 120 steps;
* the hinged hand (20 hinges, 40 point joints, a kinematic palm): its closing batch keeps every
  joint closed while the fingers press on the object (its oracle parity is in the hand tests).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_05020_b300 import ipc
from paper_2503_05020_b300 import scenes as S

pytestmark = pytest.mark.gpu

G = 9.8
TRAJ_TOL = 1e-6


def test_hanging_cube_settles_at_the_closed_form_sag():
    k, a, l = 1e3, 0.02, 0.1
    p = S.scene_params(0.01, newton_tol=1e-6)
    p["pcg_rel_tol"] = 1e-12
    env = S.pendulum_env(k_joint=k, n_steps=200, arm=l, half=a / 2)
    sc = ipc.Scene(p)
    eid = sc.add_env(env)
    sc.step(200)
    assert sc.status(eid)["status"] == "DONE"
    x = sc.dofs(eid)
    m, V = 1000.0 * a ** 3, a ** 3
    sag = m * G / k
    eps = l * m * G / (8.0 * p["kappa_affine"] * V)
    assert abs(x[14] - (-l - sag - l * eps)) <= 3e-4 * sag
    assert np.abs(x[12:14]).max() < 1e-12


def test_jointed_cube_swinging_into_a_wall_matches_the_oracle():
    p = S.parity_params(S.scene_params(0.005))
    env = S.pendulum_env(k_joint=1e4, n_steps=120, theta0=0.3, wall_y=-0.021, mu=0.4)
    o = O.OracleEnv(p, env)
    sc = ipc.Scene(p)
    eid = sc.add_env(env)
    rng = np.random.default_rng(5)
    x0, _ = o.state()
    for q in (x0 + rng.normal(size=x0.size) * 1e-4, x0 + rng.normal(size=x0.size) * 1e-3):
        Eo, go = o.eval(q)
        Eg, gg = sc.eval(eid, q)
        assert abs(Eg - Eo) <= 1e-10 * abs(Eo), (Eg, Eo)
        assert np.abs(gg - go).max() <= 1e-10 * np.abs(go).max()
    touched = 0
    for k in range(120):
        o.step(1)
        sc.step(1)
        xo, _ = o.state()
        touched += len(sc.contacts(eid)) > 0
        if k % 20 == 19:
            assert np.abs(sc.dofs(eid) - xo).max() <= TRAJ_TOL, k
    assert touched > 0  # the swing reached the wall
    assert sc.status(eid)["status"] == "DONE" and o.status()["status"] == "DONE"
    assert sc.invariants(eid) == {"intersections": 0, "inverted": 0}


def _anchor(x, n_soft_dofs, b, xb):
    q = x[n_soft_dofs + 12 * b: n_soft_dofs + 12 * b + 12]
    return q[:3] + xb[0] * q[3:6] + xb[1] * q[6:9] + xb[2] * q[9:12]


def test_hinged_hands_close_with_their_joints_held():
    p = S.scene_params(0.005)
    p["dhat"] = 5e-4
    n_close = 60
    envs = [S.hand_grasp_env(i, n_steps=n_close, close_steps=n_close) for i in range(4)]
    sc = ipc.Scene(p)
    ids = [sc.add_env(e) for e in envs]
    sc.step(n_close)
    for env, eid in zip(envs, ids):
        assert sc.status(eid)["status"] == "DONE"
        x = sc.dofs(eid)
        nsd = 3 * len(env["soft"][0]["verts"])
        gap = max(np.linalg.norm(_anchor(x, nsd, j["a"], j["anchor_a"]) - _anchor(x, nsd, j["b"], j["anchor_b"]))
                  for j in env["joints"])
        # a joint of 1e5 N/m opens by force / k: a few newtons of grip open it by tens of microns,
        # far below the links' 5.5 mm radius
        assert gap < 1e-4, gap
        assert sc.invariants(eid) == {"intersections": 0, "inverted": 0}
