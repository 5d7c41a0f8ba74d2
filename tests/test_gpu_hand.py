"""Rigid-hand grasp scenes: 20 PD-driven affine links (about 500 triangles each) around a seeded
star-shaped soft object of about 22k tets, dhat = 5e-4 m (needs a B300).

Against the oracle (one environment; the oracle needs ~30 s per time step here, so outputs are
sampled): candidate lists bit-exact, energy and gradient within 1e-10 at two perturbed states,
and the first projected-Newton direction in parity settings. On the GPU alone: a batch of hands
closing on their objects keeps every environment alive, intersection-free and without inverted
tets.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_05020_b300 import ipc
from paper_2503_05020_b300 import scenes as S

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def params():
    p = S.scene_params(0.005)
    p["dhat"] = 5e-4
    return p


def test_hand_candidates_energy_and_newton_direction_match_the_oracle():
    p = params()
    env = S.hand_grasp_env(0)
    o = O.OracleEnv(p, env)
    x, v = o.state()
    sc = ipc.Scene(p)
    eid = sc.add_env(env)
    assert np.array_equal(sc.candidates(eid), o.candidates(x))
    rng = np.random.default_rng(11)
    # perturbed states: at the start itself the potential is ~1e-11 J (the links sit almost on
    # their first targets), too close to zero for a relative comparison of totals
    for q in (x + rng.normal(size=x.size) * 1e-5, x + rng.normal(size=x.size) * 1e-4):
        Eo, go = o.eval(q)
        Eg, gg = sc.eval(eid, q)
        assert abs(Eg - Eo) <= 1e-10 * abs(Eo), (Eg, Eo)
        assert np.abs(gg - go).max() <= 1e-10 * np.abs(go).max()
    pp = S.parity_params(p)
    o = O.OracleEnv(pp, env)
    sc = ipc.Scene(pp)
    eid = sc.add_env(env)
    po = o.newton_direction()
    pg = sc.newton_direction(eid)
    assert np.abs(pg - po).max() <= 1e-8 * np.abs(po).max()


def test_hand_batch_closes_on_the_object_without_failure():
    """Eight hands curl onto their objects (gravity off): every environment finishes the closing
    schedule intersection-free and without inverted tets, with the fingers in contact."""
    p = params()
    n_close = 120
    envs = [S.hand_grasp_env(i, n_steps=n_close, close_steps=n_close) for i in range(8)]
    sc = ipc.Scene(p)
    ids = [sc.add_env(e) for e in envs]
    sc.step(n_close)
    for e, eid in zip(envs, ids):
        st = sc.status(eid)
        assert st["status"] == "DONE", st
        inv = sc.invariants(eid)
        assert inv["intersections"] == 0 and inv["inverted"] == 0
        assert len(sc.contacts(eid)) > 0  # the fingers are on the object


def test_hinged_hands_hold_and_lift_their_objects():
    """The third configuration's grasp with the hinged hand: close 200 steps (gravity off), then
    lift the palm and the finger targets 5 cm over 100 steps with gravity on. Every object rises
    with its hand (its mean height within 1 cm of the 5 cm lift), no environment fails, crosses or
    inverts."""
    p = params()
    envs = [S.hand_grasp_env(i, n_steps=300, close_steps=200) for i in range(4)]
    sc = ipc.Scene(p)
    ids = [sc.add_env(e) for e in envs]
    sc.step(300)
    for e, eid in zip(envs, ids):
        assert sc.status(eid)["status"] == "DONE", sc.status(eid)
        assert sc.invariants(eid) == {"intersections": 0, "inverted": 0}
        n = len(e["soft"][0]["verts"])
        dz = sc.points(eid)[:n, 2].mean() - np.asarray(e["soft"][0]["verts"])[:, 2].mean()
        assert abs(dz - e["lift"]) < 0.01, dz
