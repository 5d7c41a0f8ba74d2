"""The stored oracle trajectories (tests/golden/traj100_*.json) still describe the scenes the
generators build today, and hold what their GPU test expects (no GPU needed)."""
import importlib.util
import json
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
spec = importlib.util.spec_from_file_location("make_trajectory_goldens",
                                              os.path.join(HERE, "golden", "make_trajectory_goldens.py"))
G = importlib.util.module_from_spec(spec)
spec.loader.exec_module(G)


@pytest.mark.parametrize("case", sorted(G.CASES))
def test_golden_matches_its_generators(case):
    with open(G.golden_path(case)) as f:
        gold = json.load(f)
    c = G.CASES[case]
    env, params = c["build"](), c["params"]()
    x0, v0 = G.S.grasp_state_at(env, c["start"])
    assert gold["env_fingerprint"] == G.fingerprint(env)
    assert gold["params_fingerprint"] == G.fingerprint(params)
    assert gold["start_fingerprint"] == G.fingerprint([x0, v0])
    assert gold["start_step"] == c["start"] and gold["n_steps"] == c["steps"]
    idx = np.asarray(gold["dof_indices"])
    assert np.array_equal(idx, G.sampled_dof_indices(env))
    assert idx.max() < x0.size and len(np.unique(idx)) == len(idx)
    steps = [chk["steps"] for chk in gold["checkpoints"]]
    assert steps == list(range(G.EVERY, c["steps"] + 1, G.EVERY))
    for chk in gold["checkpoints"]:
        assert len(chk["dofs"]) == len(idx) and np.all(np.isfinite(chk["dofs"]))
    # the env is still stepping at the end of the window (not failed; a window that ends with its
    # schedule finishes it)
    assert gold["final_status"]["status"] == c.get("final", "ACTIVE")
    assert gold["final_status"]["step"] == c["start"] + c["steps"]


def _checkpoints(case):
    """(env, start DOFs, sampled indices, [(steps, DOFs with the sampled entries of that
    checkpoint)]) of a stored trajectory."""
    with open(G.golden_path(case)) as f:
        gold = json.load(f)
    c = G.CASES[case]
    env = c["build"]()
    x0, _ = G.S.grasp_state_at(env, c["start"])
    idx = np.asarray(gold["dof_indices"])
    out = []
    for chk in gold["checkpoints"]:
        x = x0.copy()
        x[idx] = chk["dofs"]
        out.append((chk["steps"], x))
    return env, x0, idx, out


def _soft0_mean_shift(env, x0, idx, x):
    n0 = len(env["soft"][0]["verts"])
    sel = idx[idx < 3 * n0]
    return (x[sel] - x0[sel]).reshape(-1, 3).mean(axis=0)


def test_stored_uneven_envs_hold_or_drop_their_objects():
    """The oracle's plate squeezes end the way their scenes make them: env 8's object rises with
    its two plate pairs (3 cm by step 120) within 1%; env 22's object, between one pair, slips out
    once gravity is on and has fallen more than 10 cm while the plates rose 3 cm."""
    for case, held in (("uneven_8", True), ("uneven_22", False)):
        env, x0, idx, chks = _checkpoints(case)
        steps, x = chks[-1]
        base = 3 * sum(len(s["verts"]) for s in env["soft"])
        plate_rise = x[base + 2] - x0[base + 2]  # first plate's translation z
        assert abs(plate_rise - 0.03) < 1e-9, plate_rise
        dz = _soft0_mean_shift(env, x0, idx, x)[2]
        if held:
            assert abs(dz - plate_rise) < 0.01 * plate_rise, dz
        else:
            assert dz < -0.1, dz


def test_stored_pad_closing_squeezes_the_hull_in_place():
    """With gravity off the two pads close 3.5 mm each from opposite sides: the rigid hull
    between them moves less than 0.5 mm and its A stays within 1e-2 of a rotation's."""
    env, x0, idx, chks = _checkpoints("pad_grasp_0")
    base = 3 * sum(len(s["verts"]) for s in env["soft"])
    for steps, x in chks:
        assert np.abs(x[base:base + 3] - x0[base:base + 3]).max() < 5e-4, steps
        A = x[base + 3:base + 12].reshape(3, 3).T
        assert np.abs(A @ A.T - np.eye(3)).max() < 1e-2, steps
    shift = _soft0_mean_shift(env, x0, idx, chks[-1][1])
    assert abs(shift[0] + 3.5e-3) < 5e-4, shift  # the first pad's mean moves with its base layer


def test_stored_hand_leaves_the_object_at_rest_until_the_fingers_arrive():
    """Gravity is off while the hand closes: no force acts on the free soft object until a finger
    reaches it, so its sampled vertices stay where they started (to rounding) through step 180,
    and the fingers have moved it by step 200."""
    env, x0, idx, chks = _checkpoints("hand_0")
    n0 = len(env["soft"][0]["verts"])
    sel = idx[idx < 3 * n0]
    for steps, x in chks:
        moved = np.abs(x[sel] - x0[sel]).max()
        if steps <= 180:
            assert moved < 1e-12, (steps, moved)
        else:
            assert moved > 1e-3, (steps, moved)


def test_stored_hand_grasp_holds_and_lifts_the_object():
    """The oracle's whole hand grasp in the configuration's settings: the fingers close on the
    object with gravity off (steps 0-200), then palm and finger targets rise 5 cm in 100 steps
    with gravity on. The object rises with the hand: its sampled vertices' mean height follows
    the palm's (the last affine body's) rise within 1 mm at every checkpoint of the lift (the
    closing fingers have pushed it up 2.2 mm by step 200; under its weight it then trails the palm
    by 0.5 mm) and ends within 1 mm of the full 5 cm, and the run finishes its schedule without
    failing."""
    with open(G.golden_path("hand_0_hold")) as f:
        gold = json.load(f)
    assert gold["final_status"]["status"] == "DONE" and gold["final_status"]["reason"] == 0
    env, x0, idx, chks = _checkpoints("hand_0_hold")
    palm = 3 * sum(len(s["verts"]) for s in env["soft"]) + 12 * (len(env["affine"]) - 1)
    for steps, x in chks:
        rise = x[palm + 2] - x0[palm + 2]
        dz = _soft0_mean_shift(env, x0, idx, x)[2]
        if steps > 200:
            assert rise > 0 and abs(dz - rise) < 1e-3, (steps, dz, rise)
    assert abs(rise - env["lift"]) < 1e-9 and abs(dz - env["lift"]) < 1e-3, (dz, rise)


def test_stored_pad_grasp_lifts_the_hull_with_the_pads():
    """The pad configuration's env 0 as configured: the pads close on the rigid hull with gravity
    off (100 steps), then their bases rise 0.1 m in 200 steps with gravity on. The hull is held:
    its translation follows the pads' rise within 1 mm at every checkpoint (the squeeze moves it
    0.3 mm) and ends within 1 mm of 0.1 m, its A stays within 1e-3 of a rotation's, and the run
    finishes its schedule without failing."""
    with open(G.golden_path("pad_grasp_0_lift")) as f:
        gold = json.load(f)
    assert gold["final_status"]["status"] == "DONE" and gold["final_status"]["reason"] == 0
    env, x0, idx, chks = _checkpoints("pad_grasp_0_lift")
    base = 3 * sum(len(s["verts"]) for s in env["soft"])
    for steps, x in chks:
        rise = env["lift"] * max(0, steps - 100) / 200
        dz = x[base + 2] - x0[base + 2]
        assert abs(dz - rise) < 1e-3, (steps, dz, rise)
        A = x[base + 3:base + 12].reshape(3, 3).T
        assert np.abs(A @ A.T - np.eye(3)).max() < 1e-3, steps
    assert abs(dz - env["lift"]) < 1e-3, dz


def test_stored_soft_pad_grasp_lifts_the_soft_object():
    """The uneven batch's env 4 as configured: two soft pads close on a 3.3k-tet soft object with
    gravity off (100 steps), then their bases rise 0.1 m in 200 steps with gravity on. The object
    is held: when gravity comes on it settles into the soft pads over the first 40 lifting steps
    (its sampled vertices' mean height then trails the pads' rise by about 3 mm, never by 5 mm),
    then it sticks: from one later lift checkpoint to the next its lag grows by less than
    eps_v dt per step, the friction model's static/dynamic transition speed; it ends above 95%
    of the lift, and the run finishes its schedule without failing."""
    with open(G.golden_path("uneven_4_lift")) as f:
        gold = json.load(f)
    assert gold["final_status"]["status"] == "DONE" and gold["final_status"]["reason"] == 0
    env, x0, idx, chks = _checkpoints("uneven_4_lift")
    p = G.CASES["uneven_4_lift"]["params"]()
    lo = 3 * sum(len(s["verts"]) for s in env["soft"][:-1])
    hi = lo + 3 * len(env["soft"][-1]["verts"])
    sel = idx[(idx >= lo) & (idx < hi)]
    assert len(sel) > 30
    lags = []
    for steps, x in chks:
        rise = 0.1 * max(0, steps - 100) / 200
        dz = (x[sel] - x0[sel]).reshape(-1, 3).mean(axis=0)[2]
        if steps <= 100:
            assert abs(dz) < 1e-4, (steps, dz)  # gravity off: the closing pads do not lift it
        else:
            assert 0 <= rise - dz < 5e-3, (steps, dz, rise)
            lags.append(rise - dz)
    creep = np.diff(lags[1:])  # settled from the second lift checkpoint (step 140) on
    assert np.all(creep < p["eps_v"] * p["dt"] * G.EVERY), creep
    assert dz > 0.095, dz


@pytest.mark.slow
def test_oracle_still_computes_the_first_stored_checkpoint():
    """The fingerprints tie a golden to its inputs; this ties it to the oracle's code: the first
    20 steps of the smallest case, rerun now, give the stored DOFs bit for bit."""
    from oracle import oracle as O

    case = "uneven_8"
    with open(G.golden_path(case)) as f:
        gold = json.load(f)
    c = G.CASES[case]
    env, params = c["build"](), c["params"]()
    x0, v0 = G.S.grasp_state_at(env, c["start"])
    o = O.OracleEnv(params, env)
    o.set_state(x0, v0, c["start"])
    o.step(G.EVERY)
    x, _ = o.state()
    idx = np.asarray(gold["dof_indices"])
    assert np.array_equal(x[idx], np.asarray(gold["checkpoints"][0]["dofs"]))
