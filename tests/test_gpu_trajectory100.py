"""Trajectories of 100 steps and more against the oracle (needs a B300).

The oracle needs seconds to tens of seconds per time step on these scenes, so its trajectories
are stored: `tests/golden/make_trajectory_goldens.py` steps each seeded environment on the CPU
oracle in the parity settings (Newton tolerance x1e-3, CG to 1e-12) and keeps a sample of its
DOFs (evenly strided soft vertices and every affine coordinate) every 20 steps. Here the CUDA
path takes the same steps from the same state and every sampled DOF must stay within 1e-6 m of
the oracle's at every checkpoint (affine coordinates: the same bound on the translation and on
the dimensionless A entries). A golden whose scene, parameters or start state no longer match
the generators is refused, not compared.

Cases: the pad configuration's env 0 (two ~5k-tet soft pads closing on a rigid hull, steps
0-100, gravity off); two small envs of the uneven batch stepped together from their contact
state at step 20 to step 120 (a 2.3k-tet object between two pairs of plates, lifted, and a
4.4k-tet object between one pair, which slips out and falls once gravity is on). The hinged
hand's case is in `tests/test_gpu_zz_hand_trajectory.py`.
"""
import importlib.util
import json
import os

import numpy as np
import pytest

from paper_2503_05020_b300 import ipc

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TRAJ_TOL = 1e-6
HERE = os.path.dirname(os.path.abspath(__file__))


def _generator():
    spec = importlib.util.spec_from_file_location("make_trajectory_goldens",
                                                  os.path.join(HERE, "golden", "make_trajectory_goldens.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


G = _generator()


def load(case):
    """The stored oracle trajectory of a case, with its scene and parameters rebuilt from the
    generators and checked against the fingerprints the golden was written with."""
    with open(G.golden_path(case)) as f:
        gold = json.load(f)
    c = G.CASES[case]
    env, params = c["build"](), c["params"]()
    x0, v0 = G.S.grasp_state_at(env, gold["start_step"])
    assert G.fingerprint(env) == gold["env_fingerprint"], f"{case}: scene changed since the golden was written"
    assert G.fingerprint(params) == gold["params_fingerprint"], f"{case}: parameters changed"
    assert G.fingerprint([x0, v0]) == gold["start_fingerprint"], f"{case}: start state changed"
    assert gold["start_step"] == c["start"] and gold["n_steps"] == c["steps"]
    return gold, env, params, x0, v0


def run_against_goldens(cases):
    """Step the cases' envs together in one scene from their stored start and compare the sampled
    DOFs with each golden at every checkpoint. The cases must share parameters and start step."""
    loaded = [load(c) for c in cases]
    params = loaded[0][2]
    start = loaded[0][0]["start_step"]
    assert all(g["start_step"] == start and p == params for g, _, p, _, _ in loaded)
    sc = ipc.Scene(params)
    ids = []
    for gold, env, _, x0, v0 in loaded:
        eid = sc.add_env(env)
        sc.set_state(eid, x0, v0, start)
        ids.append(eid)
    done = 0
    for k, chk in enumerate(loaded[0][0]["checkpoints"]):
        sc.step(chk["steps"] - done)
        done = chk["steps"]
        for case, (gold, env, _, _, _), eid in zip(cases, loaded, ids):
            assert gold["checkpoints"][k]["steps"] == done
            idx = np.asarray(gold["dof_indices"])
            xo = np.asarray(gold["checkpoints"][k]["dofs"])
            err = np.abs(sc.dofs(eid)[idx] - xo).max()
            assert err <= TRAJ_TOL, (case, start + done, err)
            assert sc.invariants(eid) == {"intersections": 0, "inverted": 0}, (case, start + done)
    for case, (gold, _, _, _, _), eid in zip(cases, loaded, ids):
        assert sc.status(eid)["status"] == gold["final_status"]["status"], (case, sc.status(eid))


def test_pad_grasp_100_steps_match_the_oracle():
    run_against_goldens(["pad_grasp_0"])


def test_uneven_batch_small_envs_100_steps_match_the_oracle():
    run_against_goldens(["uneven_8", "uneven_22"])
