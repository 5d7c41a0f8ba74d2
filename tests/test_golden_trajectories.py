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
    # the env is still stepping at the end of the window (not failed, schedule not finished)
    assert gold["final_status"]["status"] == "ACTIVE"
    assert gold["final_status"]["step"] == c["start"] + c["steps"]
