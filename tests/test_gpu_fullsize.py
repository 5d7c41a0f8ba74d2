"""Parity at the benchmark's full size and launch configuration (needs a B300).

The 64-environment pad-grasp batch, from the contact-phase state the benchmark starts from, with
the default (throughput) solver settings and the automatic persistent-PCG launch shape. The
oracle cannot step 64 environments in seconds, so outputs are sampled: for a few environments
of the batch, candidate lists (bit-exact), energy and gradient (1e-10 relative) and one batched
time step (1e-6 m against the oracle stepping that environment alone).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_05020_b300 import ipc
from paper_2503_05020_b300 import scenes as S

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

N_ENV = 64
START = 20
SAMPLED = (0, 29, 63)


@pytest.fixture(scope="module")
def batch():
    p = S.scene_params(0.005)
    envs = [S.pad_grasp_env(i) for i in range(N_ENV)]
    sc = ipc.Scene(p)
    ids = [sc.add_env(e) for e in envs]
    states = []
    for eid, env in zip(ids, envs):
        x, v = S.pad_grasp_state_at(env, START)
        sc.set_state(eid, x, v, START)
        states.append((x, v))
    return p, envs, sc, ids, states


def test_sampled_candidates_and_energy_in_the_full_batch(batch):
    p, envs, sc, ids, states = batch
    for k in SAMPLED:
        x, v = states[k]
        o = O.OracleEnv(p, envs[k])
        o.set_state(x, v, START)
        assert np.array_equal(sc.candidates(ids[k]), o.candidates(x)), k
        Eo, go = o.eval(x)
        Eg, gg = sc.eval(ids[k], x)
        assert abs(Eg - Eo) <= 1e-10 * abs(Eo), (k, Eg, Eo)
        assert np.abs(gg - go).max() <= 1e-10 * np.abs(go).max(), k


def test_one_batched_step_of_a_sampled_env_matches_the_oracle(batch):
    p, envs, sc, ids, states = batch
    k = SAMPLED[1]
    x, v = states[k]
    sc.step(1)
    assert all(sc.status(e)["status"] == "ACTIVE" for e in ids)
    o = O.OracleEnv(p, envs[k])
    o.set_state(x, v, START)
    o.step(1)
    xo, _ = o.state()
    assert np.abs(sc.dofs(ids[k]) - xo).max() <= 1e-6
