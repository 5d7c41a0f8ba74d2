"""Uneven batch (needs a B300): one scene mixing soft-cube squeezes, pad grasps of rigid hulls and
star-shaped soft objects of log-uniform 2k-60k tets held by one or two pairs of plates, stepped
together. Properties that hold at any size: every environment's bits equal its run alone
(sampled), no environment fails, none has an intersection or an inverted tet.
"""
import numpy as np
import pytest

from paper_2503_05020_b300 import ipc
from paper_2503_05020_b300 import scenes as S

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

STEPS = 8


def uneven_envs():
    envs = []
    for i in range(24):
        envs.append(S.cube_squeeze_env(i, n_steps=60, close_steps=30, dt=0.005))
        envs.append(S.soft_object_grasp_env(i, n_steps=60, close_steps=30))
    for i in range(12):
        envs.append(S.pad_grasp_env(i, n_steps=60, close_steps=30))
    return envs


@pytest.mark.parametrize("precision", [ipc.FP64, ipc.MIXED], ids=["fp64", "mixed"])
def test_uneven_batch_envs_are_independent_and_valid(precision):
    p = S.scene_params(0.005)
    envs = uneven_envs()
    sizes = [S.env_sizes(e)["tets"] for e in envs]
    assert max(sizes) > 20 * min(sizes)  # the batch is uneven
    assert any(len(e["affine"]) == 4 for e in envs)  # a two-handed variant is in the mix
    sc = ipc.Scene(p, precision=precision)
    ids = [sc.add_env(e) for e in envs]
    sc.step(STEPS)
    for eid in ids:
        assert sc.status(eid)["status"] == "ACTIVE", sc.status(eid)
        inv = sc.invariants(eid)
        assert inv["intersections"] == 0 and inv["inverted"] == 0
    big = int(np.argmax(sizes))
    for k in (0, 1, big, len(envs) - 1):
        alone = ipc.Scene(p, precision=precision)
        a = alone.add_env(envs[k])
        alone.step(STEPS)
        assert np.array_equal(alone.dofs(a), sc.dofs(ids[k])), k


def test_uneven_benchmark_batch_matches_the_oracle_on_its_small_envs():
    """The benchmark's uneven batch (first 32 envs: plates or soft pads around soft objects of
    2k-60k tets, some with two gripper pairs) stepped together from the benchmark's start state
    for 10 steps in parity settings: its two smallest envs (a two-pair plate squeeze of 2.3k tets
    and a one-pair squeeze of 4.4k) end within 1e-6 m of the oracle running each alone; no env of
    the batch crosses or inverts."""
    from oracle import oracle as O

    p = S.parity_params(S.scene_params(0.005))
    envs = [S.uneven_batch_env(i) for i in range(32)]
    sc = ipc.Scene(p)
    ids = [sc.add_env(e) for e in envs]
    for eid, e in zip(ids, envs):
        x, v = S.grasp_state_at(e, S.UNEVEN_START_STEP)
        sc.set_state(eid, x, v, S.UNEVEN_START_STEP)
    sc.step(10)
    for eid in ids:
        assert sc.invariants(eid) == {"intersections": 0, "inverted": 0}
    small = sorted(range(32), key=lambda i: (S.env_sizes(envs[i])["tets"], i))[:2]
    for k in small:
        assert sc.status(ids[k])["status"] == "ACTIVE", sc.status(ids[k])
    assert len(envs[small[0]]["affine"]) == 4  # a two-pair variant is among them
    for k in small:
        o = O.OracleEnv(p, envs[k])
        x, v = S.grasp_state_at(envs[k], S.UNEVEN_START_STEP)
        o.set_state(x, v, S.UNEVEN_START_STEP)
        o.step(10)
        xo, _ = o.state()
        assert np.abs(sc.dofs(ids[k]) - xo).max() <= 1e-6, k
