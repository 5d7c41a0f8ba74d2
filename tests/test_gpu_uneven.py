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
