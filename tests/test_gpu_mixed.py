"""Mixed precision (FP32 Hessians and PCG, FP64 energies, gradients, barrier, CCD and line
search) against the FP64 oracle and the FP64 GPU path (needs a B300).

Bars: the grasped object's displacement within 1e-4 relative of FP64 (the grasp evaluation's
output) and the same grasp outcome; every DOF within ALL_REL, the spread the FP64 stepper shows
by itself when only its PCG tolerance changes (1e-4 to 1e-5 moves pad vertices by up to 9.2e-4
of the largest displacement on this workload); no intersection and no inverted tet; an
environment's bits the same alone and in a batch. A single soft cube (no sliding pads) is held to
1e-4 on every DOF against the oracle.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_05020_b300 import ipc
from paper_2503_05020_b300 import scenes as S

pytestmark = pytest.mark.gpu

REL = 1e-4
ALL_REL = 5e-4


def trajectory(params, envs, precision, steps, points=False):
    """DOFs (or world positions of every point: soft vertices, then each affine body's
    vertices) after each step."""
    sc = ipc.Scene(params, precision=precision)
    ids = [sc.add_env(e) for e in envs]
    get = (lambda i: sc.points(i).copy()) if points else (lambda i: sc.dofs(i).copy())
    x0 = [get(i) for i in ids]
    traj = [[] for _ in ids]
    for _ in range(steps):
        sc.step(1)
        for k, i in enumerate(ids):
            traj[k].append(get(i))
    return sc, ids, x0, [np.array(t) for t in traj]


def rel_error(a, b, x0):
    """max |a - b| over the run, relative to the largest displacement of b from x0."""
    return np.abs(a - b).max() / np.abs(b - x0).max()


def test_mixed_cube_squeeze_matches_oracle_100_steps():
    p = S.scene_params(0.01)
    env = S.cube_squeeze_env(0, n_steps=100)
    sc, ids, x0, traj = trajectory(p, [env], ipc.MIXED, 100)
    o = O.OracleEnv(p, env)
    o.step(100)
    xo, _ = o.state()
    assert sc.status(ids[0])["status"] == "DONE"
    err = np.abs(traj[0][-1] - xo).max() / np.abs(xo - x0[0]).max()
    assert err <= REL, err
    inv = sc.invariants(ids[0])
    assert inv["intersections"] == 0 and inv["inverted"] == 0


def object_points(env):
    """Rows of the grasped rigid object (the first affine body) in the point list."""
    n_soft = sum(len(s["verts"]) for s in env["soft"])
    return slice(n_soft, n_soft + len(env["affine"][0]["verts"]))


@pytest.mark.slow
def test_mixed_pad_grasp_full_schedule_matches_fp64_and_lifts_the_same():
    """Four uneven pad-grasp environments, batched, over the whole close-and-lift schedule."""
    p = S.scene_params(0.005)
    envs = [S.pad_grasp_env(i) for i in range(4)]
    steps = len(envs[0]["targets"])
    sc64, ids64, x0, t64 = trajectory(p, envs, ipc.FP64, steps, points=True)
    sc32, ids32, _, t32 = trajectory(p, envs, ipc.MIXED, steps, points=True)
    for k, env in enumerate(envs):
        assert sc64.status(ids64[k])["status"] == "DONE"
        assert sc32.status(ids32[k])["status"] == "DONE"
        err = rel_error(t32[k], t64[k], x0[k])
        assert err <= ALL_REL, (k, err)
        obj = object_points(env)
        err_obj = np.abs(t32[k][:, obj] - t64[k][:, obj]).max() / np.abs(t64[k] - x0[k]).max()
        assert err_obj <= REL, (k, err_obj)
        lift64 = (t64[k][-1, obj, 2] - x0[k][obj, 2]).mean()
        lift32 = (t32[k][-1, obj, 2] - x0[k][obj, 2]).mean()
        held64, held32 = lift64 > 0.05, lift32 > 0.05
        assert held64 == held32, (k, lift64, lift32)
        inv = sc32.invariants(ids32[k])
        assert inv["intersections"] == 0 and inv["inverted"] == 0


def test_mixed_env_is_bit_identical_alone_and_in_a_batch():
    p = S.scene_params(0.01)
    cube = S.cube_squeeze_env(0, n_steps=12, close_steps=6)
    alone = ipc.Scene(p, precision=ipc.MIXED)
    a = alone.add_env(cube)
    alone.step(12)
    batch = ipc.Scene(p, precision=ipc.MIXED)
    batch.add_env(S.pad_grasp_env(0, n_steps=12, close_steps=6))
    b = batch.add_env(cube)
    batch.add_env(S.resting_env("rigid", n_steps=12))
    batch.step(12)
    assert np.array_equal(alone.dofs(a), batch.dofs(b))
    assert batch.status(b)["status"] == "DONE"
