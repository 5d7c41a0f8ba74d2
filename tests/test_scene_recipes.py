"""The synthetic inputs that stand in for the paper's assets have the shapes and distributions
of the workloads they represent (no GPU): the single-env soft cube squeeze and the 64-env pad
grasp (two soft wedge pads of about 5k tets with three cutouts each, a rigid convex hull object
of 1584 triangles, seeded material and friction ranges), generated deterministically per seed."""
import numpy as np

from paper_2503_05020_b300 import scenes as S


def test_cube_squeeze_recipe():
    env = S.cube_squeeze_env(0, n_steps=100)
    soft = env["soft"][0]
    v, t = np.asarray(soft["verts"]), np.asarray(soft["tets"])
    assert len(v) == 125 and len(t) == 384
    grid = np.round((v + 0.025) / 0.0125) * 0.0125 - 0.025  # the 5x5x5 lattice of a 0.05 m cube
    assert 0 < np.abs(v - grid).max() <= 1e-5  # seeded jitter U(-1e-5, 1e-5)
    assert (soft["E"], soft["nu"], soft["rho"]) == (1e5, 0.4, 1000.0)
    assert env["mu"] == 0.5
    T, g, h = env["targets"], env["gravity"], 0.01
    assert len(T) == len(g) == 100 and np.all(g[:50] == 0) and np.all(g[50:] == 1)
    right0 = env["affine"][0]["q0"][0] - 0.005  # plate face = centre - half thickness
    assert abs(right0 - v[:, 0].max() - 1.5e-3) < 1e-12  # plates start 1.5 dhat from the faces
    assert np.allclose(np.diff(T[:50, 1, 0]), -0.01 * h) and np.allclose(np.diff(T[:50, 2, 0]), 0.01 * h)
    assert np.allclose(np.diff(T[50:, 1, 2]), 0.02 * h)  # lift at 0.02 m/s
    assert all(a["kinematic"] for a in env["affine"])


def test_pad_grasp_recipe_and_seed_ranges():
    mus, rhos = [], []
    for k in range(6):
        env = S.pad_grasp_env(k)
        pads, obj = env["soft"], env["affine"][0]
        assert len(pads) == 2 and len(env["affine"]) == 1 and not obj["kinematic"]
        for pad in pads:
            n = len(pad["tets"])
            assert 4000 <= n < 6 * 6 * 8 * 18  # ~5k: the full 6x8x18 Kuhn grid less three cutouts
            assert (pad["E"], pad["nu"]) == (2e5, 0.45)
            assert 0 < pad["kin"].sum() < len(pad["kin"])  # the gripper drives the outer layer
        assert len(obj["tris"]) == 1584
        ext = np.ptp(np.asarray(obj["verts"]), axis=0)
        assert np.all(ext >= 0.03 * 0.7) and np.all(ext <= 0.08)  # an ellipsoid of 0.03-0.08 m diameters
        mus.append(env["mu"])
        rhos.append(obj["rho"])
        assert len(env["targets"]) == 300 and np.all(env["gravity"][:100] == 0) and np.all(env["gravity"][100:] == 1)
        assert abs(env["targets"][-1, 0, 2] - 0.1) < 1e-12  # lifted 0.1 m
    assert all(0.3 <= m <= 0.8 for m in mus) and len(set(mus)) == 6
    assert all(500.0 <= r <= 1500.0 for r in rhos)
    a, b = S.pad_grasp_env(3), S.pad_grasp_env(3)
    assert np.array_equal(a["soft"][0]["verts"], b["soft"][0]["verts"]) and a["mu"] == b["mu"]
    assert not np.array_equal(S.pad_grasp_env(4)["affine"][0]["verts"], a["affine"][0]["verts"])


def test_hand_grasp_recipe():
    """Rigid hand of 20 PD-driven affine links of about 500 triangles each, grasping a star-shaped
    soft object of about 20k tets with E log-uniform over [1e4, 1e6] Pa and nu U(0.3, 0.48). The
    links hang from a kinematic palm in five chains of four, one hinge (two point joints on the
    finger's bending axis) between neighbours; every joint's anchors coincide at the start."""
    for k in range(2):
        env = S.hand_grasp_env(k)
        obj, links, palm = env["soft"][0], env["affine"][:20], env["affine"][20]
        assert 18_000 <= len(obj["tets"]) <= 24_000
        assert 1e4 <= obj["E"] <= 1e6 and 0.3 <= obj["nu"] <= 0.48
        assert len(env["affine"]) == 21 and all(450 <= len(a["tris"]) <= 550 for a in links)
        assert all(a["pd"] > 0 and not a["kinematic"] for a in links) and palm["kinematic"]
        assert len(env["targets"]) == 400 and np.all(env["gravity"][:200] == 0) and np.all(env["gravity"][200:] == 1)
        J = env["joints"]
        assert len(J) == 40 and sorted((j["a"], j["b"]) for j in J) == sorted(
            [(20, 4 * f) for f in range(5)] * 2 + [(4 * f + i, 4 * f + i + 1) for f in range(5) for i in range(3)] * 2)

        def world(b, xb):
            q = env["affine"][b]["q0"]
            return q[:3] + xb[0] * q[3:6] + xb[1] * q[6:9] + xb[2] * q[9:12]

        assert max(np.linalg.norm(world(j["a"], j["anchor_a"]) - world(j["b"], j["anchor_b"])) for j in J) < 1e-12


def test_request_schedule_closes_lifts_and_shakes_15_degrees_at_2_hz():
    """A serving request: 80 closing steps with gravity off, 60 lifting 0.1 m, then 60 steps of a
    +-15 deg shake about the grasp axis at 2 Hz (dt = 5 ms: the peak falls on the 25th step)."""
    env = S.grasp_request_env(0)
    T, g = env["targets"], env["gravity"]
    assert len(T) == 200 and np.all(g[:80] == 0) and np.all(g[80:] == 1)
    assert abs(T[139, 0, 2] - 0.1) < 1e-12
    ang = []
    for s in range(140, 200):
        A = np.stack([T[s, 0, 3:6], T[s, 0, 6:9], T[s, 0, 9:12]], axis=1)
        ang.append(np.degrees(np.arccos(np.clip((np.trace(A) - 1.0) / 2.0, -1.0, 1.0))))
    assert abs(max(ang) - 15.0) < 1e-9 and int(np.argmax(ang)) == 24
