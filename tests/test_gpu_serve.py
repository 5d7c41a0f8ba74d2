"""Serving loop on the GPU: continuous batching keeps every result identical to the same
request run alone, and admission by HBM budget bounds the resident batch (needs a B300)."""
import numpy as np
import pytest

from paper_2503_05020_b300 import ipc
from paper_2503_05020_b300 import scenes as S
from paper_2503_05020_b300.serve import GraspServer, Request

pytestmark = pytest.mark.gpu


def short_request(i):
    return S.grasp_request_env(100 + i, close_steps=20, lift_steps=12, shake_steps=12)


def alone(params, env, precision):
    sc = ipc.Scene(params, precision=precision)
    eid = sc.add_env(env)
    sc.step(len(env["targets"]))
    assert sc.status(eid)["status"] == "DONE"
    return sc.dofs(eid)


@pytest.mark.parametrize("precision", [ipc.FP64, ipc.MIXED], ids=["fp64", "mixed"])
def test_served_results_are_identical_to_results_alone(precision):
    p = S.scene_params(0.005)
    envs = [short_request(i) for i in range(4)]
    arrivals = [0.0, 0.01, 0.25, 0.6]
    reqs = [Request(i, e, t) for i, (e, t) in enumerate(zip(envs, arrivals))]
    srv = GraspServer(p, precision=precision, max_envs=8, admit_period=2, steps_per_call=2)
    rep = srv.run(reqs)
    assert rep["completed"] == 4, rep
    assert any(r.admitted < q.finished and r.admitted > q.admitted for r in reqs for q in reqs), \
        "no request joined a running batch"
    for r in reqs:
        assert r.status == "DONE"
        assert np.array_equal(r.result["dofs"], alone(p, r.env, precision)), r.rid
    assert rep["p99_latency_s"] >= rep["p50_latency_s"] > 0


def test_hbm_budget_bounds_the_resident_batch():
    p = S.scene_params(0.005)
    envs = [short_request(i) for i in range(4)]
    per_env = max(ipc.estimate_bytes(e) for e in envs)
    reqs = [Request(i, e, 0.0) for i, e in enumerate(envs)]
    srv = GraspServer(p, hbm_budget_bytes=int(2.5 * per_env), max_envs=8, admit_period=1)
    rep = srv.run(reqs)
    assert rep["completed"] == 4 and rep["rejected"] == 0
    assert rep["max_active"] == 2


@pytest.mark.slow
def test_served_labels_and_held_object_match_the_oracle():
    """Two requests of the serving configuration (plates squeezing soft objects of 1.7k and 2.3k
    tets: close, lift 5 cm, shake +/-15 deg at 2 Hz, hold), served together in FP64 and in mixed
    precision at the default tolerances, against the FP64 oracle running each request alone:
    the same Sec. III-D label (the smaller object is dropped, the larger held), and the held
    object's points end within 1e-4 of its displacement of the oracle's."""
    from oracle import oracle as O
    from paper_2503_05020_b300.serve import initial_points, object_points, object_result

    p = S.scene_params(0.005)
    ids = (4, 5)
    envs = [S.serving_request_env(i) for i in ids]
    ref = []
    for env in envs:
        o = O.OracleEnv(p, env)
        assert o.step(len(env["targets"])) == "DONE"
        x, v = o.state()
        pts = o.points(x)
        ref.append((pts, object_result(env, pts, initial_points(env), v, o.contact_bodies(x), p["eps_v"], p["dt"])))
    assert [r[1]["stable"] for r in ref] == [False, True]
    for prec in (ipc.FP64, ipc.MIXED):
        reqs = [Request(k, e, 0.0) for k, e in enumerate(envs)]
        GraspServer(p, precision=prec, max_envs=8, admit_period=8, steps_per_call=8).run(reqs)
        for r, (pts_o, res_o), env in zip(reqs, ref, envs):
            assert r.status == "DONE"
            assert r.result["stable"] == res_o["stable"] and r.result["in_contact"] == res_o["in_contact"]
            if res_o["stable"]:
                sl = object_points(env)
                disp = float(np.abs(pts_o[sl] - initial_points(env)[sl]).max())
                err = float(np.abs(r.result["points"][sl] - pts_o[sl]).max())
                assert err <= 1e-4 * disp, (prec, err, disp)


def test_grasp_result_query_matches_its_definition():
    """IPC_Q_GRASP_RESULT of a finished serving request (the held 2.3k-tet object) against the
    Sec. III-D outcome computed from the env's own point, velocity and contact queries: same
    contact flag and label, the same centre-of-mass motion over the last step and rise."""
    from paper_2503_05020_b300.serve import initial_points, object_result

    p = S.scene_params(0.005)
    env = S.serving_request_env(5)
    sc = ipc.Scene(p)
    eid = sc.add_env(env)
    sc.step(len(env["targets"]))
    assert sc.status(eid)["status"] == "DONE"
    g = sc.grasp_result(eid)
    ref = object_result(env, sc.points(eid), initial_points(env), sc.velocities(eid), sc.contact_handles(eid),
                        p["eps_v"], p["dt"])
    assert (g["in_contact"], g["stable"]) == (ref["in_contact"], ref["stable"]) == (True, True)
    assert abs(g["com_step"] - ref["com_step"]) <= 1e-12 + 1e-9 * ref["com_step"]
    assert abs(g["com_rise"] - ref["object_disp"][2]) <= 1e-12
    assert abs(g["com_rise"] - env["lift"]) < 0.01  # held through the shake: it rose with the grippers
