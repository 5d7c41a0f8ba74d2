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
