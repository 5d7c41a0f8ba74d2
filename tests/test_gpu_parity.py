"""CUDA path vs the CPU oracle, through the C ABI (needs a B300).

Bars: candidate lists bit-exact; energy and gradient at the same state within 1e-10 relative
(FP64); trajectories within 1e-6 m; isolation of environments bit-exact.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_05020_b300 import ipc
from paper_2503_05020_b300 import scenes as S

pytestmark = pytest.mark.gpu

E_TOL = 1e-10
TRAJ_TOL = 1e-6


def oracle_state(params, env, steps):
    o = O.OracleEnv(params, env)
    if steps:
        o.step(steps)
    x, v = o.state()
    return o, x, v


def pads_pressed(env, shift):
    """Initial DOFs of a pad scene with both soft pads moved `shift` towards the object."""
    o = O.OracleEnv(S.scene_params(0.005), env)
    x, v = o.state()
    n0 = len(env["soft"][0]["verts"])
    n1 = len(env["soft"][1]["verts"])
    xs = x.copy()
    xs[: 3 * n0].reshape(-1, 3)[:, 0] -= shift
    xs[3 * n0: 3 * (n0 + n1)].reshape(-1, 3)[:, 0] += shift
    return xs, v


def test_candidates_and_contacts_bit_exact_cube():
    p = S.scene_params(0.01)
    env = S.cube_squeeze_env(0, n_steps=40, close_steps=20)
    o, x, v = oracle_state(p, env, 25)
    sc = ipc.Scene(p)
    eid = sc.add_env(env)
    sc.set_state(eid, x, v, 25)
    cg = sc.candidates(eid)
    co = o.candidates(x)
    assert len(co) > 100
    assert cg.shape == co.shape and np.array_equal(cg, co)
    kg = sc.contacts(eid)
    ko, d2 = o.contacts(x)
    assert len(ko) > 10
    assert np.array_equal(kg[:, :3], ko[:, :3])


def test_candidates_bit_exact_pads_and_hull():
    p = S.scene_params(0.005)
    env = S.pad_grasp_env(0)
    x, v = pads_pressed(env, 1.2e-3)
    o = O.OracleEnv(p, env)
    o.set_state(x, v, 0)
    sc = ipc.Scene(p)
    eid = sc.add_env(env)
    sc.set_state(eid, x, v, 0)
    cg = sc.candidates(eid)
    co = o.candidates(x)
    assert len(co) > 1000
    assert np.array_equal(cg, co)
    kg = sc.contacts(eid)
    ko, _ = o.contacts(x)
    assert len(ko) > 0
    assert np.array_equal(kg[:, :3], ko[:, :3])


def _energy_parity(p, env, x, v, step, q):
    o = O.OracleEnv(p, env)
    o.set_state(x, v, step)
    Eo, go = o.eval(q)
    sc = ipc.Scene(p)
    eid = sc.add_env(env)
    sc.set_state(eid, x, v, step)
    Eg, gg = sc.eval(eid, q)
    assert abs(Eg - Eo) <= E_TOL * abs(Eo), (Eg, Eo)
    assert np.abs(gg - go).max() <= E_TOL * np.abs(go).max(), np.abs(gg - go).max() / np.abs(go).max()
    return Eo, go


def test_energy_gradient_parity_cube_with_contact_and_friction():
    p = S.scene_params(0.01)
    env = S.cube_squeeze_env(0, n_steps=40, close_steps=20)
    o, x, v = oracle_state(p, env, 25)
    rng = np.random.default_rng(5)
    q = x + rng.normal(size=x.size) * 2e-6
    q[3 * 125:] = x[3 * 125:]  # plates stay where they are
    _energy_parity(p, env, x, v, 25, q)


def test_energy_gradient_parity_pads_and_rigid_hull():
    p = S.scene_params(0.005)
    env = S.pad_grasp_env(1)
    x, v = pads_pressed(env, 1.3e-3)
    rng = np.random.default_rng(6)
    q = x + rng.normal(size=x.size) * 1e-7
    _energy_parity(p, env, x, v, 120, q)  # a lifting step: gravity on


def test_energy_gradient_parity_rigid_on_incline():
    p = S.scene_params(0.01)
    env = S.resting_env("rigid", n_steps=30, mu=0.4, incline_deg=15)
    o, x, v = oracle_state(p, env, 10)
    q = x.copy()
    q[:12] += np.random.default_rng(7).normal(size=12) * 1e-6
    _energy_parity(p, env, x, v, 10, q)


@pytest.mark.parametrize("body", ["tet", "rigid", "block"])
def test_resting_trajectory_parity(body):
    p = S.parity_params(S.scene_params(0.01))
    env = S.resting_env(body, n_steps=40)
    o = O.OracleEnv(p, env)
    o.step(40)
    xo, _ = o.state()
    sc = ipc.Scene(p)
    eid = sc.add_env(env)
    sc.step(40)
    assert sc.status(eid)["status"] == "DONE"
    assert np.abs(sc.dofs(eid) - xo).max() <= TRAJ_TOL


def test_free_fall_closed_form_gpu():
    h = 0.01
    p = S.parity_params(S.scene_params(h))
    env = S.single_tet_env(n_steps=10)
    sc = ipc.Scene(p)
    eid = sc.add_env(env)
    x0 = sc.dofs(eid)
    sc.step(10)
    x = sc.dofs(eid)
    vz, z = 0.0, 0.0
    for _ in range(10):
        vz -= h * 9.8
        z += h * vz
    assert np.allclose((x - x0).reshape(-1, 3)[:, 2], z, rtol=1e-9)


@pytest.mark.slow
def test_cube_grasp_trajectory_parity_100_steps():
    """The cube-squeeze grasp, 100 steps of close (gravity off) and lift (gravity on): GPU and
    oracle trajectories agree within 1e-6 m at every 20th step, with no intersection."""
    p = S.parity_params(S.scene_params(0.01))
    env = S.cube_squeeze_env(0)
    o = O.OracleEnv(p, env)
    sc = ipc.Scene(p)
    eid = sc.add_env(env)
    for k in range(5):
        o.step(20)
        sc.step(20)
        xo, _ = o.state()
        xg = sc.dofs(eid)
        err = np.abs(xg - xo).max()
        assert err <= TRAJ_TOL, (k, err)
    assert sc.status(eid)["status"] == "DONE"
    inv = sc.invariants(eid)
    assert inv == {"intersections": 0, "inverted": 0}
    dz = xg[: 3 * 125].reshape(-1, 3)[:, 2].mean() - S.cube_squeeze_env(0)["soft"][0]["verts"][:, 2].mean()
    assert dz > 0.009  # lifted with the plates (1 cm)


def test_pad_grasp_steps_parity():
    """Soft pads squeezing the rigid hull, a few steps with gravity on."""
    p = S.parity_params(S.scene_params(0.005))
    env = S.pad_grasp_env(2, n_steps=3, close_steps=10, squeeze=2e-3)
    x, v = pads_pressed(env, 1.0e-3)
    o = O.OracleEnv(p, env)
    o.set_state(x, v, 0)
    o.step(3)
    sc = ipc.Scene(p)
    eid = sc.add_env(env)
    sc.set_state(eid, x, v, 0)
    sc.step(3)
    assert sc.status(eid)["status"] == o.status()["status"] == "DONE"
    xo, _ = o.state()
    assert np.abs(sc.dofs(eid) - xo).max() <= TRAJ_TOL


def test_batched_env_is_bit_identical_to_alone_and_isolated_from_failures():
    """Sec. III-A: envs evolve independently. An env stepped in a batch with an uneven partner
    and a failing partner gives exactly the bits it gives alone; the failure stays local."""
    p = S.scene_params(0.01)
    cube = S.cube_squeeze_env(0, n_steps=12, close_steps=6)
    alone = ipc.Scene(p)
    a = alone.add_env(cube)
    alone.step(12)
    xa = alone.dofs(a)
    batch = ipc.Scene(p)
    b0 = batch.add_env(S.resting_env("rigid", n_steps=12))
    b1 = batch.add_env(cube)
    bad_env = S.resting_env("block", n_steps=12)
    b2 = batch.add_env(bad_env)
    xb2 = batch.dofs(b2)
    vb2 = np.zeros_like(xb2)
    vb2[0] = np.nan  # a non-finite state injected from the host
    batch.set_state(b2, xb2, vb2, 0)
    batch.step(12)
    assert np.array_equal(batch.dofs(b1), xa)
    work = ("newton_iters", "pcg_iters", "ls_halvings", "steps", "accd_iters")
    assert {k: batch.status(b1)[k] for k in work} == {k: alone.status(a)[k] for k in work}
    assert batch.status(b1)["status"] == "DONE"
    assert batch.status(b0)["status"] == "DONE"
    st = batch.status(b2)
    assert st["status"] == "FAILED" and st["reason"] == "non_finite"


def test_newton_cap_fails_only_that_env():
    p = S.scene_params(0.01)
    p["max_newton"] = 1
    sc = ipc.Scene(p)
    a = sc.add_env(S.cube_squeeze_env(0, n_steps=30, close_steps=20))
    b = sc.add_env(S.spinning_body_env(n_steps=3, omega=(0, 0, 0)))
    sc.step(30)
    sa, sb = sc.status(a), sc.status(b)
    assert sa["status"] == "FAILED" and sa["reason"] == "newton_cap"
    assert sb["status"] == "DONE"


@pytest.mark.parametrize("pcg_cluster", [0, -1], ids=["persistent", "tiled"])
@pytest.mark.parametrize("case", ["tet", "rigid", "block", "cube"])
def test_newton_direction_parity(case, pcg_cluster):
    """The first projected-Newton direction (Hessian assembly + PCG) matches the oracle's CG
    solve at the same state, in parity settings (PCG to 1e-12), with the persistent
    per-environment solve and with the multi-launch tiled one."""
    p = S.parity_params(S.scene_params(0.01))
    if case == "cube":
        env = S.cube_squeeze_env(0, n_steps=40, close_steps=20)
        _, x, v = oracle_state(S.scene_params(0.01), env, 25)
        step = 25
    else:
        env = S.resting_env(case, n_steps=40)
        x = v = None
        step = 0
    o = O.OracleEnv(p, env)
    sc = ipc.Scene(p, pcg_cluster=pcg_cluster)
    eid = sc.add_env(env)
    if x is not None:
        o.set_state(x, v, step)
        sc.set_state(eid, x, v, step)
    po = o.newton_direction()
    pg = sc.newton_direction(eid)
    assert np.abs(pg - po).max() <= 1e-8 * np.abs(po).max(), np.abs(pg - po).max() / np.abs(po).max()


def pressed_cube_state():
    env = S.cube_squeeze_env(0, n_steps=40, close_steps=20)
    _, x, v = oracle_state(S.scene_params(0.01), env, 25)
    return env, x, v, 25


def test_persistent_pcg_bits_do_not_depend_on_cluster_size_or_batch():
    """The persistent solve sums every dot product per slice / per body and adds an env's slots
    in an order fixed by the env alone: cluster sizes 1, 2, 4, 8, 16 and the automatic choice, alone
    or next to a larger env, give the same bits; the tiled multi-launch solve agrees to rounding."""
    p = S.parity_params(S.scene_params(0.01))
    env, x, v, step = pressed_cube_state()
    dirs = {}
    for c in (1, 2, 4, 8, 16, 0, -1):
        sc = ipc.Scene(p, pcg_cluster=c)
        eid = sc.add_env(env)
        sc.set_state(eid, x, v, step)
        dirs[c] = sc.newton_direction(eid)
        if c > 0:
            assert sc.scene_counters(eid)["pcg_cluster"] == c
        elif c < 0:
            assert sc.scene_counters(eid)["pcg_cluster"] == 0
    big = ipc.Scene(p)
    big.add_env(S.pad_grasp_env(0, n_steps=40, close_steps=10))
    eid = big.add_env(env)
    big.set_state(eid, x, v, step)
    dirs["batch"] = big.newton_direction(eid)
    for k in (2, 4, 8, 16, 0, "batch"):
        assert np.array_equal(dirs[k], dirs[1]), k
    scale = np.abs(dirs[1]).max()
    assert np.abs(dirs[-1] - dirs[1]).max() <= 1e-9 * scale


def test_persistent_pcg_trajectory_matches_tiled():
    """Whole steps of the pad grasp with the persistent and the tiled PCG (default settings,
    PCG to 1e-4): both stay on the same trajectory to well inside 1e-6 m."""
    p = S.scene_params(0.005)
    env = S.pad_grasp_env(1, n_steps=30, close_steps=10)
    out = []
    for c in (0, -1):
        sc = ipc.Scene(p, pcg_cluster=c)
        eid = sc.add_env(env)
        sc.step(4)
        assert sc.status(eid)["status"] in ("ACTIVE", "DONE")
        out.append(sc.dofs(eid))
    assert np.abs(out[0] - out[1]).max() <= 1e-6


def test_pd_target_body_energy_gradient_and_trajectory_parity():
    """Free rigid box pulled toward a moving scheduled pose by the PD target potential: energy
    and gradient at a perturbed state (1e-10) and a 60-step trajectory (1e-6 m) match the oracle."""
    p = S.scene_params(0.01)
    env = S.pd_body_env(k_pd=900.0, n_steps=60, target_shift=(0.01, -0.02, 0.005), shift_steps=30)
    o, x, v = oracle_state(p, env, 7)
    q = x + np.random.default_rng(3).normal(size=x.size) * 1e-4
    _energy_parity(p, env, x, v, 7, q)
    pp = S.parity_params(p)
    o = O.OracleEnv(pp, env)
    o.step(60)
    xo, _ = o.state()
    sc = ipc.Scene(pp)
    eid = sc.add_env(env)
    sc.step(60)
    assert sc.status(eid)["status"] == "DONE"
    assert np.abs(sc.dofs(eid) - xo).max() <= TRAJ_TOL


def test_contacts_from_swept_candidates_give_the_same_bits_as_fresh_traversals():
    """Inside a time step the line-search trials and the later Newton iterations take their
    contacts from the step filter's swept candidates (boxes over [x, x + p] grown by dhat/2);
    a BVH traversal at every evaluation must give the same bits: same DOFs, same Newton,
    line-search, PCG and ACCD counts. Pad grasp from its contact phase and the squeezed cube."""
    pad = S.pad_grasp_env(3)
    x, v = S.pad_grasp_state_at(pad, 20)
    cube, xc, vc, step = pressed_cube_state()
    cases = [(S.scene_params(0.005), pad, x, v, 20, 6), (S.scene_params(0.01), cube, xc, vc, step, 6)]
    for p, env, x0, v0, s0, n in cases:
        out = []
        for fresh in (False, True):
            sc = ipc.Scene(p, fresh_broad_phase=fresh)
            eid = sc.add_env(env)
            sc.set_state(eid, x0, v0, s0)
            sc.step(n)
            out.append((sc.dofs(eid), sc.status(eid)))
        assert out[0][1]["status"] == "ACTIVE" and out[0][1]["ls_halvings"] >= 0
        assert out[0][1] == out[1][1]
        assert np.array_equal(out[0][0], out[1][0])


def test_one_call_of_k_steps_gives_the_bits_of_k_calls_of_one_step():
    """Inside one ipc_step call every env runs its steps at its own pace (an env done with a step
    starts the next while others still iterate). Each env's results must be those of stepping
    the batch one step per call: same DOFs and the same Newton, line-search, PCG and ACCD counts."""
    envs = [S.pad_grasp_env(i) for i in range(4)] + [S.cube_squeeze_env(1, n_steps=40, close_steps=20, dt=0.005)]
    p = S.scene_params(0.005)
    out = []
    for per_call in (6, 1):
        sc = ipc.Scene(p)
        ids = [sc.add_env(e) for e in envs]
        for eid, env in zip(ids[:4], envs[:4]):
            x, v = S.pad_grasp_state_at(env, 20)
            sc.set_state(eid, x, v, 20)
        for _ in range(6 // per_call):
            sc.step(per_call)
        out.append([(sc.dofs(e), sc.status(e)) for e in ids])
    for (xa, sa), (xb, sb) in zip(*out):
        assert sa["status"] == "ACTIVE" and sa == sb
        assert np.array_equal(xa, xb)


def test_batched_pad_grasps_do_the_work_of_each_alone():
    """Two pad grasps in contact stepped together: each env's DOFs and its Newton, line-search,
    PCG and ACCD counts equal those of stepping it alone (an env whose line search accepts keeps
    its point while the other env goes on halving)."""
    p = S.scene_params(0.005)
    envs = [S.pad_grasp_env(i) for i in range(2)]

    def run(which):
        sc = ipc.Scene(p)
        ids = [sc.add_env(envs[k]) for k in which]
        for eid, k in zip(ids, which):
            x, v = S.pad_grasp_state_at(envs[k], 20)
            sc.set_state(eid, x, v, 20)
        sc.step(3)
        return [(sc.dofs(e), sc.status(e)) for e in ids]

    both = run([0, 1])
    for k in (0, 1):
        (xa, sa), = run([k])
        assert sa["status"] == "ACTIVE" and sa == both[k][1]
        assert np.array_equal(xa, both[k][0])


def test_adapted_stiffness_trajectory_and_kappa_parity():
    """The single-env configuration as written: the squeezed cube (close 50 steps, lift 50) with
    the adapted barrier stiffness over all 100 steps. Per step, the GPU's kappa equals the
    oracle's (1e-9 relative: the step-start least squares sums in another order) and the
    trajectories agree within 1e-6 m; the stiffness did adapt."""
    p = dict(S.parity_params(S.scene_params(0.01)), kappa_adapt=True)
    env = S.cube_squeeze_env(0, n_steps=100)
    o = O.OracleEnv(p, env)
    sc = ipc.Scene(p)
    eid = sc.add_env(env)
    ks = []
    for k in range(100):
        o.step(1)
        sc.step(1)
        ks.append(o.kappa())
        assert abs(sc.kappa(eid) / o.kappa() - 1.0) <= 1e-9, (k, sc.kappa(eid), o.kappa())
        if k % 10 == 9:
            xo, _ = o.state()
            assert np.abs(sc.dofs(eid) - xo).max() <= TRAJ_TOL, k
    assert max(ks) > p["kappa"]
    assert sc.status(eid)["status"] == "DONE" and o.status()["status"] == "DONE"
    assert sc.invariants(eid) == {"intersections": 0, "inverted": 0}


def test_tet_stress_query_matches_the_oracle():
    """Per-tet von Mises stress of the squeezed cube at a pressed state: GPU query and oracle
    agree to 1e-12 of the largest stress, and the squeeze stresses the cube."""
    env, x, v, step = pressed_cube_state()
    p = S.scene_params(0.01)
    sc = ipc.Scene(p)
    eid = sc.add_env(env)
    sc.set_state(eid, x, v, step)
    nt = len(env["soft"][0]["tets"])
    sg = sc.tet_stress(eid)
    so = O.OracleEnv(p, env).tet_stress(x, nt)
    assert sg.shape == (nt,)
    assert np.abs(sg - so).max() <= 1e-12 * np.abs(so).max()
    assert so.max() > 0.0


def test_contact_force_query_matches_the_oracle():
    """Normal contact forces of the squeezed cube at a pressed state, in the contact list's order:
    GPU query and oracle agree to 1e-10 relative; the list matches the contacts query."""
    env, x, v, step = pressed_cube_state()
    p = S.scene_params(0.01)
    sc = ipc.Scene(p)
    eid = sc.add_env(env)
    sc.set_state(eid, x, v, step)
    fg = sc.contact_forces(eid)
    o = O.OracleEnv(p, env)
    fo = o.contact_forces(x)
    assert len(fg) == len(sc.contacts(eid)) == len(fo) > 0
    assert np.abs(fg - fo).max() <= 1e-10 * np.abs(fo).max()


def test_friction_force_query_matches_the_oracle():
    """Friction forces of a rigid box sliding down a 20 deg incline (mu = 0.2) after 20 steps:
    the GPU's and the oracle's lagged friction stencils give the same forces (compared sorted:
    the two lists may order an env's stencils differently) to 1e-6 relative."""
    p = S.scene_params(0.01, newton_tol=1e-8)
    env = S.resting_env("rigid", n_steps=30, mu=0.2, incline_deg=20.0)
    o = O.OracleEnv(p, env)
    o.step(20)
    sc = ipc.Scene(p)
    eid = sc.add_env(env)
    sc.step(20)
    xo, _ = o.state()
    fo = np.sort(o.friction_forces(xo))
    fg = np.sort(sc.friction_forces(eid))
    assert len(fg) == len(fo) >= 3
    assert np.abs(fg - fo).max() <= 1e-6 * fo.max()


def test_axis_gravity_phases_match_the_oracle():
    """A rigid box resting on the ground through the six axis-aligned gravity phases of the
    evaluation protocol (codes 2..7, five steps each, after five steps of plain gravity): GPU
    and oracle trajectories agree within 1e-6 m."""
    p = S.parity_params(S.scene_params(0.01))
    codes = [1] * 5 + [c for c in range(2, 8) for _ in range(5)]
    env = S.resting_env("rigid", n_steps=len(codes), mu=0.5)
    env["gravity"] = np.asarray(codes, dtype=np.uint8)
    o = O.OracleEnv(p, env)
    sc = ipc.Scene(p)
    eid = sc.add_env(env)
    for k in range(0, len(codes), 5):
        o.step(5)
        sc.step(5)
        xo, _ = o.state()
        assert np.abs(sc.dofs(eid) - xo).max() <= TRAJ_TOL, k
    assert sc.status(eid)["status"] == "DONE"


@pytest.mark.parametrize("slots", [1, 3])
def test_spilled_collect_traversals_give_the_same_candidates_and_bits(slots):
    """A collect traversal keeps up to `collect_slots` partners per query; a query with more sends
    the pass to a count-then-fill traversal (the candidate-buffer overflow case). With 1 or 3
    slots nearly every pass spills: the candidate and contact lists of the squeezed cube still
    equal the oracle's, and ten steps of the pad grasp from its contact phase give the same bits,
    Newton, line-search, PCG and ACCD counts as with the default 128 slots."""
    p = S.scene_params(0.01)
    env = S.cube_squeeze_env(0, n_steps=40, close_steps=20)
    o, x, v = oracle_state(p, env, 25)
    sc = ipc.Scene(p, collect_slots=slots)
    eid = sc.add_env(env)
    sc.set_state(eid, x, v, 25)
    assert np.array_equal(sc.candidates(eid), o.candidates(x))
    ko, _ = o.contacts(x)
    assert len(ko) > 10 and np.array_equal(sc.contacts(eid)[:, :3], ko[:, :3])
    assert sc.scene_counters(eid)["collect_spills"] > 0

    pp = S.scene_params(0.005)
    pad = S.pad_grasp_env(0)
    xs, vs = S.pad_grasp_state_at(pad, 20)
    runs = []
    for c in (0, slots):
        s2 = ipc.Scene(pp, collect_slots=c)
        e2 = s2.add_env(pad)
        s2.set_state(e2, xs, vs, 20)
        s2.step(10)
        st = s2.status(e2)
        runs.append((s2.dofs(e2), [st[k] for k in ("newton_iters", "pcg_iters", "ls_halvings", "accd_iters")],
                     s2.scene_counters(e2)["collect_spills"]))
    assert runs[0][2] == 0 and runs[1][2] > 0
    assert np.array_equal(runs[0][0], runs[1][0]) and runs[0][1] == runs[1][1]


def test_energy_trace_query_matches_the_oracle_trace():
    """IPC_Q_ENERGY_TRACE: the incremental potential at every Newton iterate of a step, as the
    oracle records it, for the squeezed cube's 12th step (in contact, eight iterations, the first
    with the plates still off target; parity settings): same number of iterates, energies within
    1e-9 relative."""
    p = S.parity_params(S.scene_params(0.01))
    env = S.cube_squeeze_env(0, n_steps=40, close_steps=20)
    o = O.OracleEnv(p, env)
    o.trace(True)
    sc = ipc.Scene(p)
    eid = sc.add_env(env)
    for k in range(12):
        o.step(1)
        sc.step(1)
    rows = o.trace_energies()
    last = rows[rows[:, 0] == rows[:, 0].max()]
    eo = last[:, 3]
    eg = sc.energy_trace(eid)
    assert len(eo) >= 2 and len(eg) == len(eo), (len(eg), len(eo))
    assert np.all(np.abs(eg - eo) <= 1e-9 * np.abs(eo)), (eg, eo)
    # once the kinematic parts sit on their targets (the oracle's flag), the line search never
    # raises the energy
    free = eg[last[:, 2] == 0]
    assert len(free) >= 2 and np.all(np.diff(free) <= 1e-12 * np.abs(free[:-1]))
