"""Scene-level pins of the CPU oracle: closed-form motions, static equilibrium, friction limits,
rigidity, finite-difference gradients and the stepping invariants (no GPU)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_05020_b300 import scenes as S

G = 9.8


def test_free_fall_matches_implicit_euler_closed_form():
    """No contact, rigid translation: v_{n+1} = v_n + h g and x_{n+1} = x_n + h v_{n+1}."""
    h = 0.01
    p = S.scene_params(h)
    env = S.single_tet_env(n_steps=10)
    e = O.OracleEnv(p, env)
    x0, _ = e.state()
    assert e.step(10) == "DONE"
    x, v = e.state()
    vz = 0.0
    z = 0.0
    for _ in range(10):
        vz = vz - h * G
        z = z + h * vz
    assert np.allclose(v.reshape(-1, 3)[:, 2], vz, rtol=1e-9)
    assert np.allclose((x - x0).reshape(-1, 3)[:, 2], z, rtol=1e-9)
    assert np.allclose((x - x0).reshape(-1, 3)[:, :2], 0, atol=1e-12)


@pytest.mark.parametrize("body", ["tet", "rigid", "block"])
def test_resting_body_contact_forces_balance_weight(body):
    """Static equilibrium on a ground triangle: sum of kappa |b'(d_k)| = m g (barrier in N)."""
    p = S.scene_params(0.01, newton_tol=1e-8)
    env = S.resting_env(body, n_steps=150)
    e = O.OracleEnv(p, env)
    assert e.step(150) == "DONE"
    x, v = e.state()
    _, d2 = e.contacts(x)
    assert len(d2) >= 3 and np.all(np.sqrt(d2) < p["dhat"]) and np.all(d2 > 0)
    F = sum(p["kappa"] * abs(O.barrier(math.sqrt(q), p["dhat"])[1]) for q in d2)
    if body == "rigid":
        M, vol = e.body_mass(0)
        m = M[0, 0]
    else:
        m = e.soft_mass(len(env["soft"][0]["verts"])).sum()
    tol = 5e-5 if body == "block" else 1e-5
    assert abs(F / (m * G) - 1) < tol
    # the contact-force query reports the same normal forces
    assert abs(e.contact_forces(x).sum() / (m * G) - 1) < tol


def _slope_velocity(e, env, incline_deg):
    x, v = e.state()
    th = math.radians(incline_deg)
    down = np.array([math.cos(th), 0, -math.sin(th)])  # direction of steepest descent
    return float(v[0:3] @ down)


@pytest.mark.slow
def test_incline_stick_and_slip():
    """Rigid box on a 20 deg incline: mu > tan(th) sticks (creep below eps_v); mu < tan(th)
    slides with acceleration g (sin th - mu cos th). A tight Newton tolerance is used because
    the normal forces that friction lags are only as accurate as the force residual, and a
    step-size stopping rule leaves large residuals against the stiff barrier."""
    th = 20.0
    p = S.scene_params(0.01, newton_tol=1e-8)
    env = S.resting_env("rigid", n_steps=60, mu=0.5, incline_deg=th)
    e = O.OracleEnv(p, env)
    assert e.step(60) == "DONE"
    assert abs(_slope_velocity(e, env, th)) < p["eps_v"]
    mu = 0.2
    env = S.resting_env("rigid", n_steps=60, mu=mu, incline_deg=th)
    e = O.OracleEnv(p, env)
    e.step(20)
    v20 = _slope_velocity(e, env, th)
    e.step(30)
    v50 = _slope_velocity(e, env, th)
    a = (v50 - v20) / (30 * 0.01)
    ref = G * (math.sin(math.radians(th)) - mu * math.cos(math.radians(th)))
    assert abs(a / ref - 1) < 0.02


def test_spinning_body_stays_rigid():
    p = S.scene_params(0.01)
    env = S.spinning_body_env(n_steps=20, omega=(0, 0, 20.0))
    e = O.OracleEnv(p, env)
    assert e.step(20) == "DONE"
    x, _ = e.state()
    A = np.stack([x[3:6], x[6:9], x[9:12]], axis=1)
    assert np.abs(A @ A.T - np.eye(3)).max() < 1e-3
    # it did rotate: about 20 rad/s * 0.2 s = 4 rad, up to implicit-Euler damping
    ang = math.atan2(A[1, 0], A[0, 0])
    assert abs(ang) > 0.3


def _fd_check(e, q, idx, rel=1e-5):
    E, g = e.eval(q)
    scale = np.abs(g).max()
    for i in idx:
        h = 1e-8 if i < e.ndof else 1e-8
        qp = q.copy()
        qm = q.copy()
        qp[i] += h
        qm[i] -= h
        fd = (e.eval(qp, grad=False) - e.eval(qm, grad=False)) / (2 * h)
        assert abs(fd - g[i]) <= rel * scale + 1e-9 * abs(g[i]), (i, fd, g[i], scale)


def test_env_gradient_matches_finite_differences_with_contact_and_friction():
    """Whole incremental potential (inertia, Neo-Hookean, barrier, lagged friction, affine
    inertia/orthogonality) against central differences at a state with active contacts."""
    p = S.scene_params(0.01)
    env = S.cube_squeeze_env(0, n_steps=40, close_steps=20)
    e = O.OracleEnv(p, env)
    e.step(30)  # plates in contact, lifting phase (gravity and friction active)
    x, v = e.state()
    c, _ = e.contacts(x)
    assert len(c) > 10
    rng = np.random.default_rng(0)
    q = x + rng.normal(size=x.size) * 1e-6
    # pick DOFs of surface vertices touching the plates plus random ones
    idx = sorted(set(rng.choice(e.ndof, 40, replace=False).tolist()) | {0, 1, 2})
    _fd_check(e, q, idx)


def test_env_gradient_fd_rigid_body_terms():
    p = S.scene_params(0.01)
    env = S.resting_env("rigid", n_steps=30, mu=0.4, incline_deg=10)
    e = O.OracleEnv(p, env)
    e.step(20)
    x, _ = e.state()
    q = x.copy()
    q[3:12] += np.random.default_rng(1).normal(size=9) * 1e-4  # break orthogonality a little
    _fd_check(e, q, list(range(12)))


def test_hessian_is_symmetric_psd():
    p = S.scene_params(0.01)
    env = S.cube_squeeze_env(0, n_steps=40, close_steps=20)
    e = O.OracleEnv(p, env)
    e.step(25)
    x, _ = e.state()
    H = e.hessian(x)
    assert np.allclose(H, H.T, atol=1e-12 * np.abs(H).max())
    # free block (soft DOFs): PSD up to round-off
    n = 3 * 125
    w = np.linalg.eigvalsh(H[:n, :n])
    assert w.min() > -1e-10 * w.max()


def test_line_search_energy_is_monotone():
    """Within each step, every unconstrained Newton iteration does not increase the energy."""
    p = S.scene_params(0.01)
    env = S.cube_squeeze_env(0, n_steps=30, close_steps=15)
    e = O.OracleEnv(p, env)
    e.trace(True)
    assert e.step(30) == "DONE"
    tr = e.trace_energies()
    n_checked = 0
    for k in range(len(tr) - 1):
        s, it, constrained, E = tr[k]
        s2, it2, _, E2 = tr[k + 1]
        if s2 == s and it2 == it + 1 and constrained == 0:
            assert E2 <= E
            n_checked += 1
    assert n_checked > 10


def test_constraint_candidates_are_conservative():
    """Every non-excluded pair closer than dhat appears among the dhat/2-inflated candidates."""
    p = S.scene_params(0.01)
    env = S.cube_squeeze_env(0, n_steps=40, close_steps=20)
    e = O.OracleEnv(p, env)
    e.step(25)
    x, _ = e.state()
    cand = {tuple(r) for r in e.candidates(x)}
    contacts, d2 = e.contacts(x)
    assert len(contacts) > 0
    for r in contacts:
        assert (r[0], r[1], r[2]) in cand
    assert np.all(d2 < p["dhat"] ** 2)
    # the list's form (what the GPU list must equal bit for bit): sorted by (kind, i, j), no
    # duplicate, each edge-edge pair once with i < j; the same for the swept (CCD) list
    for c in (e.candidates(x), e.candidates(x, e.newton_direction())):
        rows = [tuple(r) for r in c]
        assert rows == sorted(set(rows)) and len(rows) > 0
        ee = c[c[:, 0] == 1]
        assert len(ee) > 0 and np.all(ee[:, 1] < ee[:, 2])


@pytest.mark.slow
@pytest.mark.parametrize("mu, lifts", [(0.5, True), (0.0, False)])
def test_cube_grasp_lift_outcome_and_invariants(mu, lifts):
    """Plates squeeze the cube with gravity off, then lift with gravity on: with friction the
    cube follows the plates up; without friction it is not lifted. No intersection and no
    inverted tet at any checked step."""
    p = S.scene_params(0.01)
    env = S.cube_squeeze_env(0, n_steps=50, close_steps=30, mu=mu)
    e = O.OracleEnv(p, env)
    x0, _ = e.state()
    z0 = x0[: 3 * 125].reshape(-1, 3)[:, 2].mean()
    for s in range(5):
        e.step(10)
        x, _ = e.state()
        inv = e.invariants(x)
        assert inv["intersections"] == 0 and inv["inverted"] == 0 and inv["min_dist"] > 0
    assert e.status()["status"] == "DONE"
    x, _ = e.state()
    dz = x[: 3 * 125].reshape(-1, 3)[:, 2].mean() - z0
    plate_dz = 20 * 0.01 * 0.02
    if lifts:
        assert abs(dz - plate_dz) < 0.1 * plate_dz
    else:
        assert dz < 0.2 * plate_dz


def test_pd_target_body_sags_by_g_over_kpd():
    """A free box held toward its initial pose by the PD target potential
    1/2 h^2 k_pd (q - q^)^T (M4 x I3) (q - q^) settles under gravity where k_pd * offset = g:
    an offset of g / k_pd straight down, with A staying at I (implicit Euler damps the
    oscillation; omega h = 0.2 decays it by ~1e-4 over 500 steps)."""
    k = 400.0
    p = S.scene_params(0.01)
    env = S.pd_body_env(k_pd=k, n_steps=500)
    e = O.OracleEnv(p, env)
    e.step(500)
    x, v = e.state()
    assert abs(x[2] - (-G / k)) <= 2e-3 * G / k
    assert np.abs(x[:2]).max() < 1e-9
    assert np.abs(x[3:12] - S.IDENTITY_Q[3:12]).max() < 1e-6


def test_env_gradient_fd_pd_target_term():
    p = S.scene_params(0.01)
    env = S.pd_body_env(k_pd=900.0, n_steps=30, target_shift=(0.01, -0.02, 0.005), shift_steps=10)
    e = O.OracleEnv(p, env)
    e.step(5)
    x, _ = e.state()
    q = x + np.random.default_rng(2).normal(size=x.size) * 1e-4
    _fd_check(e, q, list(range(12)))


@pytest.mark.parametrize("floor", [1.0, 1e-2, 1e-4, 1e3])
def test_adapted_stiffness_at_rest_balances_the_contact_vertices_weight(floor):
    """Adapted barrier stiffness at a step start: the kappa that minimises |g_E + kappa G| over
    the free DOFs (g_E: gradient of every other term, G: the barrier's per unit kappa). A soft
    block at rest with its 9 bottom vertices a gap d above a fixed ground triangle, gravity on,
    has g_E = m_i h^2 g on each vertex and G = h^2 b'(d) on the bottom ones, so kappa equals
    g times the bottom vertices' mean mass over |b'(d)| (b' written out from
    b(d) = -(d - dhat)^2 ln(d / dhat)), clamped to [floor, 1000 floor] with the scene's kappa
    as the floor. The floors put that value near the bottom of the range, at about 250 times
    the floor, above the range (clamped to 1000 times the floor) and below it (held at the
    floor)."""
    h = 0.01
    p = S.scene_params(h, kappa=floor)
    p["kappa_adapt"] = True
    gap = 0.5 * p["dhat"]
    env = S.resting_env("block", n_steps=2, gap=gap)
    e = O.OracleEnv(p, env)
    e.step(1)
    verts = np.asarray(env["soft"][0]["verts"])
    m = e.soft_mass(len(verts))
    bottom = np.abs(verts[:, 2] - gap) < 1e-12
    assert bottom.sum() == 9
    d, dh = gap, p["dhat"]
    b1 = -2.0 * (d - dh) * math.log(d / dh) - (d - dh) ** 2 / d
    balance = G * m[bottom].mean() / abs(b1)
    if balance <= floor:
        assert e.kappa() == floor
    elif balance < 1000.0 * floor:
        assert abs(e.kappa() / balance - 1.0) < 1e-9
    else:
        assert e.kappa() == 1000.0 * floor


def test_adapted_stiffness_stays_in_its_bounds_and_keeps_the_invariants():
    """Squeezed cube with the adapted stiffness: every step's kappa lies in [kappa, 1000 kappa]
    of the scene, and the run stays free of intersections and inverted tets; without adaptation
    the stiffness is the scene's throughout."""
    p = S.scene_params(0.01)
    env = S.cube_squeeze_env(0, n_steps=30, close_steps=15)
    fixed = O.OracleEnv(p, env)
    fixed.step(3)
    assert fixed.kappa() == p["kappa"]
    pa = dict(p, kappa_adapt=True)
    e = O.OracleEnv(pa, env)
    ks = []
    for _ in range(30):
        assert e.step(1) in ("ACTIVE", "DONE")
        ks.append(e.kappa())
        x, _ = e.state()
        inv = e.invariants(x)
        assert inv["intersections"] == 0 and inv["inverted"] == 0
    assert min(ks) >= p["kappa"] and max(ks) <= 1000.0 * p["kappa"]
    assert max(ks) > p["kappa"]  # contact made the stiffness adapt


def test_friction_forces_of_a_sliding_and_a_sticking_box():
    """Rigid box on a 20 deg incline. Sliding (mu = 0.2 < tan 20 deg): every lagged friction
    stencil is past the smoothing, so the friction forces add up to mu m g cos th (kinetic
    friction). Sticking (mu = 0.5): they balance the slope component of the weight, m g sin th."""
    th = math.radians(20.0)
    p = S.scene_params(0.01, newton_tol=1e-8)
    for mu, expect in ((0.2, lambda m: mu * m * G * math.cos(th)), (0.5, lambda m: m * G * math.sin(th))):
        env = S.resting_env("rigid", n_steps=30, mu=mu, incline_deg=20.0)
        e = O.OracleEnv(p, env)
        e.step(30)
        x, _ = e.state()
        f = e.friction_forces(x)
        M, _vol = e.body_mass(0)
        assert len(f) >= 3
        assert abs(f.sum() / expect(M[0, 0]) - 1.0) < 0.02, (mu, f.sum(), expect(M[0, 0]))


@pytest.mark.parametrize("code", [2, 3, 4, 5, 6, 7])
def test_axis_gravity_phase_free_fall(code):
    """Gravity codes 2..7 pull with the scene's |g| along +x, -x, +y, -y, +z, -z: a free tet
    falls along that axis by the implicit-Euler closed form, and not at all across it."""
    h, n = 0.01, 8
    p = S.scene_params(h)
    env = S.single_tet_env(n_steps=n)
    env["gravity"] = np.full(n, code, dtype=np.uint8)
    e = O.OracleEnv(p, env)
    x0, _ = e.state()
    e.step(n)
    x, v = e.state()
    axis, sign = (code - 2) // 2, (1.0 if code % 2 == 0 else -1.0)
    vz = z = 0.0
    for _ in range(n):
        vz += h * sign * G
        z += h * vz
    d = (x - x0).reshape(-1, 3)
    assert np.allclose(d[:, axis], z, rtol=1e-9)
    assert np.abs(np.delete(d, axis, axis=1)).max() <= 1e-12


@pytest.mark.parametrize("adapt", [False, True])
def test_friction_acts_on_tangential_motion_only_and_parallel_edges_carry_no_force(adapt):
    """A rigid cube at rest on a wider fixed box, with one edge-edge contact between exactly
    parallel edges (the two boxes' face diagonals, one above the other). The mollified barrier
    of parallel edges vanishes with its gradient, so that pair carries no normal force and the
    remaining lagged normal forces alone balance the weight (static equilibrium). Friction acts
    on the tangential part of the relative motion only: moving the cube straight up draws no
    friction force, moving it sideways by more than eps_v h draws mu times the normal forces,
    i.e. mu m g in total (Coulomb's kinetic friction). With the adapted barrier stiffness the
    lagged normal forces are those of the step's adapted kappa."""
    p = S.scene_params(0.01, newton_tol=1e-8)
    p["kappa_adapt"] = adapt
    mu = 0.5
    env = S.stacked_boxes_env(n_steps=150, mu=mu)
    e = O.OracleEnv(p, env)
    assert e.step(150) == "DONE"
    x, _ = e.state()
    M, _vol = e.body_mass(0)
    mg = M[0, 0] * G
    pairs, _d2 = e.contacts(x)
    cf = e.contact_forces(x)
    assert (e.kappa() > p["kappa"]) == adapt
    assert len(cf) == len(pairs) >= 8 and (pairs[:, 0] == 1).any()
    assert cf.min() < 1e-6 * cf.max()  # the parallel edge-edge pair
    assert abs(cf.sum() / mg - 1.0) < 1e-5
    shift = 10.0 * p["eps_v"] * p["dt"]
    for axis, expect in ((2, 0.0), (0, mu * mg), (1, mu * mg)):
        q = x.copy()
        q[axis] += shift  # the cube's translation DOFs
        f = e.friction_forces(q)
        assert len(f) == len(pairs)
        if expect == 0.0:
            assert f.sum() < 1e-3 * mu * mg
        else:
            assert abs(f.sum() / expect - 1.0) < 1e-5


def test_lumped_masses_carry_the_body_mass_and_centroid():
    """Lumped vertex masses (a quarter of each tet's rho V_e to each of its corners) add up to
    rho times the body's volume and have the body's centroid as their centre (a linear tet's
    centroid is the mean of its corners). Checked on an L-shaped block of 3 unit cells, whose
    volume and centroid follow from the cells alone."""
    a, rho = 0.01, 1300.0
    mask = np.ones((2, 2, 1), dtype=bool)
    mask[1, 1, 0] = False
    verts, tets, _ = S.kuhn_grid(2, 2, 1, (0.0, 0.0, 0.0), (2 * a, 2 * a, a), cell_mask=mask)
    tris = S.boundary_tris(verts, tets)
    soft = dict(verts=verts, tets=tets, tris=tris, E=1e5, nu=0.4, rho=rho, kin=np.zeros(len(verts), dtype=np.uint8))
    env = dict(soft=[soft], affine=[], mu=0.0, gravity=np.zeros(1, dtype=np.uint8),
               targets=np.tile(S.IDENTITY_Q, (1, 1, 1)))
    e = O.OracleEnv(S.scene_params(0.01), env)
    m = e.soft_mass(len(verts))
    cells = np.array([[0.5, 0.5, 0.5], [1.5, 0.5, 0.5], [0.5, 1.5, 0.5]]) * a
    assert abs(m.sum() / (rho * 3 * a ** 3) - 1.0) < 1e-12
    assert np.allclose(m @ verts / m.sum(), cells.mean(axis=0), rtol=1e-12, atol=1e-15)


def test_thin_rigid_plate_has_no_self_contact():
    """A free rigid plate thinner than dhat in free fall: its top and bottom faces are closer
    than dhat, but points of one rigid body never meet, so the plate has no contact candidates,
    falls by the implicit-Euler closed form and keeps A = I (no barrier pushes its faces apart)."""
    h, n = 0.01, 10
    p = S.scene_params(h)
    pv, pt = S.box_surface((0.02, 0.015, 0.25 * p["dhat"]))
    plate = dict(verts=pv, tris=pt, rho=900.0, q0=S.IDENTITY_Q.copy(), qdot0=np.zeros(12), kinematic=False)
    env = dict(soft=[], affine=[plate], mu=0.5, gravity=np.ones(n, dtype=np.uint8),
               targets=np.tile(S.IDENTITY_Q, (n, 1, 1)))
    e = O.OracleEnv(p, env)
    x0, _ = e.state()
    assert len(e.candidates(x0)) == 0
    assert e.step(n) == "DONE"
    x, _ = e.state()
    vz = z = 0.0
    for _ in range(n):
        vz -= h * G
        z += h * vz
    assert math.isclose(x[2] - x0[2], z, rel_tol=1e-9)
    assert np.abs(x[3:12] - S.IDENTITY_Q[3:12]).max() < 1e-12


def _fd_hessian(e, q, idx, step=1e-9):
    cols = []
    for i in idx:
        qp, qm = q.copy(), q.copy()
        qp[i] += step
        qm[i] -= step
        cols.append((e.eval(qp)[1] - e.eval(qm)[1]) / (2 * step))
    return np.array(cols).T


def test_hessian_matches_finite_differences_where_no_projection_acts():
    """The assembled Hessian against central differences of the gradient, at states where every
    element Hessian is already PSD, so that the projection leaves it as it is. (1) A rigid cube
    lifted 3 dhat off the box it rested on: no barrier is active, its lagged friction stencils
    are (the friction Hessian, PSD inside and past the eps_v h smoothing), and A = I (the
    orthogonality Hessian is its PSD Gauss-Newton part there). (2) A free stiff soft block at a
    strain of about 1e-6, where the Neo-Hookean Hessian is linear elasticity's up to a
    projection of eigenvalues of the order of the strain."""
    p = S.scene_params(0.01, newton_tol=1e-8)
    e = O.OracleEnv(p, S.stacked_boxes_env(n_steps=150, mu=0.5))
    assert e.step(150) == "DONE"
    x, _ = e.state()
    eh = p["eps_v"] * p["dt"]
    for slide in (0.3 * eh, 3.0 * eh):
        q = x.copy()
        q[2] += 3.0 * p["dhat"]
        q[0] += slide
        q[1] += 0.5 * slide
        assert len(e.contacts(q)[0]) == 0
        H = e.hessian(q)[:12, :12]
        Hf = _fd_hessian(e, q, range(12))[:12]
        assert np.abs(H - Hf).max() <= 1e-6 * np.abs(H).max()

    a = 0.01
    verts, tets, _ = S.kuhn_grid(2, 2, 2, (0.0, 0.0, 0.0), (2 * a, 2 * a, 2 * a))
    soft = dict(verts=verts, tets=tets, tris=S.boundary_tris(verts, tets), E=1e7, nu=0.4, rho=1000.0,
                kin=np.zeros(len(verts), dtype=np.uint8))
    env = dict(soft=[soft], affine=[], mu=0.0, gravity=np.zeros(2, dtype=np.uint8),
               targets=np.tile(S.IDENTITY_Q, (2, 1, 1)))
    e = O.OracleEnv(S.scene_params(0.01), env)
    e.step(1)
    x, _ = e.state()
    q = x + np.random.default_rng(3).normal(size=x.size) * 1e-6 * a
    H = e.hessian(q)
    Hf = _fd_hessian(e, q, range(e.ndof))
    elastic = H - np.diag(np.repeat(e.soft_mass(len(verts)), 3))
    assert np.abs(H - Hf).max() <= 1e-5 * np.abs(elastic).max()


def test_invariant_checks_report_what_they_count():
    """The invariants asserted after every step do report violations. A cube placed a gap g above
    the box it rests on has no intersection and minimum distance g (its bottom corners over the
    box's top face); pushed halfway into the box (off-centre, so that no crossing falls on a
    triangle's boundary), its vertical edges pierce the box's top face. A tet with its apex
    reflected through its base plane is inverted."""
    p = S.scene_params(0.01)
    e = O.OracleEnv(p, S.stacked_boxes_env(n_steps=2))
    x, _ = e.state()
    for gap in (0.3e-3, 2e-3):
        q = x.copy()
        q[2] = 0.02 + gap
        inv = e.invariants(q)
        assert inv["intersections"] == 0 and inv["inverted"] == 0
        assert abs(inv["min_dist"] / gap - 1.0) < 1e-9
    q = x.copy()
    q[0:3] = [0.0031, -0.0017, 0.0137]
    inv = e.invariants(q)
    assert inv["intersections"] >= 4

    e = O.OracleEnv(p, S.single_tet_env(n_steps=2))
    x, _ = e.state()
    assert e.invariants(x)["inverted"] == 0
    q = x.copy()
    q[11] = -q[11]  # apex (0, 0, 0.01) to (0, 0, -0.01): the base plane is z = 0
    assert e.invariants(q)["inverted"] == 1


def test_kinematic_bodies_sit_on_their_scheduled_poses():
    """Kinematic parts take their scheduled pose of each step exactly: a soft tet whose four
    vertices are all driven (x = p + A X0 for the step's handle pose q = (p, A)) and a
    kinematic rigid box (q equals the step's entry), on a schedule that turns about z and
    translates, one entry per step."""
    n, h = 6, 0.01
    tet = S.single_tet_env(n_steps=n)
    soft = dict(tet["soft"][0], kin=np.ones(4, dtype=np.uint8))
    bv, bt = S.box_surface((0.01, 0.01, 0.01))
    box = dict(verts=bv, tris=bt, rho=700.0, q0=S.IDENTITY_Q.copy(), qdot0=np.zeros(12), kinematic=True)
    targets = np.zeros((n, 2, 12))
    for s in range(n):
        c, sn = math.cos(0.1 * (s + 1)), math.sin(0.1 * (s + 1))
        R = np.array([[c, -sn, 0.0], [sn, c, 0.0], [0.0, 0.0, 1.0]])
        targets[s, 0] = np.concatenate([[0.001 * (s + 1), 0.0, 0.0], R[:, 0], R[:, 1], R[:, 2]])
        targets[s, 1] = np.concatenate([[0.2, 0.002 * (s + 1), 0.0], R[:, 0], R[:, 1], R[:, 2]])
    env = dict(soft=[soft], affine=[box], mu=0.0, gravity=np.ones(n, dtype=np.uint8), targets=targets)
    e = O.OracleEnv(S.scene_params(h), env)
    X0 = np.asarray(soft["verts"])
    for s in range(n):
        e.step(1)
        x, _ = e.state()
        q = targets[s, 0]
        A = np.stack([q[3:6], q[6:9], q[9:12]], axis=1)
        assert np.abs(x[:12].reshape(4, 3) - (X0 @ A.T + q[:3])).max() < 1e-15
        assert np.abs(x[12:24] - targets[s, 1]).max() < 1e-15


def test_pd_target_body_follows_the_implicit_euler_spring():
    """Gravity off, a free box pulled by the PD potential toward targets that move over the
    first steps: every step minimises 1/2 |q - q~|_M^2 + 1/2 h^2 k |q - q^|_M^2 (A stays at I,
    so the orthogonality term is zero), whose minimiser is q = (q~ + h^2 k q^) / (1 + h^2 k)
    with q~ = q + h v and q^ this step's target: the implicit-Euler recurrence of a spring."""
    k, h, n = 900.0, 0.01, 12
    env = S.pd_body_env(k_pd=k, n_steps=n, gravity=False, target_shift=(0.01, -0.02, 0.005), shift_steps=5)
    e = O.OracleEnv(S.scene_params(h, newton_tol=1e-10), env)
    q, v = S.IDENTITY_Q.copy(), np.zeros(12)
    for s in range(n):
        q_next = (q + h * v + h * h * k * env["targets"][s, 0]) / (1.0 + h * h * k)
        v, q = (q_next - q) / h, q_next
        assert e.step(1) in ("ACTIVE", "DONE")
        x, _ = e.state()
        assert np.abs(x - q).max() < 1e-9 * 0.02


def test_gated_gravity_starts_with_its_schedule():
    """Gravity gated per step (off for the first steps, as in the closing phase of a grasp): a
    free tet does not move while gravity is off, then falls by the implicit-Euler closed form."""
    h, n, off = 0.01, 8, 3
    env = S.single_tet_env(n_steps=n)
    env["gravity"] = np.array([0] * off + [1] * (n - off), dtype=np.uint8)
    e = O.OracleEnv(S.scene_params(h), env)
    x0, _ = e.state()
    vz = z = 0.0
    for s in range(n):
        e.step(1)
        if s >= off:
            vz -= h * G
            z += h * vz
        x, _ = e.state()
        assert np.allclose((x - x0).reshape(-1, 3)[:, 2], z, rtol=1e-9, atol=1e-15)


def test_failure_semantics_newton_cap_and_non_finite_state():
    """An env that does not converge within its Newton cap is marked failed (Sec. III-D: after
    N_iters iterations), as is one whose state is not finite; a failed env takes no further step."""
    p = S.scene_params(0.01)
    p["max_newton"] = 1
    e = O.OracleEnv(p, S.cube_squeeze_env(0, n_steps=10, close_steps=5))
    assert e.step(3) == "FAILED"
    st = e.status()
    assert st["reason"] == 1 and st["steps_done"] == 0 and st["newton_iters"] == 1
    x, _ = e.state()
    assert e.step(2) == "FAILED" and e.status()["newton_iters"] == 1
    assert np.array_equal(e.state()[0], x)

    e = O.OracleEnv(S.scene_params(0.01), S.resting_env("block", n_steps=5))
    x, v = e.state()
    v = v.copy()
    v[4] = np.nan
    e.set_state(x, v, 0)
    assert e.step(1) == "FAILED" and e.status()["reason"] == 3


def test_a_step_at_equilibrium_converges_in_one_newton_iteration():
    """Stopping rule |p|_inf / h < tol: once a body rests in equilibrium, the first Newton step
    of the next time step is already below the tolerance."""
    p = S.scene_params(0.01, newton_tol=1e-6)
    e = O.OracleEnv(p, S.resting_env("rigid", n_steps=200))
    e.step(190)
    n0 = e.status()["newton_iters"]
    assert e.step(5) == "ACTIVE"
    assert e.status()["newton_iters"] - n0 == 5


def _sym_fd_hessian(e, q, step):
    H = _fd_hessian(e, q, range(len(q)), step)
    return 0.5 * (H + H.T)


def _free_tet(v):
    t = np.array([[0, 1, 2, 3]], dtype=np.int32)
    if np.linalg.det(np.stack([v[1] - v[0], v[2] - v[0], v[3] - v[0]])) < 0:
        t = np.array([[0, 2, 1, 3]], dtype=np.int32)
    return dict(verts=v, tets=t, tris=S.boundary_tris(v, t), E=1e5, nu=0.4, rho=1000.0, kin=np.zeros(4, dtype=np.uint8))


def test_projection_makes_the_hessian_psd_where_the_raw_one_is_not():
    """Projected Newton: every element Hessian is projected to PSD before assembly, so the
    assembled Hessian is PSD even where the exact one (central differences of the gradient) is
    indefinite. With dt = 1 s the element terms dominate the mass: a strongly compressed and
    sheared tet (Neo-Hookean), a tet's vertex 0.3 dhat below another free tet's face (barrier),
    and an affine body at A = I/2 (orthogonality)."""
    p = S.scene_params(1.0)
    env = S.single_tet_env(n_steps=2)
    env["gravity"][:] = 0
    e = O.OracleEnv(p, env)
    e.step(1)
    x, _ = e.state()
    q = x.copy()
    q[9:12] = [0.002, 0.001, 0.003]
    cases = [(e, q, 1e-10)]

    g = 0.3 * p["dhat"]
    a = np.array([[0, 0, 0], [0.01, 0, 0], [0, 0.01, 0], [0, 0, 0.01]], dtype=np.float64)
    b = np.array([[0.002, 0.002, -g], [-0.003, -0.003, -g - 0.01], [0.007, -0.003, -g - 0.01],
                  [-0.003, 0.007, -g - 0.01]])
    env = dict(soft=[_free_tet(a), _free_tet(b)], affine=[], mu=0.0, gravity=np.zeros(2, dtype=np.uint8),
               targets=np.tile(S.IDENTITY_Q, (2, 2, 1)))
    e = O.OracleEnv(p, env)
    x, _ = e.state()
    assert len(e.contacts(x)[0]) == 1
    cases.append((e, x, 1e-11))

    bv, bt = S.box_surface((0.02, 0.015, 0.01))
    body = dict(verts=bv, tris=bt, rho=800.0, q0=S.IDENTITY_Q.copy(), qdot0=np.zeros(12), kinematic=False)
    env = dict(soft=[], affine=[body], mu=0.0, gravity=np.zeros(2, dtype=np.uint8),
               targets=np.tile(S.IDENTITY_Q, (2, 1, 1)))
    e = O.OracleEnv(p, env)
    e.step(1)
    x, _ = e.state()
    q = x.copy()
    q[3:12] *= 0.5
    cases.append((e, q, 1e-8))

    for e, q, step in cases:
        raw = _sym_fd_hessian(e, q, step)
        assert np.linalg.eigvalsh(raw).min() < -1e-2 * np.abs(raw).max()
        H = e.hessian(q)
        assert np.allclose(H, H.T, atol=1e-12 * np.abs(H).max())
        assert np.linalg.eigvalsh(H).min() > -1e-9 * np.abs(H).max()


def _bob_com(x):
    return x[12:15]


def test_joint_hangs_a_body_by_its_static_sag():
    """A cube (side a, volume V) hanging by a point joint of stiffness k, anchored l above its
    centre, settles with its joint stretched by m g / k straight down (the joint force balances
    the weight) and neither turns nor sways. The joint pulls on the column a3 of A with the
    generalized force l m g, which the orthogonality term h^2 kappa_A V |A A^T - I|^2 balances at
    A = diag(1, 1, 1 + eps), 8 kappa_A V eps = l m g: the centre hangs l eps lower still."""
    k, a, l = 1e3, 0.02, 0.1
    p = S.scene_params(0.01, newton_tol=1e-6)
    env = S.pendulum_env(k_joint=k, n_steps=200, arm=l, half=a / 2)
    e = O.OracleEnv(p, env)
    m, V = 1000.0 * a ** 3, a ** 3
    assert e.step(200) == "DONE"
    x, _ = e.state()
    sag = m * G / k
    eps = l * m * G / (8.0 * p["kappa_affine"] * V)
    assert abs(_bob_com(x)[2] - (-l - sag - l * eps)) <= 3e-4 * sag
    assert np.abs(_bob_com(x)[:2]).max() < 1e-12
    A = x[15:24].reshape(3, 3).T
    assert abs(A[2, 2] - (1.0 + eps)) <= 1e-2 * eps
    assert np.abs(A - np.diag([1.0, 1.0, A[2, 2]])).max() < 1e-12


def test_pendulum_swings_with_the_compound_pendulum_period():
    """Released at 0.05 rad, the jointed cube swings about the joint with the small-amplitude
    period of a compound pendulum, 2 pi sqrt(I_p / (m g l)), I_p = m a^2 / 6 + m l^2 (cube of
    side a, centre l below the joint), within 0.5% (implicit Euler at h omega = 0.02 shifts the
    period by far less; the joint's stretch m g / k lengthens l by 1e-5 relative)."""
    dt, n = 0.002, 700
    p = S.scene_params(dt)
    env = S.pendulum_env(k_joint=1e5, n_steps=n, theta0=0.05)
    e = O.OracleEnv(p, env)
    ys = []
    for _ in range(n):
        e.step(1)
        ys.append(_bob_com(e.state()[0])[1])
    ys = np.array(ys)
    t = (np.arange(n) + 1) * dt
    # zero crossings of the sideways position, by linear interpolation
    z = [t[i] - ys[i] * (t[i + 1] - t[i]) / (ys[i + 1] - ys[i]) for i in range(n - 1) if ys[i] * ys[i + 1] < 0]
    assert len(z) >= 3
    period = 2.0 * (z[2] - z[0]) / 2.0
    a, l = 0.02, 0.1
    T = 2 * math.pi * math.sqrt((a * a / 6 + l * l) / (G * l))
    assert abs(period / T - 1.0) < 5e-3, (period, T)
    # the swing stays in the y-z plane and the cube keeps its shape
    xs, _ = e.state()
    assert abs(_bob_com(xs)[0]) < 1e-12
    A = xs[15:24].reshape(3, 3).T
    assert np.abs(A @ A.T - np.eye(3)).max() < 1e-5  # affine stiffness keeps A near a rotation


def test_env_gradient_and_hessian_fd_joint_term():
    """The joint potential's gradient and Hessian against central differences at a state where
    the joint is stretched and turned (no contacts; the joint term is quadratic, so its
    Hessian is exact and unprojected)."""
    p = S.scene_params(0.01)
    env = S.pendulum_env(k_joint=3e3, n_steps=10, theta0=0.3)
    e = O.OracleEnv(p, env)
    e.step(2)
    x, _ = e.state()
    q = x.copy()
    q[12:15] += np.array([2e-3, -1e-3, 3e-3])
    _fd_check(e, q, list(range(24)))
    H = e.hessian(q)
    Hf = _fd_hessian(e, q, range(12, 24))
    assert np.abs(H[:, 12:24] - Hf).max() <= 1e-6 * np.abs(H).max()


def test_elastic_energy_is_the_volume_weighted_strain_energy():
    """A free soft block (side a) under a uniform deformation F has elastic energy h^2 a^3 Psi(F):
    every tet has the same F, and their rest volumes add up to the block's. With the block at rest
    and gravity off the predicted positions are the rest ones for any dt, so two time steps h1, h2
    change only the elastic term: (E(h1) - E(h2)) / (h1^2 - h2^2) = a^3 Psi(F), with Psi the
    (separately pinned) Neo-Hookean density of the element routine."""
    a, E, nu = 0.02, 2e5, 0.35
    verts, tets, _ = S.kuhn_grid(3, 3, 3, (0.0, 0.0, 0.0), (a, a, a))
    soft = dict(verts=verts, tets=tets, tris=S.boundary_tris(verts, tets), E=E, nu=nu, rho=1000.0,
                kin=np.zeros(len(verts), dtype=np.uint8))
    env = dict(soft=[soft], affine=[], mu=0.0, gravity=np.zeros(2, dtype=np.uint8),
               targets=np.tile(S.IDENTITY_Q, (2, 1, 1)))
    F = np.array([[1.05, 0.02, 0.0], [-0.01, 0.97, 0.03], [0.0, 0.01, 1.02]])
    q = (verts @ F.T).ravel()
    Es = []
    for h in (0.01, 0.02):
        e = O.OracleEnv(S.scene_params(h), env)
        Es.append(e.eval(q, grad=False))
    mu, lam = E / (2 * (1 + nu)), E * nu / ((1 + nu) * (1 - 2 * nu))
    psi, _, _ = O.neo_hookean(F, mu, lam)
    assert abs((Es[0] - Es[1]) / (0.01 ** 2 - 0.02 ** 2) / (a ** 3 * psi) - 1.0) < 1e-10


def test_edge_edge_contact_force_carries_the_rest_length_mollifier():
    """Two thin rigid bars crossing at angle theta, 0.4 dhat apart: the edge-edge contacts' normal
    forces are kappa e(c) |b'(d)| with c = |e_a x e_b|^2 and the mollifier threshold 1e-3 |rest e_a|^2
    |rest e_b|^2 of IPC 2020 (e = 1 above it, 2 c/eps - (c/eps)^2 below). At 8 degrees the crossing
    long edges are unmollified (sin^2 = 0.019 > 1e-3); at 1 degree (sin^2 = 3e-4) they carry
    e = 2 r - r^2 with r = 0.30."""
    dhat, g = 1e-3, 4e-4
    p = S.scene_params(0.01)
    hv, ht = S.box_surface((0.05, 0.002, 0.002))
    for deg, mollified in ((8.0, False), (1.0, True)):
        th = math.radians(deg)
        R = np.array([[math.cos(th), -math.sin(th), 0.0], [math.sin(th), math.cos(th), 0.0], [0.0, 0.0, 1.0]])
        qa = S.IDENTITY_Q.copy()
        qb = S.IDENTITY_Q.copy()
        qb[:3] = [0.0, 0.0, 0.004 + g]
        qb[3:6], qb[6:9], qb[9:12] = R[:, 0], R[:, 1], R[:, 2]
        bars = [dict(verts=hv, tris=ht, rho=1000.0, q0=q, qdot0=np.zeros(12), kinematic=k)
                for q, k in ((qa, True), (qb, False))]  # pairs of two kinematic bodies are skipped
        env = dict(soft=[], affine=bars, mu=0.0, gravity=np.zeros(2, dtype=np.uint8),
                   targets=np.stack([np.stack([qa, qb])] * 2))
        e = O.OracleEnv(p, env)
        x, _ = e.state()
        pts = np.concatenate([hv, hv @ R.T + qb[:3]])
        tris = np.concatenate([ht, ht + len(hv)])
        ed = sorted({(min(a, b), max(a, b)) for t in tris for a, b in ((t[0], t[1]), (t[1], t[2]), (t[2], t[0]))})
        rest = np.concatenate([hv, hv])
        C, _ = e.contacts(x)
        f = e.contact_forces(x)
        rs = []
        E_ref = 0.0  # at rest with gravity off and mu = 0 the potential is the barrier alone
        for (kind, i, j, _), fk in zip(C, f):
            if kind != 1:
                v = sorted({int(t) for t in tris.ravel()})[i]
                tri = tris[j]
                x12 = np.concatenate([pts[v], pts[tri[0]], pts[tri[1]], pts[tri[2]]])
                E_ref += p["dt"] ** 2 * p["kappa"] * O.barrier(math.sqrt(O.pair_dist2(0, x12)[0]), dhat)[0]
                continue
            (a0, a1), (b0, b1) = ed[i], ed[j]
            x12 = np.concatenate([pts[a0], pts[a1], pts[b0], pts[b1]])
            d = math.sqrt(O.pair_dist2(1, x12)[0])
            cr = np.cross(pts[a1] - pts[a0], pts[b1] - pts[b0])
            c = float(cr @ cr)
            eps = 1e-3 * float((rest[a1] - rest[a0]) @ (rest[a1] - rest[a0])) * float((rest[b1] - rest[b0]) @ (rest[b1] - rest[b0]))
            r = c / eps
            m = 1.0 if r >= 1.0 else 2.0 * r - r * r
            ref = p["kappa"] * m * abs(O.barrier(d, dhat)[1])
            assert abs(fk - ref) <= 1e-9 * ref, (deg, i, j, fk, ref)
            E_ref += p["dt"] ** 2 * p["kappa"] * m * O.barrier(d, dhat)[0]
            rs.append(r)
        assert len(rs) > 0
        E = e.eval(x, grad=False)
        assert abs(E - E_ref) <= 1e-9 * E_ref, (deg, E, E_ref)
        # at 8 degrees every crossing (long edges, top-face diagonals) is above the threshold; at 1
        # degree the long edges' crossing sits at r = sin^2(1 deg) / 1e-3 = 0.30
        assert any(r < 1.0 for r in rs) == mollified
        assert not mollified or any(abs(r - 0.30) < 0.01 for r in rs)


def _head_on_cube(gap, speed, n_steps=1):
    """A free rigid cube a gap above the fixed ground triangle, falling straight down at `speed`
    with gravity off (no friction): the predicted pose is x~ = x^t + h v, a pure translation."""
    env = S.resting_env("rigid", n_steps=n_steps, gap=gap)
    env["gravity"][:] = 0
    env["affine"][0]["qdot0"] = np.zeros(12)
    env["affine"][0]["qdot0"][2] = -speed
    return env


def _first_two_iterate_energies(p, env):
    e = O.OracleEnv(p, env)
    e.trace(True)
    e.step(1)
    tr = e.trace_energies()
    assert tr[0][:3].tolist() == [0, 0, 0] and tr[1][:3].tolist() == [0, 1, 0]
    return tr[0][3], tr[1][3]


def test_step_filter_stops_short_of_impact_by_the_accd_gap_fraction():
    """Step filter (ACCD, Li et al. 2021, gap fraction s = 0.1): for a cube translating head-on
    toward the ground, every closest pair (the four bottom corners over the ground triangle) has
    relative speed l_p = |p| after the mean shift, so ACCD's first advance (1 - s) d0 / l_p is
    already within s d0 of contact and the bound is alpha = (1 - s) d0 / (h V). With the gap
    large enough that the trial point is still farther than d^ from the ground, the step is
    accepted as it is, and the energy of the next iterate is the inertia term alone:
    E1 = (1 - alpha)^2 E0 (the Newton direction is exactly h v: the orthogonality term has zero
    gradient at A = I and its Hessian does not couple to the translation)."""
    h = 0.01
    p = S.scene_params(h)
    d0 = 20 * p["dhat"]
    V = 2 * d0 / h  # the free step would carry the cube a full gap past the ground
    E0, E1 = _first_two_iterate_energies(p, _head_on_cube(d0, V))
    alpha = (1 - 0.1) * d0 / (h * V)
    assert E0 > 0
    assert abs(E1 / E0 - (1 - alpha) ** 2) < 1e-9, (E1 / E0, (1 - alpha) ** 2)


def test_line_search_halves_a_trial_that_meets_the_barrier():
    """Backtracking by halving: from a gap of 3 d^ the step filter's bound 0.45 leaves the cube
    0.3 d^ above the ground, where the barrier energy (four point-triangle contacts at
    kappa = 3e6) exceeds the inertia decrease, so the trial is rejected; the halved step leaves
    it 1.65 d^ above, out of contact, and is accepted: E1 = (1 - 0.225)^2 E0."""
    h = 0.01
    p = S.scene_params(h)
    d0 = 3 * p["dhat"]
    V = 2 * d0 / h
    E0, E1 = _first_two_iterate_energies(p, _head_on_cube(d0, V))
    alpha = (1 - 0.1) * d0 / (h * V)
    gap_trial = d0 - alpha * h * V
    assert gap_trial < p["dhat"] < d0 - 0.5 * alpha * h * V
    barrier = 4 * h * h * p["kappa"] * O.barrier(gap_trial, p["dhat"])[0]
    assert (1 - alpha) ** 2 * E0 + barrier > E0  # the first trial must fail the decrease test
    assert abs(E1 / E0 - (1 - 0.5 * alpha) ** 2) < 1e-9, (E1 / E0, (1 - 0.5 * alpha) ** 2)


def test_incremental_potential_of_a_body_at_rest_above_the_ground_is_its_barrier_sum():
    """With gravity off and zero velocity, x~ = x^t, so at x^t the inertia term vanishes and an
    undeformed rigid cube (A = I, no orthogonality energy, no friction) a gap d above the ground
    has the incremental potential h^2 kappa sum_k b(d_k) over its four bottom corners, each a
    point-triangle contact at d (no mollifier). The energy-only evaluation (the line search's)
    and the one with derivatives (the Newton iterate's) must both give it."""
    h = 0.01
    p = S.scene_params(h)
    gap = 0.4 * p["dhat"]
    env = S.resting_env("rigid", n_steps=2, gap=gap)
    env["gravity"][:] = 0
    e = O.OracleEnv(p, env)
    x, _ = e.state()
    want = 4 * h * h * p["kappa"] * O.barrier(gap, p["dhat"])[0]
    assert want > 0
    E_only = e.eval(x, grad=False)
    E_full, _ = e.eval(x)
    assert abs(E_only / want - 1) < 1e-9, (E_only, want)
    assert abs(E_full / want - 1) < 1e-9, (E_full, want)
