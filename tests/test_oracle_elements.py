"""Pins of the CPU oracle's element-level functions against closed forms, brute force,
finite differences and independent library routines (no GPU)."""
import json
import math
import os

import numpy as np
import pytest
from scipy.optimize import minimize

from oracle import oracle as O
from paper_2503_05020_b300 import scenes as S

HERE = os.path.dirname(os.path.abspath(__file__))
RNG = np.random.default_rng(1234)


def rand_rotation(rng):
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def lame(E, nu):
    return E / (2 * (1 + nu)), E * nu / ((1 + nu) * (1 - 2 * nu))


# ------------------------------------------------------------------ paper parameters
def test_paper_parameters_are_defaults():
    """Sec. III-D fixes dt, kappa, dhat, eps_v and the Newton cap; the defaults must match."""
    g = json.load(open(os.path.join(HERE, "golden", "paper_parameters.json")))
    p = S.scene_params(g["dt"])
    assert p["kappa"] == g["kappa"] and p["dhat"] == g["dhat"] and p["eps_v"] == g["eps_v"]
    assert p["max_newton"] == g["max_newton"]
    assert abs(np.linalg.norm(p["gravity"]) - g["gravity_magnitude"]) < 1e-12


# ------------------------------------------------------------------ Neo-Hookean
def test_neo_hookean_zero_for_rotations():
    mu, lam = lame(1e5, 0.4)
    for _ in range(5):
        R = rand_rotation(RNG)
        psi, P, H = O.neo_hookean(R, mu, lam)
        assert abs(psi) < 1e-9 * mu
        assert np.abs(P).max() < 1e-9 * mu


def test_neo_hookean_small_strain_is_linear_elasticity():
    """Psi(I + eps) -> mu |eps|^2 + lam/2 tr(eps)^2 for a small symmetric strain."""
    mu, lam = lame(2e5, 0.45)
    e = RNG.normal(size=(3, 3))
    e = 0.5 * (e + e.T)
    for s in (1e-3, 1e-4):
        eps = s * e
        psi, _, _ = O.neo_hookean(np.eye(3) + eps, mu, lam)
        lin = mu * np.sum(eps * eps) + 0.5 * lam * np.trace(eps) ** 2
        assert abs(psi - lin) / lin < 20 * s


def test_neo_hookean_derivatives_match_finite_differences():
    mu, lam = lame(1e5, 0.3)
    F = np.eye(3) + 0.2 * RNG.normal(size=(3, 3))
    assert np.linalg.det(F) > 0
    psi, P, H = O.neo_hookean(F, mu, lam)
    h = 1e-6
    Pfd = np.zeros(9)
    Hfd = np.zeros((9, 9))
    for i in range(9):
        d = np.zeros(9)
        d[i] = h
        pp, Pp, _ = O.neo_hookean(F.ravel() + d, mu, lam)
        pm, Pm, _ = O.neo_hookean(F.ravel() - d, mu, lam)
        Pfd[i] = (pp - pm) / (2 * h)
        Hfd[i] = (Pp - Pm) / (2 * h)
    assert np.allclose(P, Pfd, rtol=1e-6, atol=1e-6 * mu)
    assert np.allclose(H, Hfd, rtol=1e-5, atol=1e-5 * mu)
    assert np.allclose(H, H.T, atol=1e-9 * mu)


# ------------------------------------------------------------------ PSD projection
def test_psd_projection_matches_numpy_eigh():
    for n in (3, 9, 12):
        A = RNG.normal(size=(n, n))
        A = A + A.T
        P = O.project_psd(A)
        w, V = np.linalg.eigh(A)
        ref = (V * np.maximum(w, 0)) @ V.T
        assert np.allclose(P, ref, atol=1e-12 * np.abs(A).max())
        assert np.linalg.eigvalsh(P).min() > -1e-12 * np.abs(A).max()


def test_psd_projection_keeps_psd_matrix():
    B = RNG.normal(size=(12, 12))
    A = B @ B.T
    assert np.allclose(O.project_psd(A), A, atol=1e-12 * np.abs(A).max())


def test_jacobi_eigenvalues_match_numpy():
    A = RNG.normal(size=(9, 9))
    A = A + A.T
    w, V = O.eigh(A)
    assert np.allclose(np.sort(w), np.linalg.eigvalsh(A), atol=1e-12 * np.abs(A).max())
    assert np.allclose(V.T @ V, np.eye(9), atol=1e-12)


# ------------------------------------------------------------------ barrier
def test_barrier_closed_form_and_smoothness_at_dhat():
    dhat = 1e-3
    b, b1, b2 = O.barrier(dhat, dhat)
    assert b == 0 and b1 == 0 and b2 == 0  # C2 at dhat
    assert np.all(O.barrier(2 * dhat, dhat) == 0)
    b, _, _ = O.barrier(dhat / 2, dhat)
    assert math.isclose(b, (dhat / 2) ** 2 * math.log(2), rel_tol=1e-14)
    for d in (1e-6, 1e-5, 3e-4, 9e-4):
        b, b1, b2 = O.barrier(d, dhat)
        h = d * 1e-5
        bp, bm = O.barrier(d + h, dhat), O.barrier(d - h, dhat)
        assert b > 0 and b1 < 0 and b2 > 0
        assert math.isclose(b1, (bp[0] - bm[0]) / (2 * h), rel_tol=1e-6)
        assert math.isclose(b2, (bp[1] - bm[1]) / (2 * h), rel_tol=1e-6)
    assert O.barrier(1e-12, dhat)[0] > O.barrier(1e-9, dhat)[0] > O.barrier(1e-6, dhat)[0]


# ------------------------------------------------------------------ distances
def brute_pt(x):
    p, a, b, c = x[0:3], x[3:6], x[6:9], x[9:12]
    u = np.linspace(0, 1, 201)
    U, V = np.meshgrid(u, u)
    m = U + V <= 1
    Q = a + U[m, None] * (b - a) + V[m, None] * (c - a)
    k = np.argmin(((Q - p) ** 2).sum(1))
    x0 = np.array([U[m][k], V[m][k]])
    f = lambda z: np.sum((a + z[0] * (b - a) + z[1] * (c - a) - p) ** 2)
    r = minimize(f, x0, method="SLSQP", bounds=[(0, 1), (0, 1)],
                 constraints=[{"type": "ineq", "fun": lambda z: 1 - z[0] - z[1]}], options={"ftol": 1e-30, "maxiter": 500})
    return min(r.fun, f(x0))


def brute_ee(x):
    a0, a1, b0, b1 = x[0:3], x[3:6], x[6:9], x[9:12]
    u = np.linspace(0, 1, 201)
    U, V = np.meshgrid(u, u)
    A = a0 + U.ravel()[:, None] * (a1 - a0)
    B = b0 + V.ravel()[:, None] * (b1 - b0)
    k = np.argmin(((A - B) ** 2).sum(1))
    f = lambda z: np.sum((a0 + z[0] * (a1 - a0) - b0 - z[1] * (b1 - b0)) ** 2)
    x0 = np.array([U.ravel()[k], V.ravel()[k]])
    r = minimize(f, x0, method="L-BFGS-B", bounds=[(0, 1), (0, 1)], options={"ftol": 1e-30, "gtol": 1e-30})
    return min(r.fun, f(x0))


@pytest.mark.parametrize("kind", [0, 1])
def test_distance_matches_brute_force(kind):
    seen = set()
    for _ in range(300):
        x = RNG.normal(size=12) * 0.01
        d2, t, _, _ = O.pair_dist2(kind, x)
        ref = brute_pt(x) if kind == 0 else brute_ee(x)
        seen.add(t)
        assert abs(d2 - ref) <= 1e-9 * max(ref, 1e-12), (kind, t, d2, ref)
    assert len(seen) >= (6 if kind == 0 else 7)  # most region types were exercised


@pytest.mark.parametrize("kind", [0, 1])
def test_distance_derivatives_match_finite_differences(kind):
    for _ in range(40):
        x = RNG.normal(size=12) * 0.01
        d2, t, g, H = O.pair_dist2(kind, x)
        h = 1e-8
        for i in range(12):
            e = np.zeros(12)
            e[i] = h
            fp = O.pair_dist2_typed(kind, t, x + e)
            fm = O.pair_dist2_typed(kind, t, x - e)
            assert abs((fp - fm) / (2 * h) - g[i]) <= 1e-6 * max(np.abs(g).max(), 1e-12)
        # Hessian by differences of the AD gradient at fixed type
        for i in range(12):
            e = np.zeros(12)
            e[i] = 1e-7
            _, tp, gp, _ = O.pair_dist2(kind, x + e)
            _, tm, gm, _ = O.pair_dist2(kind, x - e)
            if tp != t or tm != t:
                continue
            assert np.allclose((gp - gm) / 2e-7, H[i], atol=1e-5 * max(np.abs(H).max(), 1e-12))


def test_distances_in_degenerate_configurations():
    """Closed forms where the closest-feature selection is fragile: exactly parallel edges
    (overlapping, offset along their line, and collinear with a gap), crossing edges, and a point
    exactly on a triangle's face, edge and corner."""
    E = lambda a0, a1, b0, b1: O.pair_dist2(1, np.concatenate([a0, a1, b0, b1]))[0]
    P = lambda p, a, b, c: O.pair_dist2(0, np.concatenate([p, a, b, c]))[0]
    z = np.zeros(3)
    ex, ey = np.array([1.0, 0, 0]), np.array([0, 1.0, 0])
    h = 0.003
    # parallel, overlapping in projection: the perpendicular offset
    assert math.isclose(E(z, ex, h * ey + 0.2 * ex, h * ey + 1.5 * ex), h * h, rel_tol=1e-12)
    # parallel, no overlap: the distance between the nearest endpoints
    assert math.isclose(E(z, ex, h * ey + 1.4 * ex, h * ey + 2.0 * ex), 0.4 ** 2 + h * h, rel_tol=1e-12)
    # collinear with a gap of 0.25
    assert math.isclose(E(z, ex, 1.25 * ex, 2.0 * ex), 0.25 ** 2, rel_tol=1e-12)
    # antiparallel copy shifted by h: same as parallel
    assert math.isclose(E(z, ex, h * ey + ex, h * ey), h * h, rel_tol=1e-12)
    # crossing at right angles, h apart
    ez = np.array([0, 0, 1.0])
    assert math.isclose(E(z, ex, 0.5 * ex - 0.5 * ey + h * ez, 0.5 * ex + 0.5 * ey + h * ez), h * h, rel_tol=1e-12)
    a, b, c = z, ex, ey
    assert P(np.array([0.2, 0.3, 0.0]), a, b, c) == 0.0  # on the face
    assert P(np.array([0.5, 0.0, 0.0]), a, b, c) == 0.0  # on an edge
    assert P(b.copy(), a, b, c) == 0.0  # on a corner
    assert math.isclose(P(np.array([0.7, 0.7, 0.0]), a, b, c), 2 * 0.2 ** 2, rel_tol=1e-12)  # beyond the hypotenuse


def test_pt_distance_continuous_across_regions():
    """On the boundary between two regions both typed formulas give the same distance."""
    a, b, c = np.array([0.0, 0, 0]), np.array([1.0, 0, 0]), np.array([0.0, 1, 0])
    # point above the edge ab, exactly on the plane through ab perpendicular to the face
    p = np.array([0.3, 0.0, 0.4])
    x = np.concatenate([p, a, b, c])
    d_face = O.pair_dist2_typed(0, 6, x)
    d_edge = O.pair_dist2_typed(0, 3, x)
    assert math.isclose(d_face, d_edge, rel_tol=1e-14)
    # beyond vertex b, on the boundary of the vertex and edge regions
    p = np.array([1.0, -0.2, 0.1])
    x = np.concatenate([p, a, b, c])
    assert math.isclose(O.pair_dist2_typed(0, 1, x), O.pair_dist2_typed(0, 3, x), rel_tol=1e-14)


@pytest.mark.parametrize("kind", [0, 1])
def test_closest_point_coefficients(kind):
    for _ in range(100):
        x = RNG.normal(size=12) * 0.01
        d2, _, _, _ = O.pair_dist2(kind, x)
        c, n = O.pair_closest(kind, x)
        diff = sum(c[i] * x[3 * i:3 * i + 3] for i in range(4))
        assert math.isclose(np.linalg.norm(diff), math.sqrt(d2), rel_tol=1e-8)
        assert np.allclose(diff / np.linalg.norm(diff), n, atol=1e-8)
        assert abs(c.sum()) < 1e-12  # a rigid translation has no relative displacement


# ------------------------------------------------------------------ EE mollifier, contact energy
def test_mollifier_continuity_and_limits():
    a0, a1 = np.array([0.0, 0, 0]), np.array([1.0, 0, 0])
    eps = 0.01
    perpendicular = np.concatenate([a0, a1, [0.5, -0.5, 0.1], [0.5, 0.5, 0.1]])
    parallel = np.concatenate([a0, a1, [0.0, 0.0, 0.1], [1.0, 0.0, 0.1]])
    assert O.mollifier(perpendicular, eps) == 1.0
    assert O.mollifier(parallel, eps) == 0.0
    # continuity across c = eps: |a x b|^2 = sin^2(th) for unit edges
    th = math.asin(math.sqrt(eps))
    for d in (-1e-9, 1e-9):
        b1 = np.array([0.5 + math.cos(th + d), math.sin(th + d), 0.1])
        x = np.concatenate([a0, a1, [0.5, 0, 0.1], b1])
        assert abs(O.mollifier(x, eps) - 1.0) < 1e-6
    # C1 at c = eps (the barrier's gradient stays continuous as edges turn through the threshold):
    # just below it, 1 - e(c) vanishes to second order in (eps - c) / eps
    for rel in (1e-2, 1e-3):
        th = math.asin(math.sqrt(eps * (1.0 - rel)))
        x = np.concatenate([a0, a1, [0.5, 0, 0.1], [0.5 + math.cos(th), math.sin(th), 0.1]])
        assert abs((1.0 - O.mollifier(x, eps)) / rel ** 2 - 1.0) < 1e-6


@pytest.mark.parametrize("kind", [0, 1])
def test_contact_barrier_derivatives_match_finite_differences(kind):
    dhat, kappa = 1e-3, 3e6
    n_checked = 0
    while n_checked < 10:
        x = RNG.normal(size=12) * 1e-3
        d2, t, _, _ = O.pair_dist2(kind, x)
        if not (1e-8 < d2 < (0.9 * dhat) ** 2):
            continue
        eps = 1e-3 * np.sum((x[3:6] - x[0:3]) ** 2) * np.sum((x[9:12] - x[6:9]) ** 2) if kind else 0.0
        E, g, H = O.contact_barrier(kind, x, dhat, kappa, eps)
        h = 1e-10
        for i in range(12):
            e = np.zeros(12)
            e[i] = h
            _, t2, _, _ = O.pair_dist2(kind, x + e)
            _, t3, _, _ = O.pair_dist2(kind, x - e)
            if t2 != t or t3 != t:
                continue
            Ep, gp, _ = O.contact_barrier(kind, x + e, dhat, kappa, eps)
            Em, gm, _ = O.contact_barrier(kind, x - e, dhat, kappa, eps)
            assert abs((Ep - Em) / (2 * h) - g[i]) <= 1e-5 * np.abs(g).max()
            assert np.allclose((gp - gm) / (2 * h), H[i], atol=1e-4 * np.abs(H).max())
        n_checked += 1


# ------------------------------------------------------------------ friction smoothing
def test_friction_f0_is_c1_and_matches_limits():
    eh = 1e-5
    f_lo = O.friction_f(eh * (1 - 1e-12), eh)
    f_hi = O.friction_f(eh * (1 + 1e-12), eh)
    assert math.isclose(f_lo[0], f_hi[0], rel_tol=1e-9) and math.isclose(f_lo[1], f_hi[1], abs_tol=1e-9)
    f0 = O.friction_f(0.0, eh)
    assert math.isclose(f0[0], eh / 3, rel_tol=1e-15) and f0[1] == 0.0
    for y in (0.1 * eh, 0.5 * eh, 0.9 * eh):
        h = 1e-6 * eh
        fp, fm = O.friction_f(y + h, eh), O.friction_f(y - h, eh)
        f = O.friction_f(y, eh)
        assert math.isclose(f[1], (fp[0] - fm[0]) / (2 * h), rel_tol=1e-6)
        assert math.isclose(f[2], (fp[1] - fm[1]) / (2 * h), rel_tol=1e-6)
        assert 0 < f[1] <= 1


# ------------------------------------------------------------------ ACCD
def true_toi(kind, x, p, n=20001):
    ts = np.linspace(0, 1, n)
    ds = np.array([O.pair_dist2(kind, x + t * p)[0] for t in ts])
    hit = np.nonzero(ds <= 0)[0]
    if len(hit):
        return ts[hit[0]]
    # refine the minimum by bisection on the sign of d^2 - tiny
    k = np.argmin(ds)
    return 1.0 if ds[k] > 1e-24 else ts[k]


@pytest.mark.parametrize("kind", [0, 1])
def test_accd_is_conservative_against_bisection(kind):
    n_hit = 0
    for trial in range(120):
        x = RNG.normal(size=12) * 0.01
        d2 = O.pair_dist2(kind, x)[0]
        if d2 < 1e-8:
            continue
        # aim the first primitive at the second so that many trials collide
        p = RNG.normal(size=12) * 0.01
        target = x[6:9] if kind == 0 else 0.5 * (x[6:9] + x[9:12])
        src = x[0:3] if kind == 0 else 0.5 * (x[0:3] + x[3:6])
        shift = 2.0 * (target - src) * RNG.uniform(0.5, 1.5)
        for i in range(2 if kind else 1):
            p[3 * i:3 * i + 3] += shift
        t, it = O.accd(kind, x, p)
        assert 0 < t <= 1
        d_at = O.pair_dist2(kind, x + t * p)[0]
        assert d_at > 0
        # no contact before t: sample the path densely
        for s in np.linspace(0, t, 200):
            assert O.pair_dist2(kind, x + s * p)[0] > 0
        if t < 1:
            n_hit += 1
            # and not grossly conservative: the gap left is about s*d at the reported time
            dist_t = math.sqrt(d_at)
            assert dist_t <= math.sqrt(d2)
    assert n_hit >= 10


def first_crossing_time(kind, x, p):
    """Exact first contact time in [0, 1] of four linearly moving points (Provot 1997): contact
    needs the four points coplanar, i.e. a root of the cubic det[x1 - x0, x2 - x0, x3 - x0](t),
    at which the point lies in the triangle (PT) or the two segments meet (EE). Plain numpy
    geometry; none of the oracle's distance code. Returns inf when the primitives never meet."""
    P = lambda t: (x + t * p).reshape(4, 3)

    def vol(t):
        q = P(t)
        return np.linalg.det(np.stack([q[1] - q[0], q[2] - q[0], q[3] - q[0]]))

    ts = np.array([0.0, 1 / 3, 2 / 3, 1.0])
    coef = np.polyfit(ts, [vol(t) for t in ts], 3)
    roots = sorted(r.real for r in np.roots(coef) if abs(r.imag) < 1e-9 and -1e-12 <= r.real <= 1 + 1e-12)
    for t in roots:
        q = P(t)
        if kind == 0:  # barycentric coordinates of the point in the triangle's plane
            A = np.stack([q[2] - q[1], q[3] - q[1]], axis=1)
            uv, *_ = np.linalg.lstsq(A, q[0] - q[1], rcond=None)
            if uv.min() >= -1e-9 and uv.sum() <= 1 + 1e-9:
                return t
        else:  # a0 + s (a1 - a0) = b0 + u (b1 - b0)
            A = np.stack([q[1] - q[0], -(q[3] - q[2])], axis=1)
            su, *_ = np.linalg.lstsq(A, q[2] - q[0], rcond=None)
            if su.min() >= -1e-9 and su.max() <= 1 + 1e-9:
                return t
    return math.inf


@pytest.mark.parametrize("kind", [0, 1])
def test_accd_stops_before_primitives_pass_through_each_other(kind):
    """Fast motions that carry one primitive straight through the other within the step (a
    path that dense distance sampling can step over): the ACCD time is at most the exact first
    crossing time, never past it, and the pair is still apart there."""
    rng = np.random.default_rng(99 + kind)
    n_cross = 0
    for _ in range(200):
        x = rng.normal(size=12) * 0.01
        if kind == 0:  # the point goes through a random interior point of the triangle
            w = rng.dirichlet([2.0, 2.0, 2.0])
            through = w[0] * x[3:6] + w[1] * x[6:9] + w[2] * x[9:12]
            src = x[0:3]
        else:  # the first edge's midpoint goes through a random point of the second edge
            u = rng.uniform(0.2, 0.8)
            through = (1 - u) * x[6:9] + u * x[9:12]
            src = 0.5 * (x[0:3] + x[3:6])
        p = rng.normal(size=12) * 0.002
        shift = (through - src) / rng.uniform(0.2, 0.6)  # crossing near t in [0.2, 0.6]
        for i in range(2 if kind else 1):
            p[3 * i:3 * i + 3] = shift + p[3 * i:3 * i + 3] * 0.1
        if O.pair_dist2(kind, x)[0] < 1e-10:
            continue
        tc = first_crossing_time(kind, x, p)
        t, _ = O.accd(kind, x, p)
        assert 0 < t <= 1
        assert O.pair_dist2(kind, x + t * p)[0] > 0
        if tc <= 1:
            n_cross += 1
            assert t < tc, (t, tc)
    assert n_cross >= 100


def test_accd_returns_one_without_contact():
    x = np.array([0, 0, 0.1, 0, 0, 0, 1, 0, 0, 0, 1, 0], dtype=float)
    p = np.zeros(12)
    p[0:3] = [0.1, 0.1, 0.0]  # slides parallel to the triangle, never touches
    t, _ = O.accd(0, x, p)
    assert t == 1.0
    t, it = O.accd(0, x, np.zeros(12))
    assert t == 1.0 and it == 0


def test_accd_head_on_toi():
    """A point falling straight onto a triangle: contact at t* = 0.1/0.2 = 0.5; ACCD stops
    just before it, leaving at least the s = 0.1 fraction of the initial gap."""
    x = np.array([0.2, 0.2, 0.1, 0, 0, 0, 1, 0, 0, 0, 1, 0], dtype=float)
    p = np.zeros(12)
    p[2] = -0.2
    t, _ = O.accd(0, x, p)
    assert 0.45 - 1e-12 <= t < 0.5
    assert O.pair_dist2(0, x + t * p)[0] ** 0.5 >= 0.1 * 0.1 * 0.99


# ------------------------------------------------------------------ mass properties
def test_box_mass_properties_closed_form():
    hx, hy, hz = 0.03, 0.02, 0.01
    v, t = S.box_surface((hx, hy, hz))
    c = np.array([0.1, -0.2, 0.05])
    rho = 700.0
    M, vol = O.mass_properties(v + c, t, rho)
    V = 8 * hx * hy * hz
    m = rho * V
    assert math.isclose(vol, V, rel_tol=1e-12)
    assert math.isclose(M[0, 0], m, rel_tol=1e-12)
    assert np.allclose(M[0, 1:], m * c, rtol=1e-12)
    second = m * (np.diag([hx * hx, hy * hy, hz * hz]) / 3.0) + m * np.outer(c, c)
    assert np.allclose(M[1:, 1:], second, rtol=1e-11, atol=1e-16)
    assert np.allclose(M, M.T)


def test_rotated_box_mass_properties_closed_form():
    """A box turned by a random rotation R and moved to c: second moment
    m (R diag(h^2/3) R^T + c c^T), whose off-diagonal entries are all nonzero, so a product of
    inertia with a wrong sign or a swapped index fails here though not on the axis-aligned box."""
    rng = np.random.default_rng(42)
    h = np.array([0.04, 0.025, 0.01])
    v, t = S.box_surface(tuple(h))
    R = rand_rotation(rng)
    c = np.array([-0.03, 0.07, 0.02])
    rho = 1234.0
    M, vol = O.mass_properties(v @ R.T + c, t, rho)
    m = rho * 8 * h.prod()
    assert math.isclose(vol, 8 * h.prod(), rel_tol=1e-12)
    assert math.isclose(M[0, 0], m, rel_tol=1e-12)
    assert np.allclose(M[0, 1:], m * c, rtol=1e-12)
    assert np.allclose(M[1:, 0], m * c, rtol=1e-12)
    second = m * (R @ np.diag(h * h / 3.0) @ R.T + np.outer(c, c))
    assert np.abs(second - second.diagonal().mean() * np.eye(3)).min() > 0
    assert np.allclose(M[1:, 1:], second, rtol=1e-11, atol=1e-14 * m)


def test_tetrahedron_mass_properties_closed_form():
    """One tetrahedron as a closed 4-triangle surface: volume |det|/6, first moment V s/4 and the
    textbook second moment V/20 (sum_a x_a x_a^T + s s^T), s the sum of the corners."""
    rng = np.random.default_rng(7)
    for _ in range(5):
        x = rng.uniform(-0.05, 0.05, size=(4, 3))
        if np.linalg.det(np.stack([x[1] - x[0], x[2] - x[0], x[3] - x[0]])) < 0:
            x[[1, 2]] = x[[2, 1]]
        tris = np.array([[0, 2, 1], [0, 1, 3], [0, 3, 2], [1, 2, 3]], dtype=np.int32)
        rho = 900.0
        M, vol = O.mass_properties(x, tris, rho)
        V = np.linalg.det(np.stack([x[1] - x[0], x[2] - x[0], x[3] - x[0]])) / 6.0
        s = x.sum(axis=0)
        assert math.isclose(vol, V, rel_tol=1e-11)
        assert math.isclose(M[0, 0], rho * V, rel_tol=1e-11)
        assert np.allclose(M[0, 1:], rho * V * s / 4.0, rtol=1e-10, atol=1e-16)
        second = rho * V / 20.0 * (x.T @ x + np.outer(s, s))
        assert np.allclose(M[1:, 1:], second, rtol=1e-10, atol=1e-18)


def test_hull_mass_positive_definite():
    rng = S.SplitMix64(7)
    v, t = S.hull_object(rng, 200)
    M, vol = O.mass_properties(v, t, 1000.0)
    assert vol > 0 and np.linalg.eigvalsh(M).min() > 0
    assert len(t) == 1584


def exact_segment_d2(x):
    """Exact squared distance between segments a0a1 and b0b1 of the given doubles, in rational
    arithmetic: the minimum of the convex quadratic |a0 + s d1 - b0 - t d2|^2 over [0,1]^2 is at
    the interior stationary point when that lies inside, else on one of the four sides, where it
    is a clamped one-dimensional minimum."""
    from fractions import Fraction as Fr

    P = [[Fr(float(v)) for v in x[3 * i:3 * i + 3]] for i in range(4)]
    d1 = [P[1][k] - P[0][k] for k in range(3)]
    d2 = [P[3][k] - P[2][k] for k in range(3)]
    r = [P[0][k] - P[2][k] for k in range(3)]
    dot = lambda u, v: sum(ui * vi for ui, vi in zip(u, v))
    a, b, e, c, f = dot(d1, d1), dot(d1, d2), dot(d2, d2), dot(d1, r), dot(d2, r)
    q = lambda s, t: dot(*[[r[k] + s * d1[k] - t * d2[k] for k in range(3)]] * 2)
    clamp = lambda v: min(max(v, Fr(0)), Fr(1))
    cands = []
    den = a * e - b * b
    if den > 0:
        s, t = (b * f - c * e) / den, (a * f - b * c) / den
        if 0 <= s <= 1 and 0 <= t <= 1:
            cands.append(q(s, t))
    for s0 in (Fr(0), Fr(1)):
        cands.append(q(s0, clamp((f + s0 * b) / e)))
    for t0 in (Fr(0), Fr(1)):
        cands.append(q(clamp((t0 * b - c) / a), t0))
    return min(cands)


def crossing_edges(rng, L1, L2, h, sin2):
    """Two edges whose lines pass h apart at interior points of both, at angle theta with
    sin^2 theta = sin2, in a random frame."""
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    u, w, n = Q[:, 0], Q[:, 1], Q[:, 2]
    st = math.sqrt(sin2)
    d1 = L1 * u
    d2 = L2 * (math.sqrt(1.0 - sin2) * u + st * w)
    a0 = rng.normal(size=3) * 0.01
    s, t = rng.uniform(0.2, 0.8), rng.uniform(0.2, 0.8)
    b0 = a0 + s * d1 + h * n - t * d2
    return np.concatenate([a0, a0 + d1, b0, b0 + d2])


def test_near_parallel_edge_band_within_its_error_bound():
    """Reading 7's band: edges with sin^2 theta <= 1e-10 are treated as parallel, so their closest
    pair is taken on an endpoint (never the interior line-line pair). Against the exact minimum
    the oracle's distance can then only be too large, and by at most max(|e_a|, |e_b|) sin theta
    (the separation of the two lines changes by at most that much along an edge). Just outside
    the band (sin^2 theta from 1e-9 to 1e-7) the oracle must return the exact minimum, the
    interior line-line distance, to 1e-9 relative."""
    rng = np.random.default_rng(20250306)
    for sin2 in (1e-12, 3e-12, 1e-11, 3e-11):
        for _ in range(25):
            L1, L2 = rng.uniform(0.004, 0.02, size=2)
            h = rng.uniform(1e-5, 1e-3)
            x = crossing_edges(rng, L1, L2, h, sin2)
            d2, t, _, _ = O.pair_dist2(1, x)
            ex = float(exact_segment_d2(x))
            assert t != 8, "an edge pair inside the parallel band was typed line-line"
            assert d2 >= ex * (1 - 1e-12)
            assert math.sqrt(d2) - math.sqrt(ex) <= max(L1, L2) * math.sqrt(sin2) * (1 + 1e-6) + 1e-15
    for sin2 in (1e-9, 1e-8, 1e-7):
        for _ in range(25):
            L1, L2 = rng.uniform(0.004, 0.02, size=2)
            h = rng.uniform(1e-5, 1e-3)
            x = crossing_edges(rng, L1, L2, h, sin2)
            d2, t, _, _ = O.pair_dist2(1, x)
            ex = float(exact_segment_d2(x))
            assert t == 8
            assert abs(d2 - ex) <= 1e-9 * ex, (sin2, d2, ex)


def test_accd_common_translation_needs_no_advance():
    """Additive CCD subtracts the pair's mean displacement: two primitives carried by the same
    translation never approach each other, so the step is the whole [0, 1] with no advancement,
    however large the translation (Li, Kaufman & Jiang 2021)."""
    rng = np.random.default_rng(17)
    for kind in (0, 1):
        for _ in range(10):
            x = rng.normal(size=12) * 0.01
            d = rng.normal(size=3) * 0.05
            p = np.tile(d, 4)
            t, it = O.accd(kind, x, p)
            assert t == 1.0 and it == 0, (kind, t, it)
