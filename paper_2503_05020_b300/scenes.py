"""Seeded synthetic grasp scenes: the inputs shared by the CUDA path, the oracle and the tests.

This module only builds geometry, material parameters and kinematic schedules. It holds none
of the simulator's arithmetic (no energies, distances, CCD or solves), so both the CUDA path and
the CPU oracle can be fed from it without sharing any of the method.

The paper's assets (UMI/LEAP meshes, DexGraspNet objects) are not available, so every scene is
a procedural stand-in with the shapes, sizes and parameter ranges of the grasp-validation
workload of Sec. III-D (dt, kappa, dhat, eps_v) and the domain randomisation of Sec. III-B
(Young's modulus, friction coefficient and object scale drawn per environment).

Env dict layout (all arrays numpy, C-contiguous):

    soft:    list of {verts (n,3) f64, tets (m,4) i32, tris (f,3) i32 outward,
                      E, nu, rho (floats), kin (n,) u8: 1 = vertex driven by the schedule}
    affine:  list of {verts (n,3) f64 rest surface, tris (f,3) i32 outward, rho,
                      q0 (12,) f64, qdot0 (12,) f64, kinematic (bool)}
    mu:      friction coefficient of the environment
    gravity: (n_steps,) u8, 1 = gravity acts during that step
    targets: (n_steps, n_soft + n_affine, 12) f64 — for each step s the affine map
             q = (p, a1, a2, a3) that a kinematic body (or a soft body's kinematic vertices,
             mapped from their initial positions) must reach at the end of step s.
    joints:  (optional) list of {a, b: affine body indices, anchor_a, anchor_b: (3,) rest-frame
             anchors, k: stiffness N/m} — point joints 1/2 k |x_a - x_b|^2; two on one axis
             make a hinge.

Affine coordinates q = (p, a1, a2, a3) place a rest point xb at p + xb[0] a1 + xb[1] a2 + xb[2] a3
(the a_i are the columns of A).
"""
from __future__ import annotations

import math
import numpy as np

BASE_SEED = 20250306
MASK64 = (1 << 64) - 1

IDENTITY_Q = np.array([0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0, 1], dtype=np.float64)


class SplitMix64:
    """SplitMix64 (Steele, Lea & Flood 2014): a counter-based 64-bit generator."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))

    def uniform_array(self, n: int, lo: float, hi: float) -> np.ndarray:
        return np.array([self.uniform(lo, hi) for _ in range(n)], dtype=np.float64)

    def randint(self, lo: int, hi: int) -> int:
        """Integer in [lo, hi)."""
        return lo + int(self.uniform() * (hi - lo)) % max(hi - lo, 1)

    def normal(self) -> float:
        u1 = max(self.uniform(), 1e-300)
        u2 = self.uniform()
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)


# --------------------------------------------------------------------------- meshes

def _orient_tets(verts: np.ndarray, tets: np.ndarray) -> np.ndarray:
    """Swap two vertices of every tet whose rest orientation is negative."""
    a, b, c, d = (verts[tets[:, i]] for i in range(4))
    det = np.einsum("ij,ij->i", np.cross(b - a, c - a), d - a)
    tets = tets.copy()
    neg = det < 0
    tets[neg, 2], tets[neg, 3] = tets[neg, 3].copy(), tets[neg, 2].copy()
    return tets


def kuhn_grid(nx: int, ny: int, nz: int, lo, hi, cell_mask: np.ndarray | None = None):
    """Box [lo, hi] split into nx*ny*nz cells, each cut into 6 Kuhn tets along its main diagonal.

    cell_mask[i, j, k] == False removes that cell. Unused vertices are dropped.
    Returns (verts (n,3) f64, tets (m,4) i32, grid_index (n,3) i32 of each kept vertex).
    """
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    gi, gj, gk = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    grid = np.stack([gi.ravel(), gj.ravel(), gk.ravel()], axis=1)
    verts = lo + (hi - lo) * grid / np.array([nx, ny, nz], dtype=np.float64)

    # cells in (i, j, k) order, each cut into 6 tets: one per order in which the path from its
    # lowest to its highest corner steps along the three axes
    ci, cj, ck = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    cells = np.stack([ci.ravel(), cj.ravel(), ck.ravel()], axis=1)
    if cell_mask is not None:
        cells = cells[np.asarray(cell_mask, dtype=bool).ravel()]
    strides = np.array([(ny + 1) * (nz + 1), nz + 1, 1], dtype=np.int64)
    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    corner = np.zeros((6, 4), dtype=np.int64)  # vertex-id offset of each path corner
    for a, p in enumerate(perms):
        c = np.zeros(3, dtype=np.int64)
        for q, ax in enumerate(p):
            c[ax] += 1
            corner[a, q + 1] = c @ strides
    tets = ((cells.astype(np.int64) @ strides)[:, None, None] + corner[None]).reshape(-1, 4)
    used = np.unique(tets)
    remap = -np.ones(len(verts), dtype=np.int64)
    remap[used] = np.arange(len(used))
    verts = verts[used]
    grid = grid[used]
    tets = remap[tets]
    tets = _orient_tets(verts, tets)
    return verts, tets.astype(np.int32), grid.astype(np.int32)


def boundary_tris(verts: np.ndarray, tets: np.ndarray) -> np.ndarray:
    """Faces used by exactly one tet, oriented so that the normal points out of that tet, sorted
    by their vertex triples."""
    tets = np.asarray(tets, dtype=np.int64)
    if len(tets) == 0:
        return np.zeros((0, 3), dtype=np.int32)
    # face k of a tet leaves out its vertex k (kept vertices in tet order)
    keep = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]])
    faces = tets[:, keep].reshape(-1, 3)
    opp = tets.reshape(-1)
    s = np.sort(faces, axis=1)
    nv = np.int64(max(len(verts), 1))
    _, first, counts = np.unique((s[:, 0] * nv + s[:, 1]) * nv + s[:, 2], return_index=True, return_counts=True)
    sel = first[counts == 1]
    f, d = faces[sel], opp[sel]
    a, b, c = verts[f[:, 0]], verts[f[:, 1]], verts[f[:, 2]]
    n = np.cross(b - a, c - a)
    inward = np.einsum("ij,ij->i", n, verts[d] - a) > 0
    f[inward, 1], f[inward, 2] = f[inward, 2].copy(), f[inward, 1].copy()
    f = f[np.lexsort((f[:, 2], f[:, 1], f[:, 0]))]
    return f.astype(np.int32)


def box_surface(half_extents) -> tuple[np.ndarray, np.ndarray]:
    """Closed, outward-oriented 8-vertex 12-triangle box centred at the origin."""
    hx, hy, hz = half_extents
    v = np.array([[sx * hx, sy * hy, sz * hz] for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)])
    quads = [(0, 1, 3, 2), (4, 6, 7, 5), (0, 4, 5, 1), (2, 3, 7, 6), (0, 2, 6, 4), (1, 5, 7, 3)]
    tris = []
    for a, b, c, d in quads:
        tris += [(a, b, c), (a, c, d)]
    tris = np.asarray(tris, dtype=np.int64)
    # orient outward
    cen = v.mean(axis=0)
    for t in tris:
        n = np.cross(v[t[1]] - v[t[0]], v[t[2]] - v[t[0]])
        if np.dot(n, v[t[0]] - cen) < 0:
            t[1], t[2] = t[2], t[1]
    return v.astype(np.float64), tris.astype(np.int32)


def convex_hull_surface(points: np.ndarray) -> np.ndarray:
    """Outward triangles of the convex hull (qhull via scipy, used only to build inputs)."""
    from scipy.spatial import ConvexHull

    hull = ConvexHull(points)
    tris = hull.simplices.astype(np.int64).copy()
    cen = points[hull.vertices].mean(axis=0)
    for t in tris:
        n = np.cross(points[t[1]] - points[t[0]], points[t[2]] - points[t[0]])
        if np.dot(n, points[t[0]] - cen) < 0:
            t[1], t[2] = t[2], t[1]
    used = np.unique(tris)
    remap = -np.ones(len(points), dtype=np.int64)
    remap[used] = np.arange(len(used))
    return points[used].copy(), remap[tris].astype(np.int32)


def subdivide_midpoint(verts: np.ndarray, tris: np.ndarray):
    """One 1->4 midpoint subdivision (the surface geometry does not change)."""
    verts = [tuple(v) for v in verts]
    mid = {}
    out = []

    def m(a, b):
        key = (min(a, b), max(a, b))
        if key not in mid:
            mid[key] = len(verts)
            va, vb = verts[a], verts[b]
            verts.append(tuple(0.5 * (x + y) for x, y in zip(va, vb)))
        return mid[key]

    for a, b, c in tris:
        ab, bc, ca = m(a, b), m(b, c), m(c, a)
        out += [(a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca)]
    return np.asarray(verts, dtype=np.float64), np.asarray(out, dtype=np.int32)


def star_ball(rng: SplitMix64, n: int, r0: float, n_harm: int = 3, amp: float = 0.15):
    """Star-shaped soft object: a Kuhn-gridded ball, radially warped by seeded low harmonics."""
    lo = np.array([-1.0, -1.0, -1.0])
    hi = np.array([1.0, 1.0, 1.0])
    c = (np.arange(n) + 0.5) / n * 2.0 - 1.0
    ci, cj, ck = np.meshgrid(c, c, c, indexing="ij")
    mask = (ci ** 2 + cj ** 2 + ck ** 2) <= 1.0
    verts, tets, _ = kuhn_grid(n, n, n, lo, hi, mask)
    coeffs = [(rng.uniform(-amp, amp), rng.normal(), rng.normal(), rng.normal()) for _ in range(n_harm)]
    r = np.linalg.norm(verts, axis=1)
    dirs = verts / np.maximum(r[:, None], 1e-12)
    scale = np.ones(len(verts))
    for a, kx, ky, kz in coeffs:
        k = np.array([kx, ky, kz])
        k = k / max(np.linalg.norm(k), 1e-12)
        scale += a * (dirs @ k) ** 2
    verts = verts * (r0 * scale)[:, None]
    return verts, tets


# ----------------------------------------------------------------------- parameters

def scene_params(dt: float, dhat: float = 1e-3, kappa: float = 3e6, eps_v: float = 1e-3,
                 newton_tol: float | None = None, pcg_rel_tol: float = 1e-4,
                 max_newton: int = 100, max_ls: int = 40, max_pcg: int = 1000,
                 kappa_affine: float = 1e8, gravity=(0.0, 0.0, -9.8)) -> dict:
    """Solver parameters. Defaults follow Sec. III-D: kappa = 3e6 kg/s^2, dhat = 1e-3 m,
    eps_v = 1e-3 m/s, at most 100 Newton iterations; the Newton tolerance defaults to
    1e-2 * dt in m/s on the infinity norm of the Newton step divided by dt."""
    return dict(dt=float(dt), dhat=float(dhat), kappa=float(kappa), eps_v=float(eps_v),
                newton_tol=float(1e-2 * dt if newton_tol is None else newton_tol),
                pcg_rel_tol=float(pcg_rel_tol), max_newton=int(max_newton), max_ls=int(max_ls),
                max_pcg=int(max_pcg), kappa_affine=float(kappa_affine),
                gravity=tuple(float(g) for g in gravity))


def parity_params(params: dict) -> dict:
    """Tight solve settings for trajectory parity: Newton tolerance x1e-3, PCG to 1e-12."""
    p = dict(params)
    p["newton_tol"] = params["newton_tol"] * 1e-3
    p["pcg_rel_tol"] = 1e-12
    p["max_pcg"] = max(params["max_pcg"], 20000)
    return p


def _translation_q(p) -> np.ndarray:
    q = IDENTITY_Q.copy()
    q[:3] = p
    return q


# -------------------------------------------------------------------- configurations

def cube_squeeze_env(env_id: int = 0, base_seed: int = BASE_SEED, n_steps: int = 100,
                     close_steps: int | None = None, dt: float = 0.01, dhat: float = 1e-3,
                     mu: float = 0.5, cells: int = 4, size: float = 0.05,
                     E: float = 1e5, nu: float = 0.4, rho: float = 1000.0,
                     close_speed: float = 0.01, lift_speed: float = 0.02) -> dict:
    """Soft 0.05 m cube (5x5x5 vertices, 384 Kuhn tets) squeezed by two kinematic rigid plates.

    Plates start 1.5*dhat from the faces, close at `close_speed` with gravity off, then lift at
    `lift_speed` with gravity on (the gravity gating of the grasp protocol, Sec. III-D).
    Vertices get a seeded jitter U(-1e-5, 1e-5) m.
    """
    rng = SplitMix64(base_seed + env_id)
    h = size / 2
    verts, tets, _ = kuhn_grid(cells, cells, cells, (-h, -h, -h), (h, h, h))
    verts = verts + rng.uniform_array(verts.size, -1e-5, 1e-5).reshape(verts.shape)
    tris = boundary_tris(verts, tets)
    gap = 1.5 * dhat
    pt = 0.005  # plate half thickness
    pv, ptris = box_surface((pt, 0.04, 0.04))
    xmax = verts[:, 0].max()
    xmin = verts[:, 0].min()
    pl = dict(verts=pv, tris=ptris, rho=1000.0, q0=_translation_q((xmax + gap + pt, 0, 0)),
              qdot0=np.zeros(12), kinematic=True)
    pr = dict(verts=pv.copy(), tris=ptris.copy(), rho=1000.0,
              q0=_translation_q((xmin - gap - pt, 0, 0)), qdot0=np.zeros(12), kinematic=True)
    if close_steps is None:
        close_steps = n_steps // 2
    targets = np.zeros((n_steps, 3, 12))
    gravity = np.zeros(n_steps, dtype=np.uint8)
    for s in range(n_steps):
        nc = min(s + 1, close_steps)
        nl = max(s + 1 - close_steps, 0)
        dx = close_speed * dt * nc
        dz = lift_speed * dt * nl
        targets[s, 0] = IDENTITY_Q
        targets[s, 1] = _translation_q((xmax + gap + pt - dx, 0, dz))
        targets[s, 2] = _translation_q((xmin - gap - pt + dx, 0, dz))
        gravity[s] = 1 if s >= close_steps else 0
    soft = dict(verts=verts, tets=tets, tris=tris, E=E, nu=nu, rho=rho,
                kin=np.zeros(len(verts), dtype=np.uint8))
    lift = lift_speed * dt * max(n_steps - close_steps, 0)
    return dict(soft=[soft], affine=[pl, pr], mu=mu, gravity=gravity, targets=targets, object=("soft", 0), lift=lift)


def finger_pad(rng: SplitMix64, side: int, inner_x: float, E: float, nu: float,
               rho: float = 1100.0, n=(6, 8, 18), thick=0.015, width=0.04, height=0.08,
               taper=0.35, n_cutouts=3):
    """Tapered soft finger pad on a Kuhn grid with seeded rectangular cutouts.

    side=+1 puts the pad at x >= inner_x (flat contact face at x = inner_x), side=-1 mirrors it.
    The outermost vertex layer is kinematic (driven by the gripper).
    """
    nx, ny, nz = n
    mask = np.ones((nx, ny, nz), dtype=bool)
    for _ in range(n_cutouts):
        i0 = rng.randint(1, nx - 2)
        i1 = min(i0 + rng.randint(1, 3), nx - 1)
        j0 = rng.randint(0, ny - 2)
        j1 = min(j0 + rng.randint(2, 5), ny)
        k0 = rng.randint(1, nz - 4)
        k1 = min(k0 + rng.randint(2, 6), nz - 1)
        mask[i0:i1, j0:j1, k0:k1] = False
    verts, tets, grid = kuhn_grid(nx, ny, nz, (0, -width / 2, -height / 2), (thick, width / 2, height / 2), mask)
    # taper: the pad thins linearly towards its top; the contact face x=0 stays flat.
    zrel = (verts[:, 2] + height / 2) / height
    verts[:, 0] *= 1.0 - taper * zrel
    kin = (grid[:, 0] == nx).astype(np.uint8)
    verts[:, 0] = inner_x + verts[:, 0] if side > 0 else -inner_x - verts[:, 0]
    tets = _orient_tets(verts, tets.astype(np.int64)).astype(np.int32)
    tris = boundary_tris(verts, tets)
    return dict(verts=verts, tets=tets, tris=tris, E=E, nu=nu, rho=rho, kin=kin)


def hull_object(rng: SplitMix64, n_points: int = 200, dmin: float = 0.03, dmax: float = 0.08,
                subdivide: bool = True):
    """Convex hull of seeded points on an ellipsoid whose per-axis diameters are U(dmin, dmax);
    one midpoint subdivision brings 200 hull points to 1584 triangles."""
    radii = np.array([rng.uniform(dmin, dmax) / 2 for _ in range(3)])
    pts = []
    for _ in range(n_points):
        d = np.array([rng.normal(), rng.normal(), rng.normal()])
        d /= max(np.linalg.norm(d), 1e-12)
        pts.append(d * radii)
    pts = np.asarray(pts)
    verts, tris = convex_hull_surface(pts)
    if subdivide:
        verts, tris = subdivide_midpoint(verts, tris)
    return verts, tris


def pad_grasp_env(env_id: int = 0, base_seed: int = BASE_SEED, n_steps: int = 300,
                  close_steps: int = 100, dt: float = 0.005, dhat: float = 1e-3,
                  squeeze: float = 2e-3, lift: float = 0.1, pad_cells=(6, 8, 18),
                  object_points: int = 200) -> dict:
    """Two soft wedge finger pads (~5k tets each, E=2e5 Pa, nu=0.45) grasping a rigid affine
    hull object (density U(500,1500)); mu ~ U(0.3, 0.8). Close with gravity off, then lift
    0.1 m with gravity on."""
    rng = SplitMix64(base_seed + env_id)
    mu = rng.uniform(0.3, 0.8)
    ov, otris = hull_object(rng, object_points)
    rho_o = rng.uniform(500.0, 1500.0)
    gap = 1.5 * dhat
    xr = ov[:, 0].max() + gap
    xl = -ov[:, 0].min() + gap
    pad_r = finger_pad(rng, +1, xr, 2e5, 0.45, n=pad_cells)
    pad_l = finger_pad(rng, -1, xl, 2e5, 0.45, n=pad_cells)
    obj = dict(verts=ov, tris=otris, rho=rho_o, q0=IDENTITY_Q.copy(), qdot0=np.zeros(12), kinematic=False)
    close_speed_r = (gap + squeeze) / (close_steps * dt)
    lift_steps = max(n_steps - close_steps, 1)
    lift_speed = lift / (lift_steps * dt)
    targets = np.zeros((n_steps, 3, 12))
    gravity = np.zeros(n_steps, dtype=np.uint8)
    for s in range(n_steps):
        nc = min(s + 1, close_steps)
        nl = max(s + 1 - close_steps, 0)
        dx = close_speed_r * dt * nc
        dz = lift_speed * dt * nl
        targets[s, 0] = _translation_q((-dx, 0, dz))
        targets[s, 1] = _translation_q((dx, 0, dz))
        targets[s, 2] = IDENTITY_Q
        gravity[s] = 1 if s >= close_steps else 0
    return dict(soft=[pad_r, pad_l], affine=[obj], mu=mu, gravity=gravity, targets=targets,
                object=("affine", 0), lift=lift)


def _rot_x(deg: float) -> np.ndarray:
    a = math.radians(deg)
    c, s = math.cos(a), math.sin(a)
    return np.array([[1.0, 0.0, 0.0], [0.0, c, -s], [0.0, s, c]])


def grasp_request_env(req_id: int, base_seed: int = BASE_SEED + 7919, close_steps: int = 80, lift_steps: int = 60,
                      shake_steps: int = 60, shake_deg: float = 15.0, shake_hz: float = 2.0, dt: float = 0.005,
                      lift: float = 0.1, pad_cells=(6, 8, 18), object_points: int = 200) -> dict:
    """A grasp-evaluation request: the pad grasp of one seeded object (uneven hull sizes), closed
    in `close_steps`, lifted by `lift` in `lift_steps`, then shaken about the grasp (x) axis through
    the lifted object centre by shake_deg * sin(2 pi shake_hz t) for `shake_steps`."""
    n_cl = close_steps + lift_steps
    env = pad_grasp_env(req_id, base_seed=base_seed, n_steps=n_cl, close_steps=close_steps, dt=dt, lift=lift,
                        pad_cells=pad_cells, object_points=object_points)
    last = env["targets"][-1]
    c = np.array([0.0, 0.0, lift])
    frames = []
    for k in range(1, shake_steps + 1):
        R = _rot_x(shake_deg * math.sin(2.0 * math.pi * shake_hz * k * dt))
        fr = last.copy()
        for b in range(2):  # the two pads: x = R (X0 + t - c) + c
            t = last[b, :3]
            q = np.zeros(12)
            q[:3] = R @ (t - c) + c
            q[3:6], q[6:9], q[9:12] = R[:, 0], R[:, 1], R[:, 2]
            fr[b] = q
        frames.append(fr)
    if frames:
        env["targets"] = np.concatenate([env["targets"], np.array(frames)], axis=0)
        env["gravity"] = np.concatenate([env["gravity"], np.ones(shake_steps, dtype=np.uint8)])
    return env


def initial_dofs(env: dict) -> np.ndarray:
    """DOF vector of an env at its initial state: soft vertices (x, y, z) in body order, then the
    12 affine coordinates q0 of every affine body."""
    parts = [s["verts"].reshape(-1) for s in env["soft"]] + [np.asarray(a["q0"]) for a in env["affine"]]
    return np.concatenate(parts).astype(np.float64)


def pad_grasp_state_at(env: dict, step: int) -> tuple[np.ndarray, np.ndarray]:
    """Synthetic start of a pad-grasp env at schedule step `step`: every pad vertex translated by
    the displacement its kinematic base has reached at the end of step-1 (so the base sits on its
    target), the object at rest. Returns (DOFs, zero velocities)."""
    x = initial_dofs(env)
    off = 0
    for b, s in enumerate(env["soft"]):
        n = len(s["verts"])
        q = env["targets"][step - 1, b] if step > 0 else IDENTITY_Q
        x[3 * off: 3 * (off + n)].reshape(-1, 3)[:] += np.asarray(q[:3])
        off += n
    return x, np.zeros_like(x)


def star_object(rng: SplitMix64, tets_lo: int = 2000, tets_hi: int = 60000) -> dict:
    """Soft star-shaped object of log-uniform size in [tets_lo, tets_hi] tets: radius U(0.02,
    0.04) m, E log-uniform over 1e4-1e6 Pa, nu U(0.3, 0.45), rho 1000 kg/m^3 (Sec. III-B
    randomises stiffness and scale per object)."""
    target_tets = math.exp(rng.uniform(math.log(tets_lo), math.log(tets_hi)))
    # a Kuhn ball of n^3 cells keeps about (pi/6) n^3 cells, 6 tets each
    n = max(4, int(round((target_tets / (6 * math.pi / 6)) ** (1 / 3))))
    r0 = rng.uniform(0.02, 0.04)
    verts, tets = star_ball(rng, n, r0)
    tris = boundary_tris(verts, tets)
    E = math.exp(rng.uniform(math.log(1e4), math.log(1e6)))
    nu = rng.uniform(0.3, 0.45)
    return dict(verts=verts, tets=tets, tris=tris, E=E, nu=nu, rho=1000.0,
                kin=np.zeros(len(verts), dtype=np.uint8))


def soft_object_grasp_env(env_id: int, base_seed: int = BASE_SEED, n_steps: int = 100,
                          close_steps: int = 50, dt: float = 0.005, dhat: float = 1e-3,
                          tets_lo: int = 2000, tets_hi: int = 60000, bimanual: bool | None = None,
                          squeeze: float = 1.5e-3, lift: float = 0.05) -> dict:
    """Uneven-batch scene: a star-shaped soft object of log-uniform size in [tets_lo, tets_hi]
    held by rigid kinematic plates (one pair, or two pairs when bimanual)."""
    rng = SplitMix64(base_seed + env_id)
    soft = star_object(rng, tets_lo, tets_hi)
    verts = soft["verts"]
    mu = rng.uniform(0.3, 0.8)
    if bimanual is None:
        bimanual = rng.uniform() < 0.25
    gap = 1.5 * dhat
    pt = 0.004
    pv, ptris = box_surface((pt, 0.05, 0.05))
    axes = [0, 1] if bimanual else [0]
    plates = []
    for ax in axes:
        for sgn in (+1, -1):
            ext = verts[:, ax].max() if sgn > 0 else -verts[:, ax].min()
            c = np.zeros(3)
            c[ax] = sgn * (ext + gap + pt)
            q0 = _translation_q(c)
            if ax == 1:  # plate rotated so its thin axis is y: A maps rest x to world y
                q0[3:12] = [0, 1, 0, -1, 0, 0, 0, 0, 1]
            plates.append((ax, sgn, q0))
    if bimanual:
        # make the y plates shorter in x so the two pairs do not touch each other
        pv_y, ptris_y = box_surface((pt, 0.012, 0.05))
    speed = (gap + squeeze) / (close_steps * dt)
    lift_speed = lift / (max(n_steps - close_steps, 1) * dt)
    affine = []
    targets = np.zeros((n_steps, 1 + len(plates), 12))
    for b, (ax, sgn, q0) in enumerate(plates):
        v, t = (pv_y, ptris_y) if ax == 1 else (pv, ptris)
        affine.append(dict(verts=v.copy(), tris=t.copy(), rho=1000.0, q0=q0, qdot0=np.zeros(12), kinematic=True))
        for s in range(n_steps):
            nc = min(s + 1, close_steps)
            nl = max(s + 1 - close_steps, 0)
            q = q0.copy()
            q[ax] -= sgn * speed * dt * nc
            q[2] += lift_speed * dt * nl
            targets[s, 1 + b] = q
    targets[:, 0] = IDENTITY_Q
    gravity = (np.arange(n_steps) >= close_steps).astype(np.uint8)
    return dict(soft=[soft], affine=affine, mu=mu, gravity=gravity, targets=targets)


def _rot_z90(body: dict) -> dict:
    """A soft body turned by +90 degrees about z: (x, y, z) -> (-y, x, z) (a proper rotation keeps
    tet and triangle orientations)."""
    b = dict(body)
    v = body["verts"]
    b["verts"] = np.ascontiguousarray(np.stack([-v[:, 1], v[:, 0], v[:, 2]], axis=1))
    return b


def soft_pad_grasp_env(env_id: int, base_seed: int = BASE_SEED + 65537, n_steps: int = 300,
                       close_steps: int = 100, dt: float = 0.005, dhat: float = 1e-3, squeeze: float = 2e-3,
                       lift: float = 0.1, tets_lo: int = 2000, tets_hi: int = 60000,
                       bimanual: bool | None = None, pad_cells=(6, 8, 18)) -> dict:
    """The pad grasp with a soft object: two soft wedge finger pads (~5k tets each, E=2e5 Pa,
    nu=0.45; two pairs at right angles when bimanual) around a star-shaped soft object of
    log-uniform 2k-60k tets. Close with gravity off, then lift with gravity on."""
    rng = SplitMix64(base_seed + env_id)
    obj = star_object(rng, tets_lo, tets_hi)
    mu = rng.uniform(0.3, 0.8)
    if bimanual is None:
        bimanual = rng.uniform() < 0.25
    ov = obj["verts"]
    gap = 1.5 * dhat
    ext = {(0, +1): ov[:, 0].max(), (0, -1): -ov[:, 0].min(), (1, +1): ov[:, 1].max(), (1, -1): -ov[:, 1].min()}
    # two pairs: pads narrow enough that the x pair's edges stay clear of the y pair's faces
    width = 0.04 if not bimanual else min(0.04, 1.6 * min(ext.values()))
    pads, moves = [], []
    for ax in ([0, 1] if bimanual else [0]):
        for sgn in (+1, -1):
            pad = finger_pad(rng, sgn, ext[(ax, sgn)] + gap, 2e5, 0.45, n=pad_cells, width=width)
            pads.append(_rot_z90(pad) if ax == 1 else pad)
            moves.append((ax, sgn))
    speed = (gap + squeeze) / (close_steps * dt)
    lift_speed = lift / (max(n_steps - close_steps, 1) * dt)
    targets = np.zeros((n_steps, len(pads) + 1, 12))
    for s in range(n_steps):
        nc = min(s + 1, close_steps)
        nl = max(s + 1 - close_steps, 0)
        for b, (ax, sgn) in enumerate(moves):
            d = np.zeros(3)
            d[ax] = -sgn * speed * dt * nc
            d[2] = lift_speed * dt * nl
            targets[s, b] = _translation_q(d)
        targets[s, len(pads)] = IDENTITY_Q
    gravity = (np.arange(n_steps) >= close_steps).astype(np.uint8)
    return dict(soft=pads + [obj], affine=[], mu=mu, gravity=gravity, targets=targets,
                object=("soft", len(pads)), lift=lift)


UNEVEN_SEED = BASE_SEED + 1048576


def uneven_batch_env(env_id: int, base_seed: int = UNEVEN_SEED) -> dict:
    """One environment of the uneven batch: with equal odds the plate squeeze (a soft object
    between kinematic rigid plates: the single-env configuration's form) or the pad grasp (soft
    finger pads: the pad configuration's form), each holding a star-shaped soft object of
    log-uniform 2k-60k tets, with two gripper pairs in a quarter of the envs. dt = 5 ms. Every
    env's schedule leaves its grippers 0.7-0.8 mm from the object at step UNEVEN_START_STEP."""
    rng = SplitMix64(base_seed + env_id)
    pads = rng.uniform() < 0.5
    bimanual = rng.uniform() < 0.25
    if pads:
        return soft_pad_grasp_env(env_id, base_seed=base_seed + 7, bimanual=bimanual)
    return soft_object_grasp_env(env_id, base_seed=base_seed + 7, n_steps=150, close_steps=75,
                                 bimanual=bimanual)


UNEVEN_START_STEP = 20

SERVE_SEED = BASE_SEED + 2097152


def serving_request_env(req_id: int, base_seed: int = SERVE_SEED, close_steps: int = 70, lift_steps: int = 50,
                        shake_steps: int = 60, hold_steps: int = 20, shake_deg: float = 15.0, shake_hz: float = 2.0,
                        dt: float = 0.005, lift: float = 0.05, tets_lo: int = 1000, tets_hi: int = 100000) -> dict:
    """A grasp-evaluation request of the serving workload: with equal odds the plate squeeze or the
    soft-pad grasp of a star-shaped soft object of log-uniform tets_lo-tets_hi tets (one gripper
    pair). The grippers close from 1.5 dhat away in `close_steps` (gravity off), lift by `lift`,
    shake the object about the grasp (x) axis through its lifted centre by
    shake_deg * sin(2 pi shake_hz t), then hold still for `hold_steps` (gravity on), at the end of
    which the grasp is labelled (Sec. III-D: the object still touches a gripper and its centre of
    mass moves less than eps_v dt in the last step)."""
    rng = SplitMix64(base_seed + req_id)
    pads = rng.uniform() < 0.5
    cl = close_steps + lift_steps
    if pads:
        env = soft_pad_grasp_env(req_id, base_seed=base_seed + 7, n_steps=cl, close_steps=close_steps, dt=dt,
                                 lift=lift, tets_lo=tets_lo, tets_hi=tets_hi, bimanual=False)
    else:
        env = soft_object_grasp_env(req_id, base_seed=base_seed + 7, n_steps=cl, close_steps=close_steps, dt=dt,
                                    lift=lift, tets_lo=tets_lo, tets_hi=tets_hi, bimanual=False)
    last = env["targets"][-1]
    nb = last.shape[0]
    grip = [b for b in range(nb) if not (len(env["soft"]) > b and not np.any(env["soft"][b]["kin"]))]
    c = np.array([0.0, 0.0, lift])
    frames = []
    for k in range(1, shake_steps + hold_steps + 1):
        ang = shake_deg * math.sin(2.0 * math.pi * shake_hz * min(k, shake_steps) * dt)
        R = _rot_x(ang if k <= shake_steps else 0.0)
        fr = last.copy()
        for b in grip:  # a gripper q: x = R (A0 X + t - c) + c
            A0 = np.stack([last[b, 3:6], last[b, 6:9], last[b, 9:12]], axis=1)
            q = np.zeros(12)
            q[:3] = R @ (last[b, :3] - c) + c
            RA = R @ A0
            q[3:6], q[6:9], q[9:12] = RA[:, 0], RA[:, 1], RA[:, 2]
            fr[b] = q
        frames.append(fr)
    env["targets"] = np.concatenate([env["targets"], np.array(frames)], axis=0)
    env["gravity"] = np.concatenate([env["gravity"], np.ones(shake_steps + hold_steps, dtype=np.uint8)])
    if "object" not in env:
        env["object"] = ("soft", 0)
    env["lift"] = lift
    return env


def uneven_batch_cost(env_id: int, base_seed: int = UNEVEN_SEED) -> float:
    """Estimated work of uneven_batch_env(env_id) without building it: its tet count (the object's
    drawn size plus ~5k tets per soft pad) and its surface size, a proxy for its contacts (n_t +
    n_c, the units the per-env stages scale with). Replays only the seeded draws that fix the
    sizes."""
    rng = SplitMix64(base_seed + env_id)
    pads = rng.uniform() < 0.5
    bimanual = rng.uniform() < 0.25
    inner = SplitMix64(base_seed + 7 + env_id)
    obj = math.exp(inner.uniform(math.log(2000), math.log(60000)))
    n_pads = (4 if bimanual else 2) if pads else 0
    tets = obj + 5000.0 * n_pads
    surface = 6.0 * obj ** (2.0 / 3.0) + 2100.0 * n_pads
    return tets + surface


def lpt_shards(costs, world: int) -> list[list[int]]:
    """Greedy longest-processing-time partition of items with the given costs over `world` bins:
    items in decreasing cost (ties by index) each go to the bin with the least total so far
    (ties to the lowest bin). Every bin's items are returned in ascending order."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    bins = [[] for _ in range(world)]
    for i in order:
        b = min(range(world), key=lambda r: (load[r], r))
        load[b] += costs[i]
        bins[b].append(i)
    return [sorted(b) for b in bins]


def grasp_state_at(env: dict, step: int) -> tuple[np.ndarray, np.ndarray]:
    """Synthetic start of a grasp env at schedule step `step`: every soft body with kinematic
    vertices translated by the displacement its schedule reaches at the end of step-1, every
    kinematic affine body at its scheduled coordinates, everything else at rest where it was
    built. Returns (DOFs, zero velocities)."""
    x = initial_dofs(env)
    off = 0
    for b, s in enumerate(env["soft"]):
        n = len(s["verts"])
        if step > 0 and np.any(s["kin"]):
            x[3 * off: 3 * (off + n)].reshape(-1, 3)[:] += np.asarray(env["targets"][step - 1, b][:3])
        off += n
    ns = len(env["soft"])
    for a, body in enumerate(env["affine"]):
        if step > 0 and body["kinematic"]:
            x[3 * off + 12 * a: 3 * off + 12 * (a + 1)] = env["targets"][step - 1, ns + a]
    return x, np.zeros_like(x)


# ---------------------------------------------------------------- small test scenes

def single_tet_env(n_steps: int = 1, offset=(0.0, 0.0, 0.0)) -> dict:
    """One free tet with no contact partner (free-fall and elasticity checks)."""
    v = np.array([[0, 0, 0], [0.01, 0, 0], [0, 0.01, 0], [0, 0, 0.01]], dtype=np.float64) + np.asarray(offset)
    tets = np.array([[0, 1, 2, 3]], dtype=np.int32)
    tris = boundary_tris(v, tets)
    soft = dict(verts=v, tets=tets, tris=tris, E=1e5, nu=0.4, rho=1000.0, kin=np.zeros(4, dtype=np.uint8))
    return dict(soft=[soft], affine=[], mu=0.0, gravity=np.ones(n_steps, dtype=np.uint8),
                targets=np.tile(IDENTITY_Q, (n_steps, 1, 1)))


def _rot_y(deg: float) -> np.ndarray:
    th = math.radians(deg)
    return np.array([[math.cos(th), 0, math.sin(th)], [0, 1, 0], [-math.sin(th), 0, math.cos(th)]])


def _q_from(R: np.ndarray, p) -> np.ndarray:
    q = IDENTITY_Q.copy()
    q[:3] = p
    q[3:6], q[6:9], q[9:12] = R[:, 0], R[:, 1], R[:, 2]
    return q


def ground_triangle(L: float = 0.2):
    """One large triangle in the z=0 plane covering [-L, L]^2 (a one-sided kinematic ground:
    a body touching it meets exactly one triangle and none of its edges)."""
    v = np.array([[-L, -L, 0.0], [3 * L, -L, 0.0], [-L, 3 * L, 0.0]])
    return v, np.array([[0, 1, 2]], dtype=np.int32)


def resting_env(body: str = "tet", n_steps: int = 100, mu: float = 0.0, incline_deg: float = 0.0,
                dhat: float = 1e-3, gap: float | None = None, size: float = 0.02, E: float = 1e6,
                rho: float = 1000.0, cells: int = 2) -> dict:
    """A body resting under gravity on a fixed ground triangle inclined about the y axis.

    body = "tet": one tet with a horizontal base and its apex over the base centroid;
    "block": a soft Kuhn block; "rigid": a free affine box.
    """
    if gap is None:
        gap = 0.5 * dhat
    R = _rot_y(incline_deg)
    gv, gt = ground_triangle()
    ground = dict(verts=gv, tris=gt, rho=1000.0, q0=_q_from(R, (0, 0, 0)), qdot0=np.zeros(12), kinematic=True)
    h = size / 2
    if body == "rigid":
        bv, bt = box_surface((h, h, h))
        q0 = _q_from(R, R @ np.array([0, 0, h + gap]))
        obj = dict(verts=bv, tris=bt, rho=rho, q0=q0, qdot0=np.zeros(12), kinematic=False)
        targets = np.zeros((n_steps, 2, 12))
        targets[:, 0] = q0
        targets[:, 1] = ground["q0"]
        return dict(soft=[], affine=[obj, ground], mu=mu, gravity=np.ones(n_steps, dtype=np.uint8),
                    targets=targets)
    if body == "tet":
        r = size / 2
        base = np.array([[r * math.cos(a), r * math.sin(a), 0.0] for a in (0.3, 0.3 + 2 * math.pi / 3, 0.3 + 4 * math.pi / 3)])
        verts = np.vstack([base, [[0.0, 0.0, size]]]) + np.array([0, 0, gap])
        tets = _orient_tets(verts, np.array([[0, 1, 2, 3]])).astype(np.int32)
    else:
        verts, tets, _ = kuhn_grid(cells, cells, cells, (-h, -h, 0.0), (h, h, size))
        verts = verts + np.array([0, 0, gap])
    verts = verts @ R.T
    tris = boundary_tris(verts, tets)
    soft = dict(verts=verts, tets=tets, tris=tris, E=E, nu=0.3, rho=rho, kin=np.zeros(len(verts), dtype=np.uint8))
    targets = np.zeros((n_steps, 2, 12))
    targets[:, 0] = IDENTITY_Q
    targets[:, 1] = ground["q0"]
    return dict(soft=[soft], affine=[ground], mu=mu, gravity=np.ones(n_steps, dtype=np.uint8), targets=targets)


def stacked_boxes_env(n_steps: int = 100, mu: float = 0.0, dhat: float = 1e-3, rho: float = 1000.0) -> dict:
    """A free rigid cube (half side 0.01 m) resting, centred, on a fixed wider box (half sides
    0.02, 0.02, 0.01 m) a gap dhat/2 above its top face. Both boxes split their horizontal faces
    along the same (1, 1, 0) diagonal, so the cube's bottom diagonal lies exactly parallel to
    the fixed box's top diagonal, straight above it: an edge-edge pair with parallel edges."""
    gap = 0.5 * dhat
    lv, lt = box_surface((0.02, 0.02, 0.01))
    base = dict(verts=lv, tris=lt, rho=rho, q0=_q_from(np.eye(3), (0, 0, 0)), qdot0=np.zeros(12), kinematic=True)
    cv, ct = box_surface((0.01, 0.01, 0.01))
    q0 = _q_from(np.eye(3), (0, 0, 0.02 + gap))
    cube = dict(verts=cv, tris=ct, rho=rho, q0=q0, qdot0=np.zeros(12), kinematic=False)
    targets = np.zeros((n_steps, 2, 12))
    targets[:, 0] = q0
    targets[:, 1] = base["q0"]
    return dict(soft=[], affine=[cube, base], mu=mu, gravity=np.ones(n_steps, dtype=np.uint8), targets=targets)


def spinning_body_env(n_steps: int = 20, omega=(0.0, 0.0, 20.0)) -> dict:
    """A free rigid box spinning in free flight with gravity off (A A^T stays close to I)."""
    bv, btris = box_surface((0.02, 0.01, 0.005))
    q0 = IDENTITY_Q.copy()
    w = np.asarray(omega, dtype=np.float64)
    W = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])
    Adot = W  # d/dt of A at A = I
    qdot0 = np.zeros(12)
    qdot0[3:6], qdot0[6:9], qdot0[9:12] = Adot[:, 0], Adot[:, 1], Adot[:, 2]
    body = dict(verts=bv, tris=btris, rho=800.0, q0=q0, qdot0=qdot0, kinematic=False)
    return dict(soft=[], affine=[body], mu=0.0, gravity=np.zeros(n_steps, dtype=np.uint8),
                targets=np.tile(IDENTITY_Q, (n_steps, 1, 1)))


def link_surface(rng: SplitMix64, length: float, radius: float, n_points: int = 250):
    """A finger link: convex hull of seeded points on an ellipsoid of semi-axes (radius, radius,
    length / 2), long axis along local z (about 2 n_points - 4 triangles)."""
    radii = np.array([radius, radius, 0.5 * length])
    pts = []
    for _ in range(n_points):
        d = np.array([rng.normal(), rng.normal(), rng.normal()])
        d /= max(np.linalg.norm(d), 1e-12)
        pts.append(d * radii)
    return convex_hull_surface(np.asarray(pts))


def _q_pose(R: np.ndarray, c: np.ndarray) -> np.ndarray:
    q = np.zeros(12)
    q[:3] = c
    q[3:6], q[6:9], q[9:12] = R[:, 0], R[:, 1], R[:, 2]
    return q


def hand_grasp_env(env_id: int, base_seed: int = BASE_SEED + 104729, n_steps: int = 400, close_steps: int = 200,
                   dt: float = 0.005, dhat: float = 5e-4, cells: int = 19, k_pd: float = 2.5e5, lift: float = 0.05,
                   link_points: int = 250, k_joint: float | None = 1e5) -> dict:
    """Rigid hand of 20 PD-driven affine links (5 fingers x 4; each link a ~500-triangle hull)
    grasping a seeded star-shaped soft object (Kuhn ball of `cells`^3 cells, about 21k tets for 19;
    E log-uniform in [1e4, 1e6] Pa, nu U(0.3, 0.48)). Finger f hangs in the vertical half-plane at
    azimuth 2 pi f / 5 above and outside the object; its four joint angles curl it toward the
    object over `close_steps` (gravity off), then every link target rises by `lift` (gravity on).
    Links are free bodies pulled toward their targets by the PD target potential (k_pd 1/s^2; the
    default makes a finger press about k_pd m_link (4 mm) = 2 N into the object, enough for five
    fingers to hold its ~1 N weight by friction).
    With k_joint (N/m) the hand is articulated: each finger's first link hangs from a kinematic
    palm (a small box above the object, the last affine body) and each further link from the
    previous one by a hinge on the finger's bending axis, two point joints at +/- the link
    radius along it (20 hinges, 40 point joints); None leaves the links unjointed."""
    rng = SplitMix64(base_seed + env_id)
    E = math.exp(rng.uniform(math.log(1e4), math.log(1e6)))
    nu = rng.uniform(0.3, 0.48)
    r0 = 0.03
    verts, tets = star_ball(rng, cells, r0)
    tris = boundary_tris(verts, tets)
    rmax = float(np.linalg.norm(verts, axis=1).max())
    soft = dict(verts=verts, tets=tets, tris=tris, E=E, nu=nu, rho=1000.0, kin=np.zeros(len(verts), dtype=np.uint8))
    L, rw, gap = 0.018, 0.0055, 3.0 * dhat
    base_r, base_z = rmax + 0.028, 0.5 * rmax + 0.012
    theta0 = np.radians([-25.0, 5.0, 5.0, 5.0])      # first joint tilts the finger outward
    dtheta = np.radians([31.5, 17.5, 14.0, 10.5])    # curl: fingertips end ~13% inside the object
    links, poses = [], []  # poses[s][link] = q
    link_shapes = [link_surface(rng, L - gap, rw, link_points) for _ in range(20)]

    def finger_pose(phi: float, theta: np.ndarray, dz: float):
        er = np.array([math.cos(phi), math.sin(phi), 0.0])
        et = np.array([-math.sin(phi), math.cos(phi), 0.0])
        joint = base_r * er + np.array([0.0, 0.0, base_z + dz])
        beta, out = 0.0, []
        for k in range(4):
            beta += theta[k]
            u = -math.sin(beta) * er - math.cos(beta) * np.array([0.0, 0.0, 1.0])  # down, toward axis
            c = joint + 0.5 * L * u
            e3 = u
            e1 = et
            e2 = np.cross(e3, e1)
            out.append(_q_pose(np.stack([e1, e2, e3], axis=1), c))
            joint = joint + L * u
        return out

    phis = [2.0 * math.pi * f / 5 + rng.uniform(-0.1, 0.1) for f in range(5)]
    targets = np.zeros((n_steps, 21, 12))
    gravity = np.zeros(n_steps, dtype=np.uint8)
    for s_ in range(n_steps):
        a = min(1.0, (s_ + 1) / close_steps)
        dz = lift * max(0.0, (s_ + 1 - close_steps) / max(n_steps - close_steps, 1))
        targets[s_, 0] = IDENTITY_Q
        qs = []
        for phi in phis:
            qs += finger_pose(phi, theta0 + a * dtheta, dz)
        targets[s_, 1:] = np.array(qs)
        gravity[s_] = 1 if s_ >= close_steps else 0
    q_init = []
    for phi in phis:
        q_init += finger_pose(phi, theta0, 0.0)
    for k in range(20):
        lv, lt = link_shapes[k]
        links.append(dict(verts=lv, tris=lt, rho=1200.0, q0=q_init[k], qdot0=np.zeros(12), kinematic=False, pd=k_pd))
    mu = rng.uniform(0.5, 0.9)
    if k_joint is None:
        return dict(soft=[soft], affine=links, mu=mu, gravity=gravity, targets=targets, object=("soft", 0), lift=lift)
    # palm: a kinematic box above the object (clear of it and of the fingers), rising with the lift
    c_palm = np.array([0.0, 0.0, rmax + 0.02])
    pv, ptr = box_surface((0.01, 0.01, 0.004))
    palm = dict(verts=pv, tris=ptr, rho=1000.0, q0=_translation_q(c_palm), qdot0=np.zeros(12), kinematic=True)
    tg = np.zeros((n_steps, 22, 12))
    tg[:, :21] = targets
    for s_ in range(n_steps):
        dz = lift * max(0.0, (s_ + 1 - close_steps) / max(n_steps - close_steps, 1))
        tg[s_, 21] = _translation_q(c_palm + np.array([0.0, 0.0, dz]))
    joints = []
    for f, phi in enumerate(phis):
        er = np.array([math.cos(phi), math.sin(phi), 0.0])
        et = np.array([-math.sin(phi), math.cos(phi), 0.0])
        base = base_r * er + np.array([0.0, 0.0, base_z])
        for sgn in (+1.0, -1.0):
            joints.append(dict(a=20, b=4 * f, anchor_a=base + sgn * rw * et - c_palm,
                               anchor_b=np.array([sgn * rw, 0.0, -0.5 * L]), k=k_joint))
            for k in range(1, 4):
                joints.append(dict(a=4 * f + k - 1, b=4 * f + k, anchor_a=np.array([sgn * rw, 0.0, 0.5 * L]),
                                   anchor_b=np.array([sgn * rw, 0.0, -0.5 * L]), k=k_joint))
    return dict(soft=[soft], affine=links + [palm], mu=mu, gravity=gravity, targets=tg, object=("soft", 0),
                lift=lift, joints=joints)


def pendulum_env(k_joint: float = 1e4, n_steps: int = 100, theta0: float = 0.0, arm: float = 0.1,
                 half: float = 0.01, rho: float = 1000.0, gravity: bool = True, wall_y: float | None = None,
                 mu: float = 0.0) -> dict:
    """A rigid cube (half side `half`) hanging by a point joint from a fixed kinematic pivot: the
    joint's anchor sits `arm` above the cube's centre in the cube's frame and at the world
    origin in the pivot's; the cube starts at rest turned by theta0 about the x axis through the
    joint. Pivot and cube are far apart (no contact). With wall_y, a fixed kinematic wall (a thin
    box whose face is the plane y = wall_y, below the pivot) stands in the cube's swing."""
    bv, bt = box_surface((half, half, half))
    pv, pt_ = box_surface((half, half, half))
    pivot_c = np.array([0.0, 0.0, 0.05])
    pivot = dict(verts=pv, tris=pt_, rho=rho, q0=_translation_q(pivot_c), qdot0=np.zeros(12), kinematic=True)
    R = _rot_x(math.degrees(theta0))
    bob = dict(verts=bv, tris=bt, rho=rho, q0=_q_pose(R, R @ np.array([0.0, 0.0, -arm])), qdot0=np.zeros(12),
               kinematic=False)
    targets = np.zeros((n_steps, 2, 12))
    targets[:, 0] = pivot["q0"]
    targets[:, 1] = bob["q0"]
    joint = dict(a=0, b=1, anchor_a=-pivot_c, anchor_b=np.array([0.0, 0.0, arm]), k=k_joint)
    affine = [pivot, bob]
    if wall_y is not None:
        wv, wt = box_surface((0.05, 0.005, 0.03))
        c = np.array([0.0, wall_y - 0.005 if wall_y < 0 else wall_y + 0.005, -arm])
        affine.append(dict(verts=wv, tris=wt, rho=rho, q0=_translation_q(c), qdot0=np.zeros(12), kinematic=True))
        targets = np.concatenate([targets, np.tile(affine[-1]["q0"], (n_steps, 1, 1))], axis=1)
    return dict(soft=[], affine=affine, mu=mu, gravity=np.full(n_steps, 1 if gravity else 0, dtype=np.uint8),
                targets=targets, joints=[joint])


def pd_body_env(k_pd: float = 400.0, n_steps: int = 100, gravity: bool = True, target_shift=(0.0, 0.0, 0.0),
                shift_steps: int = 0) -> dict:
    """A free rigid box held by a PD target potential (stiffness k_pd, 1/s^2) toward its initial
    pose, or toward a pose translated by `target_shift` over the first `shift_steps` steps."""
    bv, btris = box_surface((0.02, 0.015, 0.01))
    body = dict(verts=bv, tris=btris, rho=800.0, q0=IDENTITY_Q.copy(), qdot0=np.zeros(12), kinematic=False, pd=k_pd)
    targets = np.tile(IDENTITY_Q, (n_steps, 1, 1))
    sh = np.asarray(target_shift, dtype=np.float64)
    for s in range(n_steps):
        f = min(1.0, (s + 1) / shift_steps) if shift_steps > 0 else (1.0 if sh.any() else 0.0)
        targets[s, 0, :3] = f * sh
    return dict(soft=[], affine=[body], mu=0.0, gravity=np.full(n_steps, 1 if gravity else 0, dtype=np.uint8),
                targets=targets)


def env_sizes(env: dict) -> dict:
    """Counts used to size buffers and to report workloads."""
    nv = sum(len(s["verts"]) for s in env["soft"])
    nt = sum(len(s["tets"]) for s in env["soft"])
    ntri = sum(len(s["tris"]) for s in env["soft"]) + sum(len(a["tris"]) for a in env["affine"])
    return dict(soft_verts=nv, tets=nt, tris=ntri, bodies=len(env["affine"]),
                dofs=3 * nv + 12 * len(env["affine"]), steps=len(env["gravity"]))
