"""The allocation-free energy entry point against the scene path and the oracle (needs a B300).

Some callers of this library cannot allocate device memory: real-time control loops that must
not pay for (or fail on) an allocation, and hosts whose memory manager owns every device
allocation and forbids others. ipc_elastic_energy_noalloc serves them: it takes caller-owned
device buffers and uses only a fixed scratch array inside the library. Here its per-group energy
for a deformed soft cube must equal, on two calls in a row, the energy ipc_eval reports for the
same state (where inertia, contact and friction terms vanish) and the oracle's Neo-Hookean
energy summed tet by tet.
"""
import ctypes as C

import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_05020_b300 import ipc
from paper_2503_05020_b300 import scenes as S

pytestmark = pytest.mark.gpu

TOL = 1e-10


def soft_cube_alone(n_steps=2):
    h = 0.025
    verts, tets, _ = S.kuhn_grid(4, 4, 4, (-h, -h, -h), (h, h, h))
    tris = S.boundary_tris(verts, tets)
    soft = dict(verts=verts, tets=tets, tris=tris, E=1e5, nu=0.4, rho=1000.0, kin=np.zeros(len(verts), dtype=np.uint8))
    return dict(soft=[soft], affine=[], mu=0.0, gravity=np.zeros(n_steps, dtype=np.uint8),
                targets=np.tile(S.IDENTITY_Q, (n_steps, 1, 1)))


def lame(E, nu):
    return E / (2 * (1 + nu)), E * nu / ((1 + nu) * (1 - 2 * nu))


def tet_params(verts, tets, E, nu):
    mu, lam = lame(E, nu)
    out = np.zeros((len(tets), 12))
    for t, T in enumerate(tets):
        Dm = np.stack([verts[T[1]] - verts[T[0]], verts[T[2]] - verts[T[0]], verts[T[3]] - verts[T[0]]], axis=1)
        out[t, :9] = np.linalg.inv(Dm).ravel()
        out[t, 9] = np.linalg.det(Dm) / 6.0
        out[t, 10], out[t, 11] = mu, lam
    return out


def oracle_group_energy(rest, x, tets, E, nu, h2, offs):
    """h2 V Psi(F) per tet from the oracle's Neo-Hookean energy, F = Ds Dm^-1; a tet with J <= 0
    counts 0 and flags its group. Returns (energy per group, flag per group)."""
    mu, lam = lame(E, nu)
    e_t, inv_t = np.zeros(len(tets)), np.zeros(len(tets), dtype=bool)
    for t, T in enumerate(tets):
        Dm = np.stack([rest[T[k]] - rest[T[0]] for k in (1, 2, 3)], axis=1)
        Ds = np.stack([x[T[k]] - x[T[0]] for k in (1, 2, 3)], axis=1)
        F = Ds @ np.linalg.inv(Dm)
        if np.linalg.det(F) <= 0:
            inv_t[t] = True
            continue
        psi, _, _ = O.neo_hookean(F, mu, lam)
        e_t[t] = h2 * (np.linalg.det(Dm) / 6.0) * psi
    n = len(offs) - 1
    return (np.array([e_t[offs[g]:offs[g + 1]].sum() for g in range(n)]),
            np.array([int(inv_t[offs[g]:offs[g + 1]].any()) for g in range(n)]))


def call(L, n, tets, prm, x, offs, h2, energy, inverted, ptr_shift=0):
    return L.ipc_elastic_energy_noalloc(n, C.c_void_p(tets.data_ptr() + ptr_shift), C.c_void_p(prm.data_ptr()),
                                        C.c_void_p(x.data_ptr()), len(offs) - 1, C.c_void_p(offs.data_ptr()), h2,
                                        C.c_void_p(energy.data_ptr()), C.c_void_p(inverted.data_ptr()), None)


def test_noalloc_energy_matches_scene_eval_and_oracle_twice():
    import torch

    torch.cuda.init()
    p = S.scene_params(0.01)
    env = soft_cube_alone()
    s = env["soft"][0]
    sc = ipc.Scene(p)
    eid = sc.add_env(env)
    x_def = s["verts"] * np.array([1.08, 0.97, 1.0]) + 0.02 * s["verts"][:, [1, 2, 0]]  # stretch + shear
    q = x_def.ravel()
    sc.set_state(eid, q, np.zeros_like(q), 0)
    E_ref = sc.eval(eid, q, grad=False)
    assert E_ref > 0

    dev = torch.device("cuda", 0)
    tets = torch.tensor(s["tets"], dtype=torch.int32, device=dev).contiguous()
    prm = torch.tensor(tet_params(s["verts"], s["tets"], s["E"], s["nu"]), dtype=torch.float64, device=dev).contiguous()
    x = torch.tensor(x_def, dtype=torch.float64, device=dev).contiguous()
    n = len(s["tets"])
    offs_h = [0, n // 2, n]
    offs = torch.tensor(offs_h, dtype=torch.int32, device=dev)
    energy = torch.full((2,), -1.0, dtype=torch.float64, device=dev)
    inverted = torch.full((2,), 7, dtype=torch.int32, device=dev)
    L = ipc.lib()
    h2 = p["dt"] ** 2
    e_or, inv_or = oracle_group_energy(s["verts"], x_def, s["tets"], s["E"], s["nu"], h2, offs_h)
    assert not inv_or.any()
    results = []
    for _ in range(2):
        st = call(L, n, tets, prm, x, offs, h2, energy, inverted)
        assert st == 0, L.ipc_last_error()
        torch.cuda.synchronize()
        results.append((energy.cpu().numpy().copy(), inverted.cpu().numpy().copy()))
    for e, inv in results:
        assert np.all(inv == 0)
        assert abs(e.sum() - E_ref) <= TOL * abs(E_ref), (e.sum(), E_ref)  # the scene path's energy
        assert np.all(np.abs(e - e_or) <= TOL * np.abs(e_or)), (e, e_or)  # the oracle, per group
    assert np.array_equal(results[0][0], results[1][0])

    # an inverted tet counts as zero energy and flags its group; the other group is untouched
    x_bad = x_def.copy()
    T0 = s["tets"][0]
    a, b, c = x_def[T0[1]], x_def[T0[2]], x_def[T0[3]]
    nrm = np.cross(b - a, c - a)
    nrm /= np.linalg.norm(nrm)
    x_bad[T0[0]] = x_def[T0[0]] - 2 * np.dot(x_def[T0[0]] - a, nrm) * nrm  # mirror through the opposite face
    e_or, inv_or = oracle_group_energy(s["verts"], x_bad, s["tets"], s["E"], s["nu"], h2, offs_h)
    assert inv_or[0] == 1
    xb = torch.tensor(x_bad, dtype=torch.float64, device=dev).contiguous()
    st = call(L, n, tets, prm, xb, offs, h2, energy, inverted)
    assert st == 0
    torch.cuda.synchronize()
    e, inv = energy.cpu().numpy(), inverted.cpu().numpy()
    assert np.array_equal(inv, inv_or), (inv, inv_or)
    assert np.all(np.abs(e - e_or) <= TOL * np.abs(e_or)), (e, e_or)


def test_noalloc_rejects_sizes_above_the_maximum_and_misaligned_pointers():
    L = ipc.lib()
    st = L.ipc_elastic_energy_noalloc(262144 + 1, C.c_void_p(16), C.c_void_p(16), C.c_void_p(16), 1, C.c_void_p(16),
                                      1.0, C.c_void_p(16), C.c_void_p(16), None)
    assert st == 1
    assert b"maximum" in L.ipc_last_error()
    # a tet index array that does not start on an int boundary is refused before any launch
    st = L.ipc_elastic_energy_noalloc(4, C.c_void_p(18), C.c_void_p(16), C.c_void_p(16), 1, C.c_void_p(16),
                                      1.0, C.c_void_p(16), C.c_void_p(16), None)
    assert st == 1
    assert b"aligned" in L.ipc_last_error()
