"""The allocation-free energy entry point against the scene path (needs a B300).

Some callers of this library cannot allocate device memory: real-time control loops that must
not pay for (or fail on) an allocation, and hosts whose memory manager owns every device
allocation and forbids others. ipc_elastic_energy_noalloc serves them: it
takes caller-owned device buffers and uses only a fixed scratch array inside the library. Here
its result for a deformed soft cube must equal the energy ipc_eval reports for the same state
(where inertia, contact and friction terms vanish), on two calls in a row.
"""
import ctypes as C

import numpy as np
import pytest

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


def tet_params(verts, tets, E, nu):
    mu = E / (2 * (1 + nu))
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    out = np.zeros((len(tets), 12))
    for t, T in enumerate(tets):
        Dm = np.stack([verts[T[1]] - verts[T[0]], verts[T[2]] - verts[T[0]], verts[T[3]] - verts[T[0]]], axis=1)
        out[t, :9] = np.linalg.inv(Dm).ravel()
        out[t, 9] = np.linalg.det(Dm) / 6.0
        out[t, 10], out[t, 11] = mu, lam
    return out


def test_noalloc_energy_matches_scene_eval_twice():
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
    half = n // 2
    offs = torch.tensor([0, half, n], dtype=torch.int32, device=dev)
    energy = torch.full((2,), -1.0, dtype=torch.float64, device=dev)
    inverted = torch.full((2,), 7, dtype=torch.int32, device=dev)
    L = ipc.lib()
    h2 = p["dt"] ** 2
    results = []
    for _ in range(2):
        st = L.ipc_elastic_energy_noalloc(n, C.c_void_p(tets.data_ptr()), C.c_void_p(prm.data_ptr()),
                                          C.c_void_p(x.data_ptr()), 2, C.c_void_p(offs.data_ptr()), h2,
                                          C.c_void_p(energy.data_ptr()), C.c_void_p(inverted.data_ptr()), None)
        assert st == 0, L.ipc_last_error()
        torch.cuda.synchronize()
        results.append((energy.cpu().numpy().copy(), inverted.cpu().numpy().copy()))
    for e, inv in results:
        assert np.all(inv == 0)
        assert abs(e.sum() - E_ref) <= TOL * abs(E_ref), (e.sum(), E_ref)
    assert np.array_equal(results[0][0], results[1][0])

    # an inverted tet flags its group and counts as zero energy
    x_bad = x_def.copy()
    T0 = s["tets"][0]
    a, b, c = x_def[T0[1]], x_def[T0[2]], x_def[T0[3]]
    nrm = np.cross(b - a, c - a)
    nrm /= np.linalg.norm(nrm)
    x_bad[T0[0]] = x_def[T0[0]] - 2 * np.dot(x_def[T0[0]] - a, nrm) * nrm  # mirror through the opposite face
    xb = torch.tensor(x_bad, dtype=torch.float64, device=dev).contiguous()
    st = L.ipc_elastic_energy_noalloc(n, C.c_void_p(tets.data_ptr()), C.c_void_p(prm.data_ptr()),
                                      C.c_void_p(xb.data_ptr()), 2, C.c_void_p(offs.data_ptr()), h2,
                                      C.c_void_p(energy.data_ptr()), C.c_void_p(inverted.data_ptr()), None)
    assert st == 0
    torch.cuda.synchronize()
    assert inverted.cpu().numpy()[0] == 1


def test_noalloc_rejects_sizes_above_the_maximum():
    L = ipc.lib()
    st = L.ipc_elastic_energy_noalloc(262144 + 1, C.c_void_p(1), C.c_void_p(1), C.c_void_p(1), 1, C.c_void_p(1),
                                      1.0, C.c_void_p(1), C.c_void_p(1), None)
    assert st == 1
    assert b"maximum" in L.ipc_last_error()
