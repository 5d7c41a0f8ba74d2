"""ctypes wrapper of the plain FP64 CPU oracle (ipc_oracle.cpp).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the CPU-baseline leg
of the benchmark. The product path never imports this module. It shares no code with the CUDA
path; both are fed from the seeded scene dictionaries of `paper_2503_05020_b300.scenes`.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ipc_oracle.cpp")
LIB = os.path.join(HERE, "liboracle_ipc.so")


def build(force: bool = False) -> str:
    """Compile the oracle with -O2 -ffp-contract=off (every expression rounds as written)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-pthread", SRC, "-o", LIB + ".tmp"]
        subprocess.check_call(cmd)
        os.replace(LIB + ".tmp", LIB)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        P = C.POINTER
        d, i32, vp = C.c_double, C.c_int32, C.c_void_p
        L.or_env_create.restype = vp
        L.or_env_create.argtypes = [vp, vp]
        L.or_env_destroy.argtypes = [vp]
        L.or_env_ndof.argtypes = [vp]
        L.or_env_npoints.argtypes = [vp]
        L.or_env_step.argtypes = [vp, C.c_int]
        L.or_run_batch.argtypes = [P(vp), C.c_int, C.c_int, C.c_int]
        L.or_env_get_state.argtypes = [vp, vp, vp]
        L.or_env_set_state.argtypes = [vp, vp, vp, C.c_int]
        L.or_env_status.argtypes = [vp, vp, vp, vp]
        L.or_env_eval.restype = d
        L.or_env_eval.argtypes = [vp, vp, vp]
        L.or_env_hessian.argtypes = [vp, vp, vp]
        L.or_env_newton_dir.argtypes = [vp, vp]
        L.or_env_candidates.argtypes = [vp, vp, vp, vp, C.c_int]
        L.or_env_contacts.argtypes = [vp, vp, vp, vp, C.c_int]
        L.or_env_points.argtypes = [vp, vp, vp]
        L.or_env_invariants.argtypes = [vp, vp, vp]
        L.or_env_trace.argtypes = [vp, C.c_int]
        L.or_env_kappa.restype = d
        L.or_env_kappa.argtypes = [vp]
        L.or_env_tet_stress.argtypes = [vp, vp, vp]
        L.or_env_contact_forces.argtypes = [vp, vp, vp, C.c_int]
        L.or_env_contact_bodies.argtypes = [vp, vp, vp, C.c_int]
        L.or_env_set_targets.argtypes = [vp, C.c_int, C.c_int, vp]
        L.or_env_friction_forces.argtypes = [vp, vp, vp, C.c_int]
        L.or_env_trace_get.argtypes = [vp, vp, C.c_int]
        L.or_env_body_mass.argtypes = [vp, C.c_int, vp, vp]
        L.or_env_soft_mass.argtypes = [vp, vp]
        L.or_neo_hookean.argtypes = [vp, d, d, vp, vp, vp, C.c_int]
        L.or_project_psd.argtypes = [C.c_int, vp]
        L.or_eigh.argtypes = [C.c_int, vp, vp, vp]
        L.or_barrier.argtypes = [d, d, vp]
        L.or_pair_dist2.restype = d
        L.or_pair_dist2.argtypes = [C.c_int, vp, vp, vp, vp]
        L.or_pair_dist2_typed.restype = d
        L.or_pair_dist2_typed.argtypes = [C.c_int, C.c_int, vp]
        L.or_pair_closest.argtypes = [C.c_int, vp, vp, vp]
        L.or_contact_barrier.restype = d
        L.or_contact_barrier.argtypes = [C.c_int, vp, d, d, d, vp, vp]
        L.or_mollifier.restype = d
        L.or_mollifier.argtypes = [vp, d]
        L.or_friction_f.argtypes = [d, d, vp]
        L.or_accd.restype = d
        L.or_accd.argtypes = [C.c_int, vp, vp, d, d, C.c_long, vp]
        L.or_mass_properties.argtypes = [C.c_int, vp, C.c_int, vp, d, vp, vp]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class _Params(C.Structure):
    _fields_ = [("dt", C.c_double), ("dhat", C.c_double), ("kappa", C.c_double), ("eps_v", C.c_double),
                ("newton_tol", C.c_double), ("pcg_rel_tol", C.c_double), ("kappa_affine", C.c_double),
                ("gravity", C.c_double * 3), ("max_newton", C.c_int32), ("max_ls", C.c_int32),
                ("max_pcg", C.c_int32), ("kappa_adapt", C.c_int32)]


class _Soft(C.Structure):
    _fields_ = [("n_verts", C.c_int32), ("n_tets", C.c_int32), ("n_tris", C.c_int32), ("pad", C.c_int32),
                ("verts", C.c_void_p), ("tets", C.c_void_p), ("tris", C.c_void_p), ("kin", C.c_void_p),
                ("E", C.c_double), ("nu", C.c_double), ("rho", C.c_double)]


class _Affine(C.Structure):
    _fields_ = [("n_verts", C.c_int32), ("n_tris", C.c_int32), ("kinematic", C.c_int32), ("pad", C.c_int32),
                ("verts", C.c_void_p), ("tris", C.c_void_p), ("rho", C.c_double),
                ("q0", C.c_double * 12), ("qdot0", C.c_double * 12), ("pd_stiffness", C.c_double)]


class _Joint(C.Structure):
    _fields_ = [("body_a", C.c_int32), ("body_b", C.c_int32), ("anchor_a", C.c_double * 3),
                ("anchor_b", C.c_double * 3), ("stiffness", C.c_double)]


class _Env(C.Structure):
    _fields_ = [("n_soft", C.c_int32), ("n_affine", C.c_int32), ("n_steps", C.c_int32), ("pad", C.c_int32),
                ("soft", C.c_void_p), ("affine", C.c_void_p), ("mu", C.c_double),
                ("gravity", C.c_void_p), ("targets", C.c_void_p), ("n_joints", C.c_int32), ("pad2", C.c_int32),
                ("joints", C.c_void_p)]


def _params_struct(p: dict) -> _Params:
    s = _Params()
    s.dt, s.dhat, s.kappa, s.eps_v = p["dt"], p["dhat"], p["kappa"], p["eps_v"]
    s.newton_tol, s.pcg_rel_tol, s.kappa_affine = p["newton_tol"], p["pcg_rel_tol"], p["kappa_affine"]
    for k in range(3):
        s.gravity[k] = p["gravity"][k]
    s.max_newton, s.max_ls, s.max_pcg = p["max_newton"], p["max_ls"], p["max_pcg"]
    s.kappa_adapt = int(bool(p.get("kappa_adapt", False)))
    return s


class OracleEnv:
    """One environment stepped by the CPU oracle."""

    STATUS = {0: "ACTIVE", 1: "DONE", 2: "FAILED"}

    def __init__(self, params: dict, env: dict):
        L = lib()
        self._keep = []
        soft = (_Soft * max(len(env["soft"]), 1))()
        for i, s in enumerate(env["soft"]):
            v = np.ascontiguousarray(s["verts"], dtype=np.float64)
            t = np.ascontiguousarray(s["tets"], dtype=np.int32)
            f = np.ascontiguousarray(s["tris"], dtype=np.int32)
            k = np.ascontiguousarray(s["kin"], dtype=np.uint8)
            self._keep += [v, t, f, k]
            soft[i].n_verts, soft[i].n_tets, soft[i].n_tris = len(v), len(t), len(f)
            soft[i].verts, soft[i].tets, soft[i].tris, soft[i].kin = v.ctypes.data, t.ctypes.data, f.ctypes.data, k.ctypes.data
            soft[i].E, soft[i].nu, soft[i].rho = s["E"], s["nu"], s["rho"]
        aff = (_Affine * max(len(env["affine"]), 1))()
        for i, a in enumerate(env["affine"]):
            v = np.ascontiguousarray(a["verts"], dtype=np.float64)
            f = np.ascontiguousarray(a["tris"], dtype=np.int32)
            self._keep += [v, f]
            aff[i].n_verts, aff[i].n_tris, aff[i].kinematic = len(v), len(f), int(bool(a["kinematic"]))
            aff[i].verts, aff[i].tris, aff[i].rho = v.ctypes.data, f.ctypes.data, a["rho"]
            for k in range(12):
                aff[i].q0[k] = a["q0"][k]
                aff[i].qdot0[k] = a["qdot0"][k]
            aff[i].pd_stiffness = float(a.get("pd", 0.0))
        g = np.ascontiguousarray(env["gravity"], dtype=np.uint8)
        tg = np.ascontiguousarray(env["targets"], dtype=np.float64)
        self._keep += [g, tg, soft, aff]
        d = _Env()
        d.n_soft, d.n_affine, d.n_steps = len(env["soft"]), len(env["affine"]), len(g)
        d.soft, d.affine = C.addressof(soft), C.addressof(aff)
        d.mu, d.gravity, d.targets = env["mu"], g.ctypes.data, tg.ctypes.data
        js = env.get("joints", [])
        jt = (_Joint * max(len(js), 1))()
        for i, j in enumerate(js):
            jt[i].body_a, jt[i].body_b, jt[i].stiffness = int(j["a"]), int(j["b"]), float(j["k"])
            for k in range(3):
                jt[i].anchor_a[k], jt[i].anchor_b[k] = j["anchor_a"][k], j["anchor_b"][k]
        self._keep.append(jt)
        d.n_joints, d.joints = len(js), C.addressof(jt)
        ps = _params_struct(params)
        self.params = dict(params)
        self.h = L.or_env_create(C.byref(ps), C.byref(d))
        self.ndof = L.or_env_ndof(self.h)
        self.npoints = L.or_env_npoints(self.h)

    def __del__(self):
        if getattr(self, "h", None):
            lib().or_env_destroy(self.h)
            self.h = None

    def step(self, n: int = 1) -> str:
        return self.STATUS[lib().or_env_step(self.h, n)]

    def state(self):
        x = np.zeros(self.ndof)
        v = np.zeros(self.ndof)
        lib().or_env_get_state(self.h, _p(x), _p(v))
        return x, v

    def set_state(self, x, v, step: int):
        x = np.ascontiguousarray(x, dtype=np.float64)
        v = np.ascontiguousarray(v, dtype=np.float64)
        lib().or_env_set_state(self.h, _p(x), _p(v), step)

    def tet_stress(self, q, n_tets: int) -> np.ndarray:
        """Von Mises stress of every tet (Pa) at DOFs q."""
        q = np.ascontiguousarray(q, dtype=np.float64)
        out = np.zeros(n_tets)
        lib().or_env_tet_stress(self.h, _p(q), _p(out))
        return out

    def contact_forces(self, q) -> np.ndarray:
        """Normal force (N) of every contact at DOFs q, in the order of contacts(q)."""
        q = np.ascontiguousarray(q, dtype=np.float64)
        n = lib().or_env_contact_forces(self.h, _p(q), None, 0)
        out = np.zeros(max(n, 1))
        lib().or_env_contact_forces(self.h, _p(q), _p(out), n)
        return out[:n]

    def contact_bodies(self, q) -> np.ndarray:
        """Body handles (soft bodies first, then affine) of the two sides of every contact at q,
        in the order of contacts(q)."""
        q = np.ascontiguousarray(q, dtype=np.float64)
        n = lib().or_env_contact_bodies(self.h, _p(q), None, 0)
        out = np.zeros((max(n, 1), 2), dtype=np.int32)
        lib().or_env_contact_bodies(self.h, _p(q), _p(out), n)
        return out[:n]

    def set_targets(self, first_step: int, targets) -> None:
        """Rewrite the schedule rows first_step .. first_step + len(targets) - 1."""
        t = np.ascontiguousarray(targets, dtype=np.float64)
        lib().or_env_set_targets(self.h, first_step, len(t), _p(t))

    def friction_forces(self, q) -> np.ndarray:
        """Tangential force (N) of every lagged friction stencil of the last step at DOFs q."""
        q = np.ascontiguousarray(q, dtype=np.float64)
        n = lib().or_env_friction_forces(self.h, _p(q), None, 0)
        out = np.zeros(max(n, 1))
        lib().or_env_friction_forces(self.h, _p(q), _p(out), n)
        return out[:n]

    def kappa(self) -> float:
        """Barrier stiffness of the current (or last) step."""
        return float(lib().or_env_kappa(self.h))

    def status(self) -> dict:
        st = np.zeros(4, dtype=np.int32)
        stats = np.zeros(4, dtype=np.int64)
        a = C.c_double()
        lib().or_env_status(self.h, _p(st), _p(stats), C.byref(a))
        return dict(status=self.STATUS[int(st[0])], reason=int(st[1]), steps_done=int(st[2]), step=int(st[3]),
                    newton_iters=int(stats[0]), ls_halvings=int(stats[1]), cg_iters=int(stats[2]),
                    accd_iters=int(stats[3]), last_alpha=a.value)

    def eval(self, q, grad: bool = True):
        q = np.ascontiguousarray(q, dtype=np.float64)
        g = np.zeros(self.ndof) if grad else None
        E = lib().or_env_eval(self.h, _p(q), _p(g) if grad else None)
        return (E, g) if grad else E

    def newton_direction(self) -> np.ndarray:
        """First Newton direction of the next step at the current state."""
        out = np.zeros(self.ndof)
        lib().or_env_newton_dir(self.h, _p(out))
        return out

    def hessian(self, q) -> np.ndarray:
        q = np.ascontiguousarray(q, dtype=np.float64)
        H = np.zeros((self.ndof, self.ndof))
        lib().or_env_hessian(self.h, _p(q), _p(H))
        return H

    def candidates(self, q, p=None) -> np.ndarray:
        q = np.ascontiguousarray(q, dtype=np.float64)
        pp = None if p is None else np.ascontiguousarray(p, dtype=np.float64)
        n = lib().or_env_candidates(self.h, _p(q), None if pp is None else _p(pp), None, 0)
        out = np.zeros((max(n, 1), 3), dtype=np.int32)
        lib().or_env_candidates(self.h, _p(q), None if pp is None else _p(pp), _p(out), n)
        return out[:n]

    def contacts(self, q):
        q = np.ascontiguousarray(q, dtype=np.float64)
        n = lib().or_env_contacts(self.h, _p(q), None, None, 0)
        out = np.zeros((max(n, 1), 4), dtype=np.int32)
        d2 = np.zeros(max(n, 1))
        lib().or_env_contacts(self.h, _p(q), _p(out), _p(d2), n)
        return out[:n], d2[:n]

    def points(self, q) -> np.ndarray:
        q = np.ascontiguousarray(q, dtype=np.float64)
        out = np.zeros((self.npoints, 3))
        lib().or_env_points(self.h, _p(q), _p(out))
        return out

    def invariants(self, q) -> dict:
        q = np.ascontiguousarray(q, dtype=np.float64)
        out = np.zeros(3)
        lib().or_env_invariants(self.h, _p(q), _p(out))
        return dict(intersections=int(out[0]), inverted=int(out[1]), min_dist=float(out[2]))

    def trace(self, on: bool = True):
        lib().or_env_trace(self.h, int(on))

    def trace_energies(self) -> np.ndarray:
        """Rows (step, newton iteration, constrained phase 0/1, energy at the iterate)."""
        n = lib().or_env_trace_get(self.h, None, 0)
        out = np.zeros(max(n, 4))
        lib().or_env_trace_get(self.h, _p(out), n)
        return out[:n].reshape(-1, 4)

    def body_mass(self, b: int):
        M = np.zeros(16)
        v = C.c_double()
        lib().or_env_body_mass(self.h, b, _p(M), C.byref(v))
        return M.reshape(4, 4), v.value

    def soft_mass(self, n_soft_verts: int) -> np.ndarray:
        out = np.zeros(n_soft_verts)
        lib().or_env_soft_mass(self.h, _p(out))
        return out


def run_batch(envs: list, n_steps: int, n_threads: int):
    """Step several OracleEnv objects on n_threads host threads."""
    arr = (C.c_void_p * len(envs))(*[e.h for e in envs])
    lib().or_run_batch(arr, len(envs), n_steps, n_threads)


# ----------------------------------------------------------------- element-level helpers
def neo_hookean(F, mu, lam, project=False):
    F = np.ascontiguousarray(F, dtype=np.float64).reshape(9)
    psi = C.c_double()
    P = np.zeros(9)
    H = np.zeros(81)
    lib().or_neo_hookean(_p(F), mu, lam, C.byref(psi), _p(P), _p(H), int(project))
    return psi.value, P, H.reshape(9, 9)


def project_psd(A):
    A = np.ascontiguousarray(A, dtype=np.float64).copy()
    lib().or_project_psd(A.shape[0], _p(A))
    return A


def eigh(A):
    A = np.ascontiguousarray(A, dtype=np.float64)
    n = A.shape[0]
    w = np.zeros(n)
    V = np.zeros((n, n))
    lib().or_eigh(n, _p(A), _p(w), _p(V))
    return w, V


def barrier(d, dhat):
    out = np.zeros(3)
    lib().or_barrier(d, dhat, _p(out))
    return out


def pair_dist2(kind, x12):
    x = np.ascontiguousarray(x12, dtype=np.float64).reshape(12)
    t = C.c_int()
    g = np.zeros(12)
    H = np.zeros(144)
    d2 = lib().or_pair_dist2(kind, _p(x), C.byref(t), _p(g), _p(H))
    return d2, t.value, g, H.reshape(12, 12)


def pair_dist2_typed(kind, type_, x12):
    x = np.ascontiguousarray(x12, dtype=np.float64).reshape(12)
    return lib().or_pair_dist2_typed(kind, type_, _p(x))


def pair_closest(kind, x12):
    x = np.ascontiguousarray(x12, dtype=np.float64).reshape(12)
    c = np.zeros(4)
    n = np.zeros(3)
    lib().or_pair_closest(kind, _p(x), _p(c), _p(n))
    return c, n


def contact_barrier(kind, x12, dhat, kappa, eps_x=0.0):
    x = np.ascontiguousarray(x12, dtype=np.float64).reshape(12)
    g = np.zeros(12)
    H = np.zeros(144)
    E = lib().or_contact_barrier(kind, _p(x), dhat, kappa, eps_x, _p(g), _p(H))
    return E, g, H.reshape(12, 12)


def mollifier(x12, eps):
    x = np.ascontiguousarray(x12, dtype=np.float64).reshape(12)
    return lib().or_mollifier(_p(x), eps)


def friction_f(y, eh):
    out = np.zeros(3)
    lib().or_friction_f(y, eh, _p(out))
    return out


def accd(kind, x12, p12, s=0.1, t_c=1.0, max_iter=1_000_000):
    x = np.ascontiguousarray(x12, dtype=np.float64).reshape(12)
    p = np.ascontiguousarray(p12, dtype=np.float64).reshape(12)
    it = C.c_long()
    t = lib().or_accd(kind, _p(x), _p(p), s, t_c, max_iter, C.byref(it))
    return t, it.value


def mass_properties(verts, tris, rho):
    v = np.ascontiguousarray(verts, dtype=np.float64)
    t = np.ascontiguousarray(tris, dtype=np.int32)
    M = np.zeros(16)
    vol = C.c_double()
    lib().or_mass_properties(len(v), _p(v), len(t), _p(t), rho, _p(M), C.byref(vol))
    return M.reshape(4, 4), vol.value
