"""Python binding of the C ABI in include/ipc.h (argument marshalling only).

Every numerical step runs in the sm_103a kernels of libipc_b300.so. Loading fails loudly when
the library is missing; there is no CPU path.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libipc_b300.so")
HEADER = os.path.join(HERE, "..", "include", "ipc.h")

STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_OOM", 3: "ERR_BUDGET", 4: "ERR_CUDA", 5: "ERR_INIT_INTERSECT",
                6: "ERR_INIT_INVERTED", 7: "ERR_NO_ENV", 8: "ERR_INTERNAL"}
STATUS_CODES = {v: k for k, v in STATUS_NAMES.items()}
ENV_STATUS = {0: "ACTIVE", 1: "DONE", 2: "FAILED"}
FAIL_REASON = {0: "none", 1: "newton_cap", 2: "line_search", 3: "non_finite", 4: "initial_intersection", 5: "internal"}
FP64, MIXED = 0, 1
Q_DOFS, Q_VELOCITIES, Q_STATUS, Q_STATS, Q_CANDIDATES, Q_CONTACTS, Q_POINTS, Q_SIZES, Q_INTERSECTIONS, \
    Q_SCENE_COUNTERS, Q_ALL_STATUS, Q_KAPPA, Q_TET_STRESS, Q_CONTACT_FORCES, Q_FRICTION_FORCES, \
    Q_CONTACT_HANDLES, Q_ENERGY_TRACE, Q_GRASP_RESULT = range(18)


class IpcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class SceneDesc(C.Structure):
    _fields_ = [("dt", C.c_double), ("dhat", C.c_double), ("kappa", C.c_double), ("eps_v", C.c_double),
                ("newton_tol", C.c_double), ("pcg_rel_tol", C.c_double), ("kappa_affine", C.c_double),
                ("gravity", C.c_double * 3), ("max_newton", C.c_int32), ("max_ls_halvings", C.c_int32),
                ("max_pcg_iters", C.c_int32), ("precision", C.c_int32), ("hbm_budget_bytes", C.c_uint64),
                ("device", C.c_int32), ("pcg_cluster", C.c_int32), ("fresh_broad_phase", C.c_int32),
                ("kappa_adapt", C.c_int32), ("cuda_stream", C.c_void_p), ("collect_slots", C.c_int32)]


class SoftDesc(C.Structure):
    _fields_ = [("n_verts", C.c_int32), ("n_tets", C.c_int32), ("n_tris", C.c_int32), ("pad", C.c_int32),
                ("verts", C.c_void_p), ("tets", C.c_void_p), ("tris", C.c_void_p), ("kinematic", C.c_void_p),
                ("youngs", C.c_double), ("poisson", C.c_double), ("density", C.c_double)]


class AffineDesc(C.Structure):
    _fields_ = [("n_verts", C.c_int32), ("n_tris", C.c_int32), ("kinematic", C.c_int32), ("pad", C.c_int32),
                ("verts", C.c_void_p), ("tris", C.c_void_p), ("density", C.c_double),
                ("q0", C.c_double * 12), ("qdot0", C.c_double * 12), ("pd_stiffness", C.c_double)]


class JointDesc(C.Structure):
    _fields_ = [("body_a", C.c_int32), ("body_b", C.c_int32), ("anchor_a", C.c_double * 3),
                ("anchor_b", C.c_double * 3), ("stiffness", C.c_double)]


class EnvDesc(C.Structure):
    _fields_ = [("n_soft", C.c_int32), ("n_affine", C.c_int32), ("n_steps", C.c_int32), ("pad", C.c_int32),
                ("soft", C.c_void_p), ("affine", C.c_void_p), ("friction_mu", C.c_double),
                ("gravity_on", C.c_void_p), ("targets", C.c_void_p), ("n_joints", C.c_int32), ("pad2", C.c_int32),
                ("joints", C.c_void_p), ("grasped_object", C.c_int32), ("pad3", C.c_int32)]


_lib = None


def declared_functions() -> list[str]:
    """Names of the functions declared in include/ipc.h."""
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:ipc_status|const char\*)\s+(ipc_\w+)\s*\(", src, flags=re.M)))


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libipc_b300.so not built ({LIB_PATH}); run paper_2503_05020_b300/build.py")
        L = C.CDLL(LIB_PATH)
        vp, i32, sz = C.c_void_p, C.c_int32, C.c_size_t
        L.ipc_last_error.restype = C.c_char_p
        L.ipc_version.restype = C.c_char_p
        sigs = {
            "ipc_scene_create": [vp, vp], "ipc_scene_destroy": [vp], "ipc_env_add": [vp, vp, vp],
            "ipc_env_remove": [vp, i32], "ipc_step": [vp, i32], "ipc_query": [vp, i32, i32, vp, sz, vp],
            "ipc_env_set_state": [vp, i32, vp, vp, i32], "ipc_eval": [vp, i32, vp, vp, vp],
            "ipc_newton_direction": [vp, i32, vp], "ipc_hessian_apply": [vp, i32, vp, vp],
            "ipc_set_next_targets": [vp, vp, sz], "ipc_get_all_dofs": [vp, vp, sz, vp],
            "ipc_env_set_targets": [vp, i32, i32, i32, vp],
            "ipc_env_estimate_bytes": [vp, i32, vp], "ipc_launch_count": [vp, vp],
            "ipc_profile_enable": [vp, i32], "ipc_profile_read": [vp, i32, vp, vp, vp],
            "ipc_elastic_energy_noalloc": [i32, vp, vp, vp, i32, vp, C.c_double, vp, vp, vp],
        }
        for name, args in sigs.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        _lib = L
    return _lib


def _check(st: int):
    if st != 0:
        raise IpcError(st, lib().ipc_last_error().decode())


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class _EnvMarshal:
    """Keeps the numpy arrays of one env descriptor alive while the C call copies them."""

    def __init__(self, env: dict):
        self.keep = []
        soft = (SoftDesc * max(len(env["soft"]), 1))()
        for i, s in enumerate(env["soft"]):
            v = np.ascontiguousarray(s["verts"], dtype=np.float64)
            t = np.ascontiguousarray(s["tets"], dtype=np.int32)
            f = np.ascontiguousarray(s["tris"], dtype=np.int32)
            k = np.ascontiguousarray(s.get("kin", np.zeros(len(v))), dtype=np.uint8)
            self.keep += [v, t, f, k]
            soft[i].n_verts, soft[i].n_tets, soft[i].n_tris = len(v), len(t), len(f)
            soft[i].verts, soft[i].tets, soft[i].tris, soft[i].kinematic = v.ctypes.data, t.ctypes.data, f.ctypes.data, k.ctypes.data
            soft[i].youngs, soft[i].poisson, soft[i].density = s["E"], s["nu"], s["rho"]
        aff = (AffineDesc * max(len(env["affine"]), 1))()
        for i, a in enumerate(env["affine"]):
            v = np.ascontiguousarray(a["verts"], dtype=np.float64)
            f = np.ascontiguousarray(a["tris"], dtype=np.int32)
            self.keep += [v, f]
            aff[i].n_verts, aff[i].n_tris, aff[i].kinematic = len(v), len(f), int(bool(a["kinematic"]))
            aff[i].verts, aff[i].tris, aff[i].density = v.ctypes.data, f.ctypes.data, a["rho"]
            for k in range(12):
                aff[i].q0[k] = a["q0"][k]
                aff[i].qdot0[k] = a["qdot0"][k]
            aff[i].pd_stiffness = float(a.get("pd", 0.0))
        g = np.ascontiguousarray(env["gravity"], dtype=np.uint8)
        tg = np.ascontiguousarray(env["targets"], dtype=np.float64)
        self.keep += [g, tg, soft, aff]
        d = EnvDesc()
        d.n_soft, d.n_affine, d.n_steps = len(env["soft"]), len(env["affine"]), len(g)
        d.soft, d.affine = C.addressof(soft), C.addressof(aff)
        d.friction_mu, d.gravity_on, d.targets = env["mu"], g.ctypes.data, tg.ctypes.data
        js = env.get("joints", [])
        jt = (JointDesc * max(len(js), 1))()
        for i, j in enumerate(js):
            jt[i].body_a, jt[i].body_b, jt[i].stiffness = int(j["a"]), int(j["b"]), float(j["k"])
            for k in range(3):
                jt[i].anchor_a[k], jt[i].anchor_b[k] = j["anchor_a"][k], j["anchor_b"][k]
        self.keep.append(jt)
        d.n_joints, d.joints = len(js), C.addressof(jt)
        if "object" in env:  # 1 + the object's handle (soft bodies first, then affine bodies)
            kind, k = env["object"]
            d.grasped_object = 1 + (k if kind == "soft" else len(env["soft"]) + k)
        self.desc = d


def estimate_bytes(env: dict, precision: int = FP64) -> int:
    m = _EnvMarshal(env)
    out = C.c_uint64()
    _check(lib().ipc_env_estimate_bytes(C.byref(m.desc), precision, C.byref(out)))
    return out.value


class Scene:
    """A batch of grasp environments stepped together on one GPU."""

    def __init__(self, params: dict, precision: int = FP64, device: int = 0, stream: int | None = None,
                 hbm_budget_bytes: int = 0, pcg_cluster: int = 0, fresh_broad_phase: bool = False,
                 collect_slots: int = 0):
        d = SceneDesc()
        d.dt, d.dhat, d.kappa, d.eps_v = params["dt"], params["dhat"], params["kappa"], params["eps_v"]
        d.newton_tol, d.pcg_rel_tol, d.kappa_affine = params["newton_tol"], params["pcg_rel_tol"], params["kappa_affine"]
        for k in range(3):
            d.gravity[k] = params["gravity"][k]
        d.max_newton, d.max_ls_halvings, d.max_pcg_iters = params["max_newton"], params["max_ls"], params["max_pcg"]
        d.precision, d.hbm_budget_bytes, d.device = precision, hbm_budget_bytes, device
        d.pcg_cluster = pcg_cluster  # 0 automatic, 1/2/4/8/16 CTAs per env cluster, -1 tiled multi-launch
        d.fresh_broad_phase = int(bool(fresh_broad_phase))  # 1: a BVH traversal at every evaluation
        d.kappa_adapt = int(bool(params.get("kappa_adapt", False)))  # 1: adapted barrier stiffness per env
        d.cuda_stream = stream
        d.collect_slots = collect_slots  # partner slots per collect-traversal query (0: 128)
        self._h = C.c_void_p()
        _check(lib().ipc_scene_create(C.byref(d), C.byref(self._h)))
        self.params = dict(params)
        self.ndof = {}

    def close(self):
        if self._h:
            _check(lib().ipc_scene_destroy(self._h))
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_env(self, env: dict) -> int:
        m = _EnvMarshal(env)
        eid = C.c_int32()
        _check(lib().ipc_env_add(self._h, C.byref(m.desc), C.byref(eid)))
        self.ndof[eid.value] = 3 * sum(len(s["verts"]) for s in env["soft"]) + 12 * len(env["affine"])
        return eid.value

    def remove_env(self, eid: int):
        _check(lib().ipc_env_remove(self._h, eid))
        self.ndof.pop(eid, None)

    def step(self, n: int = 1):
        _check(lib().ipc_step(self._h, n))

    def _query(self, eid: int, kind: int, dtype, cols: int | None = None) -> np.ndarray:
        need = C.c_size_t()
        st = lib().ipc_query(self._h, eid, kind, None, 0, C.byref(need))
        if st not in (0, 1):
            _check(st)
        buf = np.zeros(max(need.value, 8) // np.dtype(dtype).itemsize, dtype=dtype)
        _check(lib().ipc_query(self._h, eid, kind, _p(buf), buf.nbytes, C.byref(need)))
        out = buf[: need.value // np.dtype(dtype).itemsize]
        return out.reshape(-1, cols) if cols else out

    def dofs(self, eid: int) -> np.ndarray:
        return self._query(eid, Q_DOFS, np.float64)

    def velocities(self, eid: int) -> np.ndarray:
        return self._query(eid, Q_VELOCITIES, np.float64)

    def status(self, eid: int) -> dict:
        v = self._query(eid, Q_STATUS, np.int32)
        s = self._query(eid, Q_STATS, np.int64)
        return dict(status=ENV_STATUS[int(v[0])], reason=FAIL_REASON.get(int(v[1]), int(v[1])), steps_done=int(v[2]),
                    step=int(v[3]), newton_iters=int(s[0]), pcg_iters=int(s[1]), ls_halvings=int(s[2]),
                    steps=int(s[3]), accd_iters=int(s[4]))

    def candidates(self, eid: int) -> np.ndarray:
        return self._query(eid, Q_CANDIDATES, np.int32, 3)

    def contacts(self, eid: int) -> np.ndarray:
        return self._query(eid, Q_CONTACTS, np.int32, 4)

    def points(self, eid: int) -> np.ndarray:
        return self._query(eid, Q_POINTS, np.float64, 3)

    def sizes(self, eid: int) -> dict:
        v = self._query(eid, Q_SIZES, np.int64)
        return dict(zip(["ndof", "points", "surface_verts", "edges", "tris", "tets", "bodies", "steps"], map(int, v)))

    def scene_counters(self, eid: int) -> dict:
        v = self._query(eid, Q_SCENE_COUNTERS, np.int64)
        keys = ["contacts", "pt_contacts", "friction", "incidence_entries", "longest_list", "candidates",
                "bsr_blocks", "sell_blocks", "pcg_cluster", "max_env_slices", "joints", "collect_spills"]
        return dict(zip(keys, map(int, v)))

    def contact_forces(self, eid: int) -> np.ndarray:
        """Normal force (N) of each contact at the env's current DOFs, in the order of contacts()."""
        return self._query(eid, Q_CONTACT_FORCES, np.float64)

    def friction_forces(self, eid: int) -> np.ndarray:
        """Tangential force (N) of each lagged friction stencil of the env's last step at its
        current DOFs."""
        return self._query(eid, Q_FRICTION_FORCES, np.float64)

    def tet_stress(self, eid: int) -> np.ndarray:
        """Von Mises stress (Pa) of each of the env's tets at its current DOFs."""
        return self._query(eid, Q_TET_STRESS, np.float64)

    def grasp_result(self, eid: int) -> dict:
        """Sec. III-D outcome of an env that names its grasped object: contact, the centre of
        mass's motion over the last step (m), the stability label and the centre's rise (m)."""
        v = self._query(eid, Q_GRASP_RESULT, np.float64)
        return {"in_contact": bool(v[0]), "com_step": float(v[1]), "stable": bool(v[2]), "com_rise": float(v[3])}

    def energy_trace(self, eid: int) -> np.ndarray:
        """Incremental potential at each Newton iterate of the env's current (or last) step."""
        return self._query(eid, Q_ENERGY_TRACE, np.float64)

    def kappa(self, eid: int) -> float:
        """The env's barrier stiffness in its current (or last) step."""
        return float(self._query(eid, Q_KAPPA, np.float64)[0])

    def all_status(self) -> dict:
        """{env id: (status, reason, next step)} for every environment, in one read-back."""
        v = self._query(-1, Q_ALL_STATUS, np.int32, 4)
        return {int(r[0]): (ENV_STATUS[int(r[1])], FAIL_REASON.get(int(r[2]), int(r[2])), int(r[3])) for r in v}

    def invariants(self, eid: int) -> dict:
        v = self._query(eid, Q_INTERSECTIONS, np.int64)
        return dict(intersections=int(v[0]), inverted=int(v[1]))

    def set_state(self, eid: int, x, v, step: int):
        x = np.ascontiguousarray(x, dtype=np.float64)
        v = np.ascontiguousarray(v, dtype=np.float64)
        _check(lib().ipc_env_set_state(self._h, eid, _p(x), _p(v), step))

    def eval(self, eid: int, q, grad: bool = True):
        q = np.ascontiguousarray(q, dtype=np.float64)
        E = C.c_double()
        g = np.zeros(len(q)) if grad else None
        _check(lib().ipc_eval(self._h, eid, _p(q), C.byref(E), _p(g)))
        return (E.value, g) if grad else E.value

    def newton_direction(self, eid: int) -> np.ndarray:
        """First Newton direction of the env's next step at its current state (diagnostic)."""
        out = np.zeros(self.ndof[eid])
        _check(lib().ipc_newton_direction(self._h, eid, _p(out)))
        return out

    def hessian_apply(self, eid: int, d) -> np.ndarray:
        """y = H d with the projected Hessian as the PCG applies it (diagnostic)."""
        d = np.ascontiguousarray(d, dtype=np.float64)
        y = np.zeros_like(d)
        _check(lib().ipc_hessian_apply(self._h, eid, _p(d), _p(y)))
        return y

    def set_env_targets(self, eid: int, first_step: int, targets: np.ndarray):
        """Rewrite the env's schedule from first_step on with targets [n_steps][body][12]."""
        t = np.ascontiguousarray(targets, dtype=np.float64)
        _check(lib().ipc_env_set_targets(self._h, eid, first_step, t.shape[0], _p(t)))

    def contact_handles(self, eid: int) -> np.ndarray:
        """Bodies (soft first, then affine) of the two sides of each contact, in contacts() order."""
        return self._query(eid, Q_CONTACT_HANDLES, np.int32, 2)

    def set_next_targets(self, targets: np.ndarray):
        t = np.ascontiguousarray(targets, dtype=np.float64)
        _check(lib().ipc_set_next_targets(self._h, _p(t), t.nbytes))

    def all_dofs(self, out: np.ndarray) -> np.ndarray:
        w = C.c_size_t()
        _check(lib().ipc_get_all_dofs(self._h, _p(out), out.nbytes, C.byref(w)))
        return out

    def all_dofs_size(self) -> int:
        w = C.c_size_t()
        lib().ipc_get_all_dofs(self._h, None, 0, C.byref(w))
        return w.value // 8

    PROF_FAMILIES = ["spmv", "elastic", "contact", "ccd", "pcg_vector", "broad", "assembly", "ls_energy", "pcg_solve",
                     "pcg_flops", "host_idle"]

    def profile(self, on: bool = True):
        _check(lib().ipc_profile_enable(self._h, int(on)))

    def profile_read(self) -> dict:
        out = {}
        for i, name in enumerate(self.PROF_FAMILIES):
            n, ms, w = C.c_int64(), C.c_double(), C.c_double()
            _check(lib().ipc_profile_read(self._h, i, C.byref(n), C.byref(ms), C.byref(w)))
            out[name] = dict(launches=n.value, ms=ms.value, work=w.value)
        return out

    def launch_count(self) -> int:
        c = C.c_int64()
        _check(lib().ipc_launch_count(self._h, C.byref(c)))
        return c.value
