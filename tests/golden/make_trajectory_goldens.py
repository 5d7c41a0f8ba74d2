"""Writes the oracle trajectories that the 100-step GPU parity tests compare against.

Each case steps one seeded grasp environment on the plain FP64 CPU oracle for 100 steps or more
in the parity settings (Newton tolerance x1e-3, CG to 1e-12), from the contact-phase start state
its schedule reaches at step 20 (the pad grasp and the hand: from their open grippers at step 0),
and stores a sample of its DOFs every 20 steps. The pad grasp's window stops at the end of its
closing: at this tolerance the oracle's Newton loop reaches its iteration cap at the first
lifting step, its line search halving the step down to 3e-11. One oracle step of
these scenes takes seconds to tens of seconds, so a test that reran the oracle for 100 steps
would take most of an hour; the GPU side of the test runs the same 100 steps live and compares
with these values. Only `oracle/` and the seeded scene generators are called here: no value
comes from the CUDA path.

Cases marked with the configuration's own settings are not parity windows: they run a whole
grasp schedule (closing, then lifting under gravity) as the configuration states it, to show
that the oracle itself holds and lifts the object; CPU tests check the stored outcome.

Usage: python tests/golden/make_trajectory_goldens.py [case ...]   (default: every case; each
case runs in its own process)
"""
from __future__ import annotations

import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2503_05020_b300 import scenes as S  # noqa: E402

START_STEP = 20
N_STEPS = 100
DT = 0.005  # every case below steps at 5 ms
EVERY = 20
SAMPLED_SOFT_VERTS = 240  # soft vertices kept per checkpoint (evenly strided), all affine DOFs


def _params(dhat=None, parity=True):
    p = S.scene_params(DT)
    if dhat is not None:
        p["dhat"] = dhat
    return S.parity_params(p) if parity else p


PARITY_SETTINGS = "parity settings (Newton tolerance x1e-3, CG to 1e-12)"
CONFIG_SETTINGS = "the configuration's settings (Newton tolerance 1e-2 dt in m/s; the oracle's CG to 1e-12)"


# case name -> recipe text, env builder, parameters, first step, steps (checkpoints every EVERY)
CASES = {
    "pad_grasp_0": dict(
        scene="scenes.pad_grasp_env(0): two ~5k-tet soft pads around a rigid 1584-triangle hull (the 64-env "
              "pad configuration's env 0), dt 5 ms, the 100 closing steps (gravity off) from the open pads",
        build=lambda: S.pad_grasp_env(0), params=lambda: _params(), start=0, steps=N_STEPS),
    "uneven_8": dict(
        scene="scenes.uneven_batch_env(8): a 2.3k-tet star-shaped soft object between two pairs of kinematic "
              "plates (the uneven batch's env 8), dt 5 ms, from the step-20 contact state",
        build=lambda: S.uneven_batch_env(8), params=lambda: _params(), start=START_STEP, steps=N_STEPS),
    "uneven_22": dict(
        scene="scenes.uneven_batch_env(22): a 4.4k-tet star-shaped soft object between one pair of kinematic "
              "plates (the uneven batch's env 22), dt 5 ms, from the step-20 contact state",
        build=lambda: S.uneven_batch_env(22), params=lambda: _params(), start=START_STEP, steps=N_STEPS),
    "hand_0": dict(
        scene="scenes.hand_grasp_env(0, n_steps=300, close_steps=200): 20 hinged PD-driven affine links "
              "curling onto a ~22k-tet star-shaped soft object, dhat 5e-4 m, dt 5 ms, from the open hand "
              "(step 0) through the first 200 steps of the closing",
        build=lambda: S.hand_grasp_env(0, n_steps=300, close_steps=200), params=lambda: _params(5e-4),
        start=0, steps=200),
    # not a parity case: the hand's whole grasp in the configuration's own settings, to show that
    # the oracle itself closes, holds and lifts the object (its schedule ends with the window)
    "hand_0_hold": dict(
        scene="scenes.hand_grasp_env(0, n_steps=300, close_steps=200): the same hinged hand and object, all "
              "300 steps: close 200 (gravity off), then palm and finger targets rise 5 cm in 100 (gravity on)",
        build=lambda: S.hand_grasp_env(0, n_steps=300, close_steps=200), params=lambda: _params(5e-4, parity=False),
        start=0, steps=300, final="DONE", settings=CONFIG_SETTINGS),
    # not a parity case: the pad configuration's env 0 as configured, closing and lifting, to show
    # that the oracle itself holds and lifts the hull (its schedule ends with the window)
    "pad_grasp_0_lift": dict(
        scene="scenes.pad_grasp_env(0): the pad configuration's env 0 through its whole schedule: close 100 "
              "steps (gravity off), then lift 0.1 m in 200 (gravity on), dt 5 ms, from the open pads",
        build=lambda: S.pad_grasp_env(0), params=lambda: _params(parity=False),
        start=0, steps=300, final="DONE", settings=CONFIG_SETTINGS),
    # not a parity case: a soft-pad grasp of a soft object from the uneven batch as configured
    "uneven_4_lift": dict(
        scene="scenes.uneven_batch_env(4): two ~4.8k-tet soft pads around a 3.3k-tet star-shaped soft object "
              "(the uneven batch's env 4), its whole schedule from the open pads: close 100 steps (gravity off), "
              "then lift 0.1 m in 200 (gravity on), dt 5 ms",
        build=lambda: S.uneven_batch_env(4), params=lambda: _params(parity=False),
        start=0, steps=300, final="DONE", settings=CONFIG_SETTINGS),
}


def fingerprint(obj) -> str:
    """sha256 of a scene description or parameter dict (keys sorted, arrays by dtype, shape and
    bytes): a test refuses a golden whose inputs no longer match the generators."""
    h = hashlib.sha256()

    def feed(o):
        if isinstance(o, dict):
            h.update(b"{")
            for k in sorted(o):
                h.update(repr(k).encode())
                feed(o[k])
            h.update(b"}")
        elif isinstance(o, (list, tuple)):
            h.update(b"[")
            for v in o:
                feed(v)
            h.update(b"]")
        elif isinstance(o, np.ndarray):
            a = np.ascontiguousarray(o)
            h.update(str(a.dtype).encode() + repr(a.shape).encode())
            h.update(a.tobytes())
        elif isinstance(o, (bool, int, float, str, np.integer, np.floating)) or o is None:
            h.update(repr(type(o).__name__).encode() + repr(o).encode())
        else:
            raise TypeError(f"cannot fingerprint {type(o)}")

    feed(obj)
    return h.hexdigest()


def sampled_dof_indices(env: dict) -> np.ndarray:
    """DOF indices kept per checkpoint: x, y, z of evenly strided soft vertices (every body's
    first and last vertex included) and the 12 coordinates of every affine body."""
    idx = []
    off = 0
    n_soft = sum(len(s["verts"]) for s in env["soft"])
    stride = max(1, n_soft // SAMPLED_SOFT_VERTS)
    for s in env["soft"]:
        n = len(s["verts"])
        vs = sorted(set(range(0, n, stride)) | {n - 1})
        for v in vs:
            idx.extend(3 * (off + v) + c for c in range(3))
        off += n
    base = 3 * off
    idx.extend(range(base, base + 12 * len(env["affine"])))
    return np.array(idx, dtype=np.int64)


def golden_path(case: str) -> str:
    return os.path.join(HERE, f"traj100_{case}.json")


def make(case: str) -> str:
    from oracle import oracle as O

    c = CASES[case]
    env = c["build"]()
    params = c["params"]()
    start, n_steps = c["start"], c["steps"]
    x0, v0 = S.grasp_state_at(env, start)
    idx = sampled_dof_indices(env)
    o = O.OracleEnv(params, env)
    o.set_state(x0, v0, start)
    checkpoints = []
    t0 = time.perf_counter()
    for k in range(EVERY, n_steps + 1, EVERY):
        o.step(EVERY)
        x, _ = o.state()
        checkpoints.append({"steps": k, "dofs": [float(v) for v in x[idx]]})
        st = o.status()
        print(f"{case}: step {start + k} {st} ({time.perf_counter() - t0:.0f} s)", flush=True)
    out = {
        "what": "plain FP64 CPU oracle trajectory (oracle/ipc_oracle.cpp), sampled DOFs every "
                f"{EVERY} steps; written by tests/golden/make_trajectory_goldens.py",
        "method": "IPC step of Sec. II-C with the per-environment solve of Sec. III-A, "
                  + c.get("settings", PARITY_SETTINGS),
        "scene": c["scene"],
        "params": {k: (list(v) if isinstance(v, tuple) else v) for k, v in params.items()},
        "start_step": start,
        "n_steps": n_steps,
        "env_fingerprint": fingerprint(env),
        "params_fingerprint": fingerprint(params),
        "start_fingerprint": fingerprint([x0, v0]),
        "dof_indices": [int(i) for i in idx],
        "checkpoints": checkpoints,
        "final_status": o.status(),
    }
    with open(golden_path(case) + ".tmp", "w") as f:
        json.dump(out, f, indent=0, separators=(",", ":"))
        f.write("\n")
    os.replace(golden_path(case) + ".tmp", golden_path(case))
    return golden_path(case)


if __name__ == "__main__":
    names = sys.argv[1:] or list(CASES)
    with mp.get_context("spawn").Pool(len(names)) as pool:
        for p in pool.imap_unordered(make, names):
            print("wrote", p, flush=True)
