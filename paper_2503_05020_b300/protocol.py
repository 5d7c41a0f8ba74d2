"""Grasp evaluation protocol (Sec. III-D) on top of the library.

Gravity is off while the gripper closes; a finger stops once the contact force between it and
the object exceeds 50 N (its remaining targets are held where it stopped); after a settling
phase gravity acts in six axis-aligned directions, 9.8 m/s^2 for 0.1 s each (the scene's
gravity magnitude; codes 2..7 of the per-step gravity schedule). The grasp is stable when the
object still touches the gripper at the last step and its centre of mass moved less than a
threshold proportional to eps_v dt during that step.

Readings where the paper gives no number: the centre of mass is the mean of the object's
points (its vertices; for a rigid body they move with it), the threshold is
`stable_factor * eps_v * dt` with stable_factor = 1 (the object slower than the friction model's
static/dynamic transition speed), and a finger is a body whose targets drive it (for the pad
grasp, each soft pad). The loop is host code over the C ABI: each closing step is one ipc_step,
followed by the contact-force and contact-body queries.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

HALT_FORCE_N = 50.0
PHASE_SECONDS = 0.1
AXIS_CODES = (2, 3, 4, 5, 6, 7)  # +x, -x, +y, -y, +z, -z


def evaluation_env(env: dict, close_steps: int, settle_steps: int, dt: float) -> dict:
    """The env with the protocol's schedule: its own targets for the first close_steps steps
    (gravity off), then the last closing targets held for settle_steps steps (gravity off) and
    for six gravity phases of round(0.1 s / dt) steps each (axis codes 2..7)."""
    T = np.asarray(env["targets"], dtype=np.float64)
    if close_steps < 1 or close_steps > len(T):
        raise ValueError("close_steps must lie within the env's schedule")
    n_phase = max(1, int(round(PHASE_SECONDS / dt)))
    n_hold = settle_steps + len(AXIS_CODES) * n_phase
    targets = np.concatenate([T[:close_steps], np.repeat(T[close_steps - 1:close_steps], n_hold, axis=0)])
    gravity = np.concatenate([np.zeros(close_steps + settle_steps, dtype=np.uint8),
                              np.repeat(np.asarray(AXIS_CODES, dtype=np.uint8), n_phase)])
    return dict(env, targets=targets, gravity=gravity)


@dataclass
class Outcome:
    stable: bool
    in_contact: bool
    com_step: float                 # centre-of-mass movement over the last step (m)
    halted: dict = field(default_factory=dict)  # finger -> closing step after which it stopped
    peak_force: dict = field(default_factory=dict)  # finger -> largest contact force (N) seen


def _finger_forces(sc, eid: int, fingers, obj: int) -> dict:
    """Sum of the contact forces between each finger and the object (N)."""
    f = sc.contact_forces(eid)
    out = {k: 0.0 for k in fingers}
    if len(f) == 0:
        return out
    h = sc.contact_handles(eid)
    for (a, b), fk in zip(h, f):
        for k in fingers:
            if {int(a), int(b)} == {k, obj}:
                out[k] += float(fk)
    return out


def _com(points: np.ndarray, sl: slice) -> np.ndarray:
    return points[sl].mean(axis=0)


def evaluate_grasp(sc, eid: int, env: dict, fingers, obj: int, obj_points: slice, close_steps: int,
                   eps_v: float, dt: float, halt_force: float = HALT_FORCE_N, stable_factor: float = 1.0) -> Outcome:
    """Run one env (already added to scene sc with the schedule of evaluation_env) through the
    protocol and label the grasp. fingers: handles of the finger bodies; obj: the object's
    handle; obj_points: the object's rows in the env's point list."""
    targets = np.asarray(env["targets"], dtype=np.float64).copy()
    n_steps = len(targets)
    halted, peak = {}, {k: 0.0 for k in fingers}
    for s in range(close_steps):
        sc.step(1)
        forces = _finger_forces(sc, eid, fingers, obj)
        for k in fingers:
            peak[k] = max(peak[k], forces[k])
            if k not in halted and forces[k] > halt_force:
                halted[k] = s
                targets[s + 1:, k] = targets[s, k]  # the finger stays where it reached at step s
                if s + 1 < n_steps:
                    sc.set_env_targets(eid, s + 1, targets[s + 1:])
    rest = n_steps - close_steps
    if rest > 1:
        sc.step(rest - 1)
    before = _com(sc.points(eid), obj_points)
    if rest >= 1:
        sc.step(1)
    after = _com(sc.points(eid), obj_points)
    com_step = float(np.linalg.norm(after - before))
    h = sc.contact_handles(eid)
    in_contact = any({int(a), int(b)} & {obj} and ({int(a), int(b)} - {obj}) & set(fingers) for a, b in h)
    stable = in_contact and com_step < stable_factor * eps_v * dt
    return Outcome(stable, in_contact, com_step, halted, peak)
