"""Host logic of the grasp evaluation protocol (no GPU): the protocol's schedule (gravity off
while closing and settling, then the six axis phases of 0.1 s), a finger held where its
contact force with the object first exceeds 50 N, and the stability label."""
import numpy as np

from paper_2503_05020_b300 import protocol as P


def test_evaluation_schedule():
    T = np.arange(10 * 3 * 12, dtype=np.float64).reshape(10, 3, 12)
    env = dict(targets=T, gravity=np.ones(10, dtype=np.uint8), soft=[], affine=[])
    ev = P.evaluation_env(env, close_steps=4, settle_steps=3, dt=0.01)
    n_phase = 10
    assert len(ev["targets"]) == len(ev["gravity"]) == 4 + 3 + 6 * n_phase
    assert np.array_equal(ev["targets"][:4], T[:4])
    assert np.all(ev["targets"][4:] == T[3])
    assert np.all(ev["gravity"][:7] == 0)
    assert list(ev["gravity"][7::n_phase]) == [2, 3, 4, 5, 6, 7]


class FakeScene:
    """Finger 0 presses the object (handle 2) with 20 N more every step, finger 1 with 5 N; the
    object's points move by `drift` per step during the hold."""

    def __init__(self, n_steps, drift):
        self.step_no, self.n_steps, self.drift = 0, n_steps, drift
        self.rewrites = []

    def step(self, n=1):
        self.step_no += n

    def contact_forces(self, eid):
        return np.array([20.0 * self.step_no, 5.0 * self.step_no])

    def contact_handles(self, eid):
        return np.array([[0, 2], [2, 1]], dtype=np.int32)

    def set_env_targets(self, eid, first, targets):
        self.rewrites.append((first, np.array(targets)))

    def points(self, eid):
        return np.full((4, 3), self.drift * self.step_no)


def test_finger_halt_and_label():
    T = np.zeros((20, 3, 12))
    for s in range(20):
        T[s, 0, 0] = T[s, 1, 0] = s  # both fingers advance one unit per step
    env = dict(targets=T)
    sc = FakeScene(20, drift=1e-7)
    out = P.evaluate_grasp(sc, 0, env, fingers=[0, 1], obj=2, obj_points=slice(0, 4), close_steps=5,
                           eps_v=1e-3, dt=0.01)
    # finger 0 passes 50 N after the third step (60 N), finger 1 never (25 N at the end)
    assert out.halted == {0: 2}
    assert out.peak_force[0] == 100.0 and out.peak_force[1] == 25.0
    first, rows = sc.rewrites[0]
    assert first == 3 and np.all(rows[:, 0, 0] == 2) and np.array_equal(rows[:, 1, 0], np.arange(3, 20))
    assert out.in_contact and out.stable  # 1.7e-7 m per step < eps_v dt = 1e-5 m
    sc = FakeScene(20, drift=1e-4)
    out = P.evaluate_grasp(sc, 0, env, fingers=[0, 1], obj=2, obj_points=slice(0, 4), close_steps=5,
                           eps_v=1e-3, dt=0.01)
    assert out.in_contact and not out.stable


class RateScene(FakeScene):
    """FakeScene with chosen per-step force rates and contact pairs."""

    def __init__(self, n_steps, drift, rates, handles):
        super().__init__(n_steps, drift)
        self.rates, self.handles = rates, np.asarray(handles, dtype=np.int32)

    def contact_forces(self, eid):
        return np.array([r * self.step_no for r in self.rates])

    def contact_handles(self, eid):
        return self.handles


def _run(sc, close_steps=5):
    T = np.zeros((20, 4, 12))
    return P.evaluate_grasp(sc, 0, dict(targets=T), fingers=[0, 1], obj=2, obj_points=slice(0, 4),
                            close_steps=close_steps, eps_v=1e-3, dt=0.01)


def test_halt_needs_a_force_above_50_newton():
    """A finger stops once its contact force exceeds 50 N: exactly 50 N (after the second step at
    25 N per step) does not stop it, 75 N after the third does."""
    out = _run(RateScene(20, 1e-7, rates=[25.0, 1.0], handles=[[0, 2], [1, 2]]))
    assert out.halted == {0: 2}


def test_stable_needs_gripper_contact_and_a_still_last_step():
    """Stable means the object touches a finger (not merely another body, such as a table of
    handle 3) at the last step, and its centre of mass moved less than eps_v dt over that last
    step alone: 1.7e-6 m per step is still, although the hold's 15 steps add up to 2.6e-5 m."""
    out = _run(RateScene(20, 1e-6, rates=[1.0, 1.0], handles=[[0, 2], [1, 2]]))
    assert out.in_contact and out.stable and out.com_step < 2e-6
    out = _run(RateScene(20, 1e-7, rates=[1.0, 1.0], handles=[[2, 3], [0, 1]]))
    assert not out.in_contact and not out.stable
