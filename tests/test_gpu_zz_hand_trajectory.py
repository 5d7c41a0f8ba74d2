"""The hinged rigid hand of the third configuration against a stored oracle trajectory (needs a
B300): 20 PD-driven affine links hinged to a kinematic palm curl onto a ~22k-tet star-shaped soft
object over 200 steps (dhat 5e-4 m); the oracle's Newton iterations per step triple over the
last 20, where the fingers reach the object. Every sampled DOF (strided object vertices, all 252
affine coordinates) stays within 1e-6 of the oracle's at each of the 10 checkpoints. The golden
is written by `tests/golden/make_trajectory_goldens.py` (case hand_0) and compared by the same
routine as the other 100-step trajectories.
"""
import pytest

from test_gpu_trajectory100 import run_against_goldens

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_hinged_hand_200_steps_match_the_oracle():
    run_against_goldens(["hand_0"])
