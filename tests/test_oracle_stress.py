"""Per-tet von Mises stress of the CPU oracle against closed forms of the Neo-Hookean Cauchy
stress sigma = (mu (F F^T - I) + lam ln J I) / J (no GPU): zero for a pure dilation,
mu gamma sqrt(3 + gamma^2) in simple shear, (mu / s) |s^2 - 1| in a uniaxial stretch."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_05020_b300 import scenes as S


def _stress_under(F):
    env = S.single_tet_env()
    soft = env["soft"][0]
    X = np.asarray(soft["verts"], dtype=np.float64)
    mu = soft["E"] / (2.0 * (1.0 + soft["nu"]))
    e = O.OracleEnv(S.scene_params(0.01), env)
    q = (X @ np.asarray(F, dtype=np.float64).T).reshape(-1)
    return e.tet_stress(q, 1)[0], mu


def test_dilation_has_no_von_mises_stress():
    vm, mu = _stress_under(1.1 * np.eye(3))
    assert abs(vm) <= 1e-9 * mu


@pytest.mark.parametrize("gamma", [1e-3, 0.2, 0.7])
def test_simple_shear(gamma):
    F = np.eye(3)
    F[0, 1] = gamma
    vm, mu = _stress_under(F)
    assert abs(vm / (mu * gamma * np.sqrt(3.0 + gamma * gamma)) - 1.0) <= 1e-10


@pytest.mark.parametrize("s", [0.8, 1.05, 1.5])
def test_uniaxial_stretch(s):
    vm, mu = _stress_under(np.diag([s, 1.0, 1.0]))
    assert abs(vm / (mu / s * abs(s * s - 1.0)) - 1.0) <= 1e-10
