"""Mutation check of the oracle's pins (test infrastructure, CPU only).

Each entry of MUTATIONS plants one plausible mistake (a dropped term, a wrong sign, index,
factor, threshold or step) in a scratch copy of ipc_oracle.cpp. The checker copies the oracle,
its Python wrapper, the scene builders and the oracle's pin tests (tests/test_oracle_*.py) into
a temporary directory, builds the mutated oracle there and runs the pins. A mutation is KILLED
when some pin fails and SURVIVED when every pin still passes; a pin suite that lets a mistake
survive does not pin the code it touches.

    python oracle/mutation_check.py            # all mutations, 4 at a time
    python oracle/mutation_check.py -j 8 barrier_sign joint_h2

The repository's own copy of the oracle is never modified.
"""
from __future__ import annotations

import argparse
import os
import shutil
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

# (name, text in ipc_oracle.cpp, replacement): the first occurrence is replaced
MUTATIONS = [
    # Neo-Hookean energy
    ("nh_trace_offset", "(tr - S(3.0))", "(tr - S(2.0))"),
    ("nh_mu_lnJ_sign", "- S(mu) * lnJ +", "+ S(mu) * lnJ +"),
    ("nh_lambda_half", "S(0.5 * lam) * lnJ * lnJ", "S(lam) * lnJ * lnJ"),
    ("nh_volume_weight", "double w = h2 * e.tvol[t];", "double w = h2 * e.tvol[t] * 0.5;"),
    # barrier, mollifier, friction smoothing
    ("barrier_sign", "return -(t * t) * log(d / S(dhat));", "return (t * t) * log(d / S(dhat));"),
    ("barrier_square", "return -(t * t) * log(d / S(dhat));", "return -(t) * log(d / S(dhat));"),
    ("barrier_cutoff", "if (value(d) >= dhat) return S(0.0);", "if (value(d) >= 0.5 * dhat) return S(0.0);"),
    ("mollifier_linear", "return -(r * r) + S(2.0) * r;", "return r;"),
    ("mollifier_eps_scale", "k.eps_x = k.kind == 1 ? 1e-3 *", "k.eps_x = k.kind == 1 ? 1e-1 *"),
    ("friction_f0_constant", "+ y * y / eh + eh / 3.0;", "+ y * y / eh;"),
    ("friction_f1_slope", "*f1 = -y * y / (eh * eh) + 2.0 * y / eh;", "*f1 = -y * y / (eh * eh) + y / eh;"),
    ("friction_lambda_kappa", "f.lambda = e.kappa * moll * std::fabs(b1);", "f.lambda = moll * std::fabs(b1);"),
    ("friction_mu", "double s = h2 * e.mu * f.lambda;", "double s = h2 * f.lambda;"),
    ("friction_eps_without_h", "const double eh = e.P.eps_v * h;", "const double eh = e.P.eps_v;"),
    ("friction_no_tangent_projection",
     "double u[3] = {rel[0] - nr * f.n[0], rel[1] - nr * f.n[1], rel[2] - nr * f.n[2]};",
     "double u[3] = {rel[0], rel[1], rel[2]};"),
    ("barrier_energy_h2", "Ebar += h2 * E.v;", "Ebar += E.v;"),
    ("barrier_derivatives_h2", "scatter(c.pts, E.g.data(), H12, h2);", "scatter(c.pts, E.g.data(), H12, 1.0);"),
    # distances
    ("pe_distance_norm", "return dot(c, c) / dot(e, e);", "return dot(c, c);"),
    ("pt_plane_square", "return e * e / dot(n, n);", "return e * e;"),
    ("ee_region_clamp", "if (t < 0) { t = 0; s = std::min(std::max(-c / a, 0.0), 1.0); }",
     "if (t < 0) { t = 0; s = std::min(std::max(c / a, 0.0), 1.0); }"),
    ("ee_parallel_band_wide", "if (den > 1e-10 * a * e) s =", "if (den > 1e-6 * a * e) s ="),
    ("ee_parallel_band_none", "if (den > 1e-10 * a * e) s =", "if (den > 1e-20 * a * e) s ="),
    # ACCD
    ("accd_first_advance", "double tl = (1.0 - s) * d / lp;", "double tl = (1.0 + s) * d / lp;"),
    ("accd_no_mean_shift", "for (int k = 0; k < 3; ++k) mean[k] = mean[k] / 4.0;",
     "for (int k = 0; k < 3; ++k) mean[k] = 0.0;"),
    ("accd_gap_fraction", "double t = accd(c[0], x12, p12, 0.1, 1.0, 1000000, &it);",
     "double t = accd(c[0], x12, p12, 0.9, 1.0, 1000000, &it);"),
    # broad phase
    ("broad_radius", "candidates(e, px, nullptr, 0.5 * e.P.dhat, cands);", "candidates(e, px, nullptr, 0.25 * e.P.dhat, cands);"),
    # masses and inertia
    ("lumped_mass_share", "e->mass[tt[k]] += S.rho * vol / 4.0;", "e->mass[tt[k]] += S.rho * vol / 3.0;"),
    ("abd_mass_second_moment", "I2[3 * i + j] += det / 120.0 *", "I2[3 * i + j] += det / 60.0 *"),
    ("predict_gravity_h", "+ hh * g[k];", "+ h * g[k];"),
    ("gravity_gate_ignored", "double hh = code ? h * h : 0.0;", "double hh = h * h;"),
    ("gravity_gate_next_step", "const int code = e.gravity[std::min(e.step, e.n_steps - 1)];",
     "const int code = e.gravity[std::min(e.step + 1, e.n_steps - 1)];"),
    ("axis_gravity_sign", "g[(code - 2) / 2] = code % 2 == 0 ? gm : -gm;", "g[(code - 2) / 2] = code % 2 == 0 ? -gm : gm;"),
    ("inertia_soft_half", "Einert += 0.5 * e.mass[i] * d * d;", "Einert += e.mass[i] * d * d;"),
    ("velocity_update", "e.v[d] = (e.x[d] - e.xt[d]) / h;", "e.v[d] = (e.x[d] - e.xt[d]);"),
    # affine body terms
    ("abd_orth_identity", "if (i == j) s = s - Dual<9>(1.0);", "if (i == j) s = s - Dual<9>(0.5);"),
    ("abd_orth_volume", "double w = h2 * e.P.kappa_affine * B.vol;", "double w = h2 * e.P.kappa_affine;"),
    ("pd_weight_h2", "const double w = h2 * B.kpd;", "const double w = B.kpd;"),
    ("pd_target_next_step", "const int st = std::min(e.step, e.n_steps - 1);",
     "const int st = std::min(e.step + 1, e.n_steps - 1);"),
    # joints
    ("joint_h2", "const double c = h2 * J.k;", "const double c = J.k;"),
    ("joint_anchor_swap", "jt.xa[k] = J.anchor_a[k]; jt.xb[k] = J.anchor_b[k];",
     "jt.xa[k] = J.anchor_b[k]; jt.xb[k] = J.anchor_a[k];"),
    ("joint_hessian_coupling_sign", "H->add(dofs[s1] + 3 * m + k, dofs[s2] + 3 * n + k, sg[s1] * sg[s2] * c",
     "H->add(dofs[s1] + 3 * m + k, dofs[s2] + 3 * n + k, c"),
    # Newton loop, line search, stiffness adaptation
    ("newton_tol_on_p", "if (!constrained && step_norm(e, p) / h < e.P.newton_tol)",
     "if (!constrained && step_norm(e, p) < e.P.newton_tol)"),
    ("line_search_third", "alpha = alpha / 2.0;", "alpha = alpha / 3.0;"),
    ("kappa_start_clamp_low", "e.kappa = std::min(std::max(k, e.P.kappa), 1000.0 * e.P.kappa);",
     "e.kappa = std::min(k, 1000.0 * e.P.kappa);"),
    ("kappa_start_sign", "const double k = -eg / gg;", "const double k = eg / gg;"),
]

PIN_TESTS = ["tests/test_oracle_elements.py", "tests/test_oracle_scenes.py", "tests/test_oracle_stress.py"]


def run_one(name: str, old: str, new: str, timeout: float = 1800.0) -> tuple[str, str, str]:
    """Build the oracle with one planted mistake in a scratch directory and run the pins there."""
    src = open(os.path.join(HERE, "ipc_oracle.cpp")).read()
    if old not in src:
        return name, "MISSING", "the text to replace is not in the oracle"
    work = tempfile.mkdtemp(prefix=f"mut_{name}_")
    try:
        skip = shutil.ignore_patterns("*.so", "*.so.tmp", "__pycache__", "mutation_check.py")
        shutil.copytree(HERE, os.path.join(work, "oracle"), ignore=skip)
        os.makedirs(os.path.join(work, "paper_2503_05020_b300"))
        for f in ("__init__.py", "scenes.py"):
            shutil.copy(os.path.join(ROOT, "paper_2503_05020_b300", f), os.path.join(work, "paper_2503_05020_b300", f))
        os.makedirs(os.path.join(work, "tests"))
        for f in ["conftest.py", *[os.path.basename(t) for t in PIN_TESTS]]:
            shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(work, "tests", f))
        if os.path.isdir(os.path.join(ROOT, "tests", "golden")):
            shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(work, "tests", "golden"))
        shutil.copy(os.path.join(ROOT, "pytest.ini"), work)
        with open(os.path.join(work, "oracle", "ipc_oracle.cpp"), "w") as f:
            f.write(src.replace(old, new, 1))
        try:
            r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *PIN_TESTS],
                               cwd=work, capture_output=True, text=True, timeout=timeout)
        except subprocess.TimeoutExpired:
            return name, "KILLED", "pins timed out (the mutated oracle no longer finishes)"
        failed = [l for l in r.stdout.splitlines() if l.startswith("FAILED") or l.startswith("ERROR")]
        if r.returncode == 0:
            return name, "SURVIVED", r.stdout.strip().splitlines()[-1] if r.stdout.strip() else ""
        return name, "KILLED", failed[0] if failed else (r.stdout + r.stderr).strip().splitlines()[-1]
    finally:
        shutil.rmtree(work, ignore_errors=True)


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("-j", type=int, default=4, help="mutations checked at once")
    ap.add_argument("names", nargs="*", help="mutations to check (default: all)")
    a = ap.parse_args()
    todo = [m for m in MUTATIONS if not a.names or m[0] in a.names]
    survived = 0
    with ThreadPoolExecutor(max(1, a.j)) as ex:
        for name, outcome, detail in ex.map(lambda m: run_one(*m), todo):
            survived += outcome != "KILLED"
            print(f"{outcome:8s} {name:28s} {detail[:120]}", flush=True)
    print(f"{len(todo) - survived} of {len(todo)} killed")
    return 1 if survived else 0


if __name__ == "__main__":
    sys.exit(main())
