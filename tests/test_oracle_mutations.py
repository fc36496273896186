"""The oracle's pins are strong enough to catch plausible mistakes.

Each case plants one mistake in a temporary copy of the oracle's C source (a
dropped term, a wrong sign, a wrong coefficient, a transposed table entry, a
wrong adjoint index), rebuilds that copy, and runs the pin suites against it:
at least one pin must fail. Nothing here touches the real oracle or a GPU.
"""

import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = {
    "velocity_without_half_force": (
        "u[a] = (m[a] + 0.5 * F[a]) / rho;\n    for (int i = 0; i < Q; ++i)\n      fout",
        "u[a] = (m[a]) / rho;\n    for (int i = 0; i < Q; ++i)\n      fout"),
    "guo_prefactor_dropped": ("(1.0 - 0.5 / tau) * guo_source", "(1.0) * guo_source"),
    "lid_term_sign": ("corr = 6.0 * weight(i)", "corr = -6.0 * weight(i)"),
    "equilibrium_quadratic_coefficient": ("4.5 * eu * eu", "4.0 * eu * eu"),
    "diagonal_weight": ("return 1.0 / 36.0;", "return 1.0 / 30.0;"),
    "velocity_columns_13_14_swapped": ("{0, 1, -1}, {0, -1, 1}", "{0, -1, 1}, {0, 1, -1}"),
    "adjoint_velocity_derivative_sign": (
        "v += (om * dfeq_du[a] + kf * dS_du[a]) * (E[j][a] - u[a]) / rho;",
        "v += (om * dfeq_du[a] + kf * dS_du[a]) * (E[j][a] + u[a]) / rho;"),
    "adjoint_bounce_back_not_transposed": (
        "lam_out[c * Q + opposite(i)] += mu[i];", "lam_out[c * Q + i] += mu[i];"),
    "moments_without_half_force": (
        "u[a * n + c] = (m[a] - 0.5 * F) / r;", "u[a * n + c] = (m[a]) / r;"),
    "lid_on_wrong_plane": ("sz == L->nz);", "sz < 0);"),
    "onsite_transverse_correction_dropped": ("  solve3(M, r, N);", "  if (0) solve3(M, r, N);"),
    "onsite_half_force_sign": ("j[a] = rho * uw[a] - 0.5 * F[a];",
                               "j[a] = rho * uw[a] + 0.5 * F[a];"),
    "onsite_edge_density_from_the_node_itself": ("rho += f[nb * Q + i];", "rho += f[c * Q + i];"),
    "onsite_lid_on_top_edges": ("if (L->lid && faces == 1 && z == L->nz - 1)",
                                "if (L->lid && z == L->nz - 1)"),
    "onsite_rebuild_weight": ("gc[i] = gc[ib] + 6.0 * weight(i) * ej - eN;",
                              "gc[i] = gc[ib] + 3.0 * weight(i) * ej - eN;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(os.path.join(ROOT, "oracle", "lbm_oracle.c")).read()
    assert old in src, "mutation site vanished; update the mutant table"
    ign = shutil.ignore_patterns("_build", "__pycache__", "*.so")
    for d in ("oracle", "tests", "paper_1309_1983_gb300"):
        shutil.copytree(os.path.join(ROOT, d), tmp_path / d, ignore=ign)
    (tmp_path / "oracle" / "lbm_oracle.c").write_text(src.replace(old, new, 1))
    (tmp_path / "pytest.ini").write_text("[pytest]\nmarkers =\n    gpu: gpu\n    slow: slow\n")
    r = subprocess.run(
        [sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
         "tests/test_oracle_pins.py", "tests/test_oracle_adjoint.py",
         "tests/test_oracle_onsite.py"],
        cwd=tmp_path, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1 and " failed" in r.stdout, r.stdout[-2000:] + r.stderr[-2000:]
