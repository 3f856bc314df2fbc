"""Planted mistakes: each mutant copy of the C oracle must fail at least one pin.

A plausible error anywhere in the oracle (a dropped term, a wrong sign, index or
factor) has to be caught by the pins in test_oracle_model / test_oracle_scheme /
test_oracle_physics. Each case below copies fdlbm_oracle.c, applies one textual
mistake, builds it into a temporary library, and runs the named pins against it
in a subprocess (FDLBM_ORACLE_LIB points the wrapper at the mutant). The mistake
is planted in the oracle, on the CPU.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "fdlbm_oracle.c")

MUTANTS = {
    # name: (original text, mistaken text, pins expected to catch it)
    "feq_drop_cubic": ("term0 + term1 + term2 + term3 + term4", "term0 + term1 + term2 + term4",
                       "tests/test_oracle_model.py::test_feq_reproduces_maxwellian_moments"),
    "feq_literal_bracket": ("n * F[k] * (term0 + term1 + term2 + term3 + term4)",
                            "n * F[k] * (term0 + term1 + term2) + term3 + term4",
                            "tests/test_oracle_model.py::test_feq_reproduces_maxwellian_moments"),
    "weights_cyclic_index": ("k + l - 4", "k + l - 3",
                             "tests/test_oracle_model.py::test_weights_match_maxwellian_radial_moments"),
    "weights_f0": ("F[0] = 1.0 - 8.0 * sumF", "F[0] = 1.0 - 4.0 * sumF",
                   "tests/test_oracle_model.py::test_feq_reproduces_maxwellian_moments"),
    "velocity_direction": ("case 3: *cx = -s;   *cy = s;", "case 3: *cx = s;    *cy = -s;",
                           "tests/test_oracle_model.py::test_velocity_set_geometry"),
    "moments_energy_factor": ("P += 0.5 * (wx * wx + wy * wy) * f[q];", "P += (wx * wx + wy * wy) * f[q];",
                              "tests/test_oracle_scheme.py::test_uniform_state_is_fixed_point"),
    "relaxation_twice": ("double acc = f0 - r * (f0 - feq[q]);", "double acc = f0 - 2.0 * r * (f0 - feq[q]);",
                         "tests/test_oracle_scheme.py::test_relaxation_decay_law"),
    "convection_sign": ("acc -= c / 2.0 * (fp1 - fm1);", "acc += c / 2.0 * (fp1 - fm1);",
                        "tests/test_oracle_scheme.py::test_advection_is_third_order"),
    "lw_factor": ("acc += c * c / 2.0 * (fp1 - 2.0 * f0 + fm1);", "acc += c * c / 4.0 * (fp1 - 2.0 * f0 + fm1);",
                  "tests/test_oracle_scheme.py::test_advection_is_third_order"),
    "dispersion_sign": ("acc += c * (1.0 - c * c) / 12.0", "acc -= c * (1.0 - c * c) / 12.0",
                        "tests/test_oracle_scheme.py::test_advection_is_third_order"),
    "dispersion_stencil": ("(fp2 - 2.0 * fp1 + 2.0 * fm1 - fm2)", "(fp2 - 2.0 * fp1 + 2.0 * fm1 + fm2)",
                           "tests/test_oracle_scheme.py::test_advection_is_third_order"),
    "viscosity_factor": ("(1.0 - fabs(kap[a])) / 2.0 *", "(1.0 - fabs(kap[a])) *",
                         "tests/test_oracle_scheme.py::test_linearised_step_equals_amplification_matrix"),
    "viscosity_abs_kappa": ("sw[a] * fabs(kap[a]) *", "sw[a] * kap[a] *",
                            "tests/test_oracle_scheme.py::test_linearised_step_equals_amplification_matrix"),
    "kappa_axis": ("kap[a] = ua * s->dt / dr[a];", "kap[a] = ua * s->dt / dr[0];",
                   "tests/test_oracle_scheme.py::test_linearised_step_equals_amplification_matrix"),
    "switch_denominator": ("(Pp + 2.0 * P0 + Pm)", "(Pp + P0 + Pm)",
                           "tests/test_oracle_scheme.py::test_switch_uses_pressure_and_is_bounded"),
    "switch_uses_density": ("double Pp = s->n[MI(s, i + di, j + dj)] * s->T[MI(s, i + di, j + dj)];",
                            "double Pp = s->n[MI(s, i + di, j + dj)];",
                            "tests/test_oracle_scheme.py::test_switch_uses_pressure_and_is_bounded"),
    "wall_no_mirror": ("int j = (axis == 1) ? (8 - i) : (4 - i);", "int j = (axis == 1) ? (i) : (4 - i);",
                       "tests/test_oracle_scheme.py::test_wall_equals_mirrored_periodic_domain"),
    "outflow_wrong_node": ("case BC_OUTFLOW: G(q, i, gj) = G(q, i, 0); break;",
                           "case BC_OUTFLOW: G(q, i, gj) = G(q, i, 1); break;",
                           "tests/test_oracle_scheme.py::test_ghost_ring_contents"),
    "periodic_offset": ("case BC_PERIODIC: G(q, gi, j) = G(q, posmod(gi, nx), j); break;",
                        "case BC_PERIODIC: G(q, gi, j) = G(q, posmod(gi + 1, nx), j); break;",
                        "tests/test_oracle_scheme.py::test_conservation_at_lambda_zero"),
}


def _build_mutant(tmp_path, name):
    orig, bad, _ = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(orig) >= 1, "mutation anchor not found: %s" % name
    mutated = src.replace(orig, bad, 1)
    cpath = tmp_path / ("%s.c" % name)
    cpath.write_text(mutated)
    lib = tmp_path / ("lib_%s.so" % name)
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-fPIC", "-shared", str(cpath),
                           "-o", str(lib), "-lm"])
    return lib


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    lib = _build_mutant(tmp_path, name)
    env = dict(os.environ, FDLBM_ORACLE_LIB=str(lib))
    target = MUTANTS[name][2]
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", target],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1, "mutant %s survived %s:\n%s" % (name, target, r.stdout[-2000:])


def test_unmutated_copy_passes(tmp_path):
    """Control: the same procedure with no mistake passes the same pins."""
    src = open(SRC).read()
    cpath = tmp_path / "same.c"
    cpath.write_text(src)
    lib = tmp_path / "lib_same.so"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-fPIC", "-shared", str(cpath),
                           "-o", str(lib), "-lm"])
    env = dict(os.environ, FDLBM_ORACLE_LIB=str(lib))
    targets = sorted({m[2] for m in MUTANTS.values()})
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider"] + targets,
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:]
