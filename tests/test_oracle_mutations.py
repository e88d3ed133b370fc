"""Mutation check of the oracle's pins: each plausible mistake below is
planted in a temporary copy of oracle/seg_oracle.c, compiled, and the pins of
tests/test_oracle_pins.py named beside it must fail against that copy
(SEG_ORACLE_LIB makes the oracle module load it).  A mistake that no pin
catches would leave the oracle's parity claim unfounded.

Each mutation is (name, function whose body is edited, text, replacement,
pins expected to catch it as a pytest -k expression).  The pins named are
the ones resting on the paper or on mathematics (minimisers, closed forms,
brute force, adjointness), not the independent re-implementation of the
unrestricted iteration.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "seg_oracle.c")
HDR = os.path.join(ROOT, "oracle", "seg_oracle.h")

_SOLVE = "int oracle_solve(const float"
_PD = "int oracle_solve_pd("
_VOL = "int oracle_solve3("

MUTATIONS = [
    # Section 2.1 / 3 fixed-point step, u- and v-steps
    ("g_sign", _SOLVE, "q1[x] = (p1[x] + tau * g1[x]) / den;", "q1[x] = (p1[x] - tau * g1[x]) / den;",
     "df_minimum or restricted_minimum"),
    ("tau_in_denominator", _SOLVE, "double den = 1.0 + tau * nrm;", "double den = 1.0 + 2.0 * tau * nrm;",
     "df_minimum or restricted_minimum or rof_subproblem"),
    ("w_sign", _SOLVE, "w[x] = d[x] - v[x] / theta;", "w[x] = d[x] + v[x] / theta;",
     "df_minimum or restricted_minimum"),
    ("u_sign", _SOLVE, "double un = v[x] - theta * d[x];", "double un = v[x] + theta * d[x];",
     "df_minimum or restricted_minimum or rof_subproblem"),
    ("v_step_without_theta", _SOLVE, "clamp01(un - theta * lambda * (double)f32[x]);",
     "clamp01(un - lambda * (double)f32[x]);", "df_minimum or restricted_minimum or large_lambda"),
    ("anisotropic_norm", _SOLVE, "double nrm = sqrt(g1[x] * g1[x] + g2[x] * g2[x]);",
     "double nrm = fabs(g1[x]) + fabs(g2[x]);", "df_minimum or restricted_minimum"),
    ("heaviside_at_zero", _SOLVE, "double h = (f < 0.0) ? 1.0 : 0.0;     /* u0 = H(-f) */",
     "double h = (f <= 0.0) ? 1.0 : 0.0;", "initialisation_is_heaviside"),
    ("stop_norm_squared", _SOLVE, "double du = sqrt(su), dv = sqrt(sv);", "double du = su, dv = sv;",
     "stopping_rule"),
    # the restriction of Section 3: how fixed pixels enter the rho step
    ("fixed_v_swapped", _SOLVE, "w[x] = d[x] - v[x] / theta;",
     "w[x] = d[x] - (region[x] == 2 ? v[x] : 1.0 - v[x]) / theta;", "restricted_minimum"),
    ("fixed_w_without_div", _SOLVE, "w[x] = d[x] - v[x] / theta;",
     "w[x] = (region[x] == 2 ? d[x] : 0.0) - v[x] / theta;", "restricted_minimum"),
    ("tv_term_kept_at_fixed_pixel", _SOLVE,
     "                if (region[x] == 2) {\n                    double nrm",
     "                if (region[x] == 2 || (x + W < n && region[x + W] == 2)"
     " || (x + 1 < n && region[x + 1] == 2)) {\n                    double nrm",
     "restricted_minimum"),
    # Chambolle's operators
    ("div_index", "void oracle_div(", "(i > 0 ? p1[IDX(i - 1, j)] : 0.0)", "(i > 1 ? p1[IDX(i - 1, j)] : 0.0)",
     "minus_adjoint_of_grad and not div3"),
    ("grad_periodic", "void oracle_grad(", "(i < H - 1) ? w[IDX(i + 1, j)] - w[IDX(i, j)] : 0.0;",
     "(i < H - 1) ? w[IDX(i + 1, j)] - w[IDX(i, j)] : w[IDX(0, j)] - w[IDX(i, j)];",
     "(minus_adjoint_of_grad or grad_div_textbook) and not div3"),
    # partition and fitting term
    ("rd_boundary_inclusive", "void oracle_domain(", "if (fabsf(f) < delta) region[x] = 2;",
     "if (fabsf(f) <= delta) region[x] = 2;", "domain_special_cases or quantile"),
    ("quantile_rank", "float oracle_quantile_delta(", "float t = a[k - 1];", "float t = a[k > 1 ? k - 2 : 0];",
     "quantile_delta_is_minimal"),
    ("ds_squared_distance", "void oracle_fitting(", "sqrt((double)d2[x]) / dmax",
     "(double)d2[x] / (double)d2max", "ds_term_distance"),
    # energies and the dual bound
    ("dual_bound_sign", "void oracle_energy(", "double c = lambda * f + d[x];", "double c = lambda * f - d[x];",
     "duality_gap_and_brute_force"),
    ("tv_anisotropic", "static double tv(", "s += sqrt(a * a + b * b);", "s += fabs(a) + fabs(b);",
     "tv_textbook_value"),
    # restricted primal-dual solver (Chambolle-Pock)
    ("pd_primal_sign", _PD, "clamp01(u[x] + tau * (d[x] - lambda", "clamp01(u[x] + tau * (-d[x] - lambda",
     "pd_reaches_the_linear or pd_two_pixel"),
    ("pd_no_extrapolation", _PD, "ub[x] = 2.0 * un - u[x];", "ub[x] = un;", "pd_two_pixel"),
    ("pd_no_projection", _PD, "double s = nrm > 1.0 ? nrm : 1.0;", "double s = 1.0;",
     "pd_reaches_the_linear or pd_two_pixel or pd_duality_gap"),
    ("pd_dual_sign", _PD, "double a = p1[x] + sigma * g1[x];\n            double b = p2[x] + sigma * g2[x];",
     "double a = p1[x] - sigma * g1[x];\n            double b = p2[x] - sigma * g2[x];",
     "pd_reaches_the_linear or pd_two_pixel"),
    ("pd_lambda_scaled", _PD, "(d[x] - lambda * (double)f32[x])", "(d[x] - 2.0 * lambda * (double)f32[x])",
     "pd_reaches_the_linear or pd_two_pixel"),
    # robust restriction
    ("box_mean_count", "void oracle_box_mean(", "(float)(sum / (double)cnt)",
     "(float)(sum / (double)((2 * r + 1) * (2 * r + 1)))", "box_mean_is_the_clipped"),
    ("robust_without_sign_disagreement", "void oracle_domain_robust(",
     "if (fabsf(m) < delta || ((f < 0.0f) != (m < 0.0f))) region[x] = 2;",
     "if (fabsf(m) < delta) region[x] = 2;", "robust_restriction_trend"),
    ("dilation_radius", "void oracle_dilate(", "for (int a = i - r; a <= i + r && c != 2; ++a)",
     "for (int a = i - r + 1; a <= i + r && c != 2; ++a)", "dilation"),
    # 3-D volumes
    ("grad3_slice_boundary", "void oracle_grad3(", "(z < D - 1) ? w[IDX3(z + 1, i, j)] - c : 0.0;",
     "(z < D - 1) ? w[IDX3(z + 1, i, j)] - c : -c;", "div3 or grad3"),
    ("div3_sign", "void oracle_div3(", "d[IDX3(z, i, j)] = a + b + c;", "d[IDX3(z, i, j)] = a + b - c;",
     "div3 or volume"),
    ("vol_anisotropic_norm", _VOL, "double nrm = sqrt(g1[x] * g1[x] + g2[x] * g2[x] + g3[x] * g3[x]);",
     "double nrm = fabs(g1[x]) + fabs(g2[x]) + fabs(g3[x]);", "volume"),
    ("vol_p3_step", _VOL, "p3[x] = (p3[x] + tau * g3[x]) / den;", "p3[x] = (p3[x] + 0.5 * tau * g3[x]) / den;",
     "volume"),
]


def _plant(tmp, name, anchor, old, new):
    src = open(SRC).read()
    k = src.index(anchor)
    head, tail = src[:k], src[k:]
    assert old in tail, (name, "text not found after", anchor)
    d = os.path.join(tmp, name)
    os.makedirs(d)
    c = os.path.join(d, "seg_oracle.c")
    with open(c, "w") as fh:
        fh.write(head + tail.replace(old, new, 1))
    shutil.copy(HDR, d)
    lib = os.path.join(d, "liboracle.so")
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                           "-fno-fast-math", "-o", lib, c, "-lm"])
    return lib


def _run_pins(lib, expr):
    env = dict(os.environ, SEG_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        "-q", "-x", "-p", "no:cacheprovider", "-m", "not gpu", "-k", expr],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-2000:]


def test_mutation_list_is_well_formed():
    names = [m[0] for m in MUTATIONS]
    assert len(names) == len(set(names))
    src = open(SRC).read()
    for name, anchor, old, new, _ in MUTATIONS:
        assert src.count(anchor) == 1, name
        assert old in src[src.index(anchor):] and old != new, name


@pytest.mark.slow
def test_every_planted_mistake_fails_a_pin(tmp_path):
    """Every mutation makes at least one of its named pins fail (pytest exit
    status 1: tests ran and failed; not 5, which would mean the -k expression
    selected nothing)."""
    libs = [(m[0], _plant(str(tmp_path), *m[:4]), m[4]) for m in MUTATIONS]
    workers = max(1, min(8, len(os.sched_getaffinity(0))))
    with ThreadPoolExecutor(workers) as ex:
        results = list(ex.map(lambda t: (t[0], t[2], *_run_pins(t[1], t[2])), libs))
    survived = [(name, expr, rc, out) for name, expr, rc, out in results if rc != 1]
    assert not survived, "\n\n".join(f"{n} [{e}] exit {rc}\n{o}" for n, e, rc, o in survived)


def test_unmutated_oracle_passes_the_same_pins(tmp_path):
    """Control: the same harness on an unmodified copy passes (so the failures
    above come from the planted mistakes, not from the harness)."""
    lib = _plant(str(tmp_path), "control", "void oracle_domain(", "region[x] = 2;", "region[x] = 2;")
    rc, out = _run_pins(lib, "restricted_minimum or domain_special_cases or tv_textbook_value")
    assert rc == 0, out
