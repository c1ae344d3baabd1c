"""The pins catch planted mistakes: each case compiles a copy of the oracle
with one plausible slip (a dropped term, a wrong sign, coefficient or index)
and requires the pins of that part of the oracle (tests/test_oracle_pins.py
without its golden regression fixture, which only guards drift, or
tests/test_oracle_transfer.py for the non-polytropic contents) to fail
against it.  The mistakes live only in temporary copies; the oracle itself is
untouched."""
import os
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "pab_oracle.c")

MUTATIONS = [
    ("viscous Rddot term of d/dt p_bw dropped", "+ 4.0 * P->mu * inv_c / P->rho;", ";"),
    ("sign of the surface-tension rate", "+ 2.0 * P->sigma * Rdot / (R * R);", "- 2.0 * P->sigma * Rdot / (R * R);"),
    ("3/2 Rdot^2 coefficient", "- 1.5 * Rdot * Rdot", "- 1.0 * Rdot * Rdot"),
    ("(1 + Rdot/c) factor sign", "(1.0 + Rdot * inv_c)", "(1.0 - Rdot * inv_c)"),
    ("SSP-RK3 second-stage weights swapped", "0.75 * y[k] + 0.25", "0.25 * y[k] + 0.75"),
    ("Simpson coefficient 4 -> 2", "simpson = 4.0;", "simpson = 2.0;"),
    ("<R^2 Rdot> with an extra R", "M2V += w[b] * r * r * v;", "M2V += w[b] * r * r * r * v;"),
    ("controller exponent 1/2", "double fac = 0.9 * cbrt(tol / err);", "double fac = 0.9 * sqrt(tol / err);"),
    ("gamma dropped from dp_b", "dp_b = -3.0 * P->gamma * p_gas * Rdot / R;", "dp_b = -3.0 * p_gas * Rdot / R;"),
    ("viscous wall stress 2 mu", "- 4.0 * P->mu * Rdot / R - 2.0", "- 2.0 * P->mu * Rdot / R - 2.0"),
    ("R dropped from the R dp_bw/(rho c) term", "R * inv_c / P->rho * dp_bw_explicit", "inv_c / P->rho * dp_bw_explicit"),
    ("(1 - Rdot/(3c)) as (1 - Rdot/c)", "(1.0 - Rdot * inv_c / 3.0)", "(1.0 - Rdot * inv_c)"),
    ("alpha source without the 3", "out[4 * C + c] = 3.0 * alpha * M2V / M3;", "out[4 * C + c] = alpha * M2V / M3;"),
    ("last trial never detected", "int last = (h >= remaining);", "int last = (h > remaining + 1.0);"),
    ("EL kernel width fixed at dx", "double h = R[n] < dx ? dx : R[n];", "double h = dx;"),
    ("EL cut at 2h", "if (!(d / h < 3.0))", "if (!(d / h < 2.0))"),
    ("EL Gaussian without the 2", "double delta = exp(-d * d / (2.0 * h * h)) / (h * h * h * norm);",
     "double delta = exp(-d * d / (h * h)) / (h * h * h * norm);"),
    ("EL cell centre off by half a cell", "double cx = (i + 0.5) * dx - x[n];", "double cx = (i + 1.0) * dx - x[n];"),
    ("EL growth rate with R instead of R^2", "double Vdot = 4.0 * M_PI * R[n] * R[n] * Rdot[n];",
     "double Vdot = 4.0 * M_PI * R[n] * Rdot[n];"),
    ("n_b from alpha: alpha outside the root", "double nb = sqrt(4.0 / 3.0 * M_PI * s / alpha[c]);",
     "double nb = sqrt(4.0 / 3.0 * M_PI * s) / alpha[c];"),
    ("mixture pressure: sign of rho <R^3 Rdot^2>",
     "p[c] = (1.0 - alpha) * p_l[c] + alpha * (moments[5 * C + c] - rho * moments[6 * C + c]);",
     "p[c] = (1.0 - alpha) * p_l[c] + alpha * (moments[5 * C + c] + rho * moments[6 * C + c]);"),
    ("stiffened gas without gamma on pi_inf", "p_l[i] = (gamma_l - 1.0) * rho_l[i] * e_l[i] - gamma_l * pi_inf;",
     "p_l[i] = (gamma_l - 1.0) * rho_l[i] * e_l[i] - pi_inf;"),
    ("alpha with 4 pi for 4/3 pi", "double alpha = 4.0 / 3.0 * M_PI * n_b[c] * M3;",
     "double alpha = 4.0 * M_PI * n_b[c] * M3;"),
    ("bin spacing over B instead of B - 1", "double dphi = 2.0 * K * s / (double)(B - 1);",
     "double dphi = 2.0 * K * s / (double)B;"),
    ("bin weights not normalised", "w[i] = w[i] / total;", "w[i] = w[i];"),
    ("polytropic exponent gamma for 3 gamma", "double p_gas = p_g0 * pow(R0 / R, 3.0 * P->gamma);",
     "double p_gas = p_g0 * pow(R0 / R, P->gamma);"),
    ("p_g0 without surface tension", "double p_g0 = P->p0 + 2.0 * P->sigma / R0 - P->pv;",
     "double p_g0 = P->p0 - P->pv;"),
    ("embedded member taken as the Euler stage", "z[k] = 0.5 * y[k] + 0.5 * (y1[k] + h * f[k]);",
     "z[k] = y1[k];"),
    ("error norm without the Rdot floor", "if (vscale < v_floor)", "if (0)"),
    ("<R^3 p_bw> with R^2", "M3P += w[b] * r3 * p_bw;", "M3P += w[b] * r * r * p_bw;"),
    ("carried proposal always h_try * fac", "h = (clipped && fac >= 1.0) ? h : h_try * fac;",
     "h = h_try * fac;"),
    ("unclipped proposal kept whatever fac", "h = (clipped && fac >= 1.0) ? h : h_try * fac;",
     "h = clipped ? h : h_try * fac;"),
    ("no forced 0.2 after a non-positive stage", "if (!positive && fac > 0.2)", "if (0)"),
]

# Mistakes in the non-polytropic contents, caught by tests/test_oracle_transfer.py.
TRANSFER_MUTATIONS = [
    ("heat term without (gamma-1)/gamma", "(gb - 1.0) / gb * T->k_bw * dT_dr", "T->k_bw * dT_dr"),
    ("vapour enthalpy with the gas constant of the gas", "T->R_v * T->T_w * mdot_v", "T->R_g * T->T_w * mdot_v"),
    ("vapour mass rate without the wall area", "*dmv = 4.0 * M_PI * R * R * mdot_v;", "*dmv = 4.0 * M_PI * R * mdot_v;"),
    ("mean temperature with one gas constant", "(m_g * T->R_g + m_v * T->R_v)", "((m_g + m_v) * T->R_g)"),
    ("sign of the compression term", "(-Rdot * p_b +", "(Rdot * p_b +"),
    ("wall temperature gradient reversed", "(T->T_w - T_mean) / R", "(T_mean - T->T_w) / R"),
    ("wall vapour fraction of the gas", "double chi_vw = rho_v_w / rho_bw;", "double chi_vw = rho_g_w / rho_bw;"),
    ("last stage weights of the four-component trial", "y3[k] = y[k] / 3.0 + 2.0 / 3.0 * (y2[k] + h * f[k]);",
     "y3[k] = y[k] / 2.0 + 1.0 / 2.0 * (y2[k] + h * f[k]);"),
    ("transfer moments without surface tension", "double p_bw = pb[k] - 4.0 * P->mu * v / r - 2.0 * P->sigma / r;",
     "double p_bw = pb[k] - 4.0 * P->mu * v / r;"),
]

# The non-polytropic section repeats some of the polytropic text; each mutation
# is placed in its own part of the file.
MARK = "/* Non-polytropic bubble contents"


def _run_mutant(name, head, tail, pins, tmp_path):
    msrc = tmp_path / "mutant.c"
    msrc.write_text(head + tail)
    lib = oracle.compile_to(str(msrc), str(tmp_path / "libmutant.so"))
    env = dict(os.environ, PAB_ORACLE_LIB=lib, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", pins),
                        "-x", "-q", "-p", "no:cacheprovider", "-k", "not golden_regression"],
                       cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"no pin caught: {name}\n{r.stdout[-2000:]}"
    assert "failed" in r.stdout


def _parts():
    src = open(SRC).read()
    i = src.index(MARK)
    return src[:i], src[i:]


@pytest.mark.parametrize("name,orig,mutant", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(name, orig, mutant, tmp_path):
    head, tail = _parts()
    assert head.count(orig) == 1, f"mutation anchor not unique: {orig}"
    _run_mutant(name, head.replace(orig, mutant), tail, "test_oracle_pins.py", tmp_path)


@pytest.mark.parametrize("name,orig,mutant", TRANSFER_MUTATIONS, ids=[m[0] for m in TRANSFER_MUTATIONS])
def test_transfer_pins_catch_planted_mistake(name, orig, mutant, tmp_path):
    head, tail = _parts()
    assert tail.count(orig) == 1, f"mutation anchor not unique: {orig}"
    _run_mutant(name, head, tail.replace(orig, mutant), "test_oracle_transfer.py", tmp_path)
