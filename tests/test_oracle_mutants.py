"""The pins must reject plausible mistakes in the oracle.

Each case copies oracle/oracle.c to a temporary directory, plants one mistake
(a flipped sign, a missing conjugate, a swapped operand, a wrong bit order, a
dropped factor ...), compiles it with gcc and runs the pins on it: at least one
pin has to fail.  Mistakes are planted only in these CPU copies.
"""
import os
import shutil
import subprocess

import pytest

import oracle
import oracle_pins as P

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

MUTANTS = {
    "rotation_sign": ("m[r][k] = (r == k ? co : 0.0) - I * si * p[r][k];",
                      "m[r][k] = (r == k ? co : 0.0) + I * si * p[r][k];"),
    "dagger_without_conjugate": ("m[0][1] = conj(m[1][0]);", "m[0][1] = m[1][0];"),
    "cnot_control_target_swapped": ("uint64_t bc = 1ull << c->q0[g], bt = 1ull << c->q1[g];",
                                    "uint64_t bc = 1ull << c->q1[g], bt = 1ull << c->q0[g];"),
    "cz_or_instead_of_and": ("if ((x & ba) && (x & bb)) psi[x] = -psi[x];",
                             "if ((x & ba) || (x & bb)) psi[x] = -psi[x];"),
    "big_endian_bit_order": ("uint64_t N = 1ull << n, bit = 1ull << q;",
                             "uint64_t N = 1ull << n, bit = 1ull << (n - 1 - q);"),
    "adjoint_missing_factor_two": ("dth[g] = 2.0 * inner_re(lam, mu, N);",
                                   "dth[g] = inner_re(lam, mu, N);"),
    "chain_rule_wrong_factor": ("gw_b[c->widx[g]] += dtheta[g] * c->coef[g] * X;",
                                "gw_b[c->widx[g]] += dtheta[g] * c->coef[g] * W;"),
    "parity_sign_flipped": ("((popcount64(x & c->zmask[t]) & 1) ? -1.0 : 1.0)",
                            "((popcount64(x & c->zmask[t]) & 1) ? 1.0 : -1.0)"),
    "probability_drops_imag": ("double p = creal(psi[x]) * creal(psi[x]) + cimag(psi[x]) * cimag(psi[x]);",
                               "double p = creal(psi[x]) * creal(psi[x]);"),
    "costate_without_observable": ("lam[xx] = d * phi[xx];", "lam[xx] = phi[xx];"),
    "derivative_sign": ("m[r][k] = (r == k ? -0.5 * si : 0.0) - I * 0.5 * co * p[r][k];",
                        "m[r][k] = (r == k ? -0.5 * si : 0.0) + I * 0.5 * co * p[r][k];"),
    "pauli_y_transposed": ("else if (kind == OR_RY) { m[0][1] = -I; m[1][0] = I; }",
                           "else if (kind == OR_RY) { m[0][1] = I; m[1][0] = -I; }"),
    "partition_extra_on_last": ("*count = base + (t < extra ? 1 : 0);",
                                "*count = base + (t >= T - extra ? 1 : 0);"),
    "angle_ignores_input": ("if (c->xidx[g] >= 0) th *= xb[c->xidx[g]];", ""),
    "rzz_phase_sign": ("cplx same = cexp(-I * 0.5 * t), diff = cexp(I * 0.5 * t);",
                       "cplx same = cexp(I * 0.5 * t), diff = cexp(-I * 0.5 * t);"),
    "rzz_derivative_sign": ("mu[x] *= -I * 0.5 * z * cexp(-I * 0.5 * t * z);",
                            "mu[x] *= I * 0.5 * z * cexp(-I * 0.5 * t * z);"),
    "hadamard_rows_swapped": ("cplx m[2][2] = {{r, r}, {r, -r}};", "cplx m[2][2] = {{r, -r}, {r, r}};"),
    "pauli_y_phase_missing": ("for (int k = 0; k < (ny & 3); ++k) ph *= I;", ""),
    "pauli_sign_on_output_index": ("double sg = (popcount64(x & zm) & 1) ? -1.0 : 1.0;",
                                   "double sg = (popcount64(y & zm) & 1) ? -1.0 : 1.0;"),
    "pauli_costate_unweighted": ("if (g) add_pauli(c, t, g[m] * c->zcoef[t], in, out);",
                                 "if (g) add_pauli(c, t, c->zcoef[t], in, out);"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_mutant(name, tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor not found: {old}"
    mut = src.replace(old, new, 1)
    cfile = tmp_path / "oracle_mut.c"
    cfile.write_text(mut)
    so = tmp_path / "liboracle_mut.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-fopenmp", str(cfile), "-o",
                    str(so), "-lm"], check=True)
    O = oracle.Oracle(str(so))
    failed = []
    for pin in P.ALL_PINS:
        try:
            pin(O)
        except AssertionError:
            failed.append(pin.__name__)
            break
    assert failed, f"mutant {name} passed every pin"
