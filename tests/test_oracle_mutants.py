"""The oracle's pins catch plausible mistakes.

Each case copies oracle.c, plants one typical slip in the copy (on the CPU,
in a temporary directory), compiles it, and checks that at least one pin
from test_oracle_pins / test_oracle_net_pins fails against the broken build.
"""
import os
import subprocess

import pytest

import oracle
from tests import test_oracle_pins as P
from tests import test_oracle_net_pins as NP
from tests import test_oracle_sap_pins as SP

MUTANTS = {
    "forward_projector_1_g": ("add_hop(out, g, -1.0, link(U, x, mu)",
                              "add_hop(out, g, +1.0, link(U, x, mu)"),
    "backward_link_not_daggered": ("mat3_dag(link(U, xb, mu), Vd);",
                                   "memcpy(Vd, link(U, xb, mu), sizeof(Vd));"),
    "t_boundary_sign_dropped": ("if (dir < 0 && c[3] == 0) return -1.0;",
                                "if (dir < 0 && c[3] == 0) return 1.0;"),
    "wrong_extent_in_wrap": ("n[mu] = (n[mu] + dir + d[mu]) % d[mu];",
                             "n[mu] = (n[mu] + dir + d[0]) % d[0];"),
    "clover_leaf_normalisation": ("(Q[3 * i + j] - conj(Q[3 * j + i])) / 8.0",
                                  "(Q[3 * i + j] - conj(Q[3 * j + i])) / 4.0"),
    "clover_leaf_orientation": ("mat3_dag(link(U, xpn, mu), a); mat3_mul(t, a, t);",
                                "memcpy(a, link(U, xpn, mu), sizeof(a)); mat3_mul(t, a, t);"),
    "clover_sign": ("I * kappa * csw * sig[p][s][r] * f[3 * ca + cb]",
                    "-I * kappa * csw * sig[p][s][r] * f[3 * ca + cb]"),
    "schur_sign": ("out[i] -= kappa * kappa * uo[i];", "out[i] += kappa * kappa * uo[i];"),
    "schur_misses_a_ee_1": ("if (Ainv) oracle_apply_site_matrices(V, Ainv, te, te);", ""),
    "cg_alpha": ("double alpha = rr / norm2(n, q);", "double alpha = rr / norm2(n, p);"),
    "transport_forward_uses_dagger": ("if (fwd) memcpy(V, link(U, x, mu), sizeof(V));",
                                      "if (fwd) mat3_dag(link(U, x, mu), V);"),
    "wgrad_missing_conj": ("acc += g[3 * i + a] * conj(tr[3 * j + a]);",
                           "acc += g[3 * i + a] * tr[3 * j + a];"),
    "sap_no_dirichlet": ("if (bid[x] != b) memset(q + 12 * x, 0, 12 * sizeof(cplx));", ";"),
    "sap_block_colour": ("return (c[0] / bs[0] + c[1] / bs[1] + c[2] / bs[2] + c[3] / bs[3]) & 1;",
                         "return (c[0] / bs[0] + c[1] / bs[1] + c[2] / bs[2]) & 1;"),
}

PINS = [
    lambda: P.test_free_field_closed_form((2, 4, 6, 8)),
    P.test_gamma5_hermiticity,
    P.test_gauge_covariance,
    lambda: P.test_dense_brute_force((2, 2, 2, 4), 1.0),
    lambda: P.test_dense_schur_complement((2, 2, 2, 2)),
    lambda: P.test_clover_constant_abelian_field(0, 1, 1),
    NP.test_layer_reduces_to_wilson_operator,
    NP.test_weight_gradient_finite_differences,
    SP.test_exact_block_solves_clear_last_colour,
    SP.test_block_solve_matches_dense_dirichlet_solve,
    P.test_solvers_against_dense_solve,  # slowest last
]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    assert src.count(old) == 1, name
    mut = tmp_path / "oracle_mut.c"
    mut.write_text(src.replace(old, new))
    so = tmp_path / "liboracle_mut.so"
    subprocess.check_call(["gcc", "-std=gnu99", "-O2", "-fcx-limited-range", "-fopenmp",
                           "-shared", "-fPIC", "-o", str(so), str(mut), "-lm"])
    prev = oracle.use_library(str(so))
    caught = []
    try:
        for pin in PINS:
            try:
                pin()
            except (AssertionError, FloatingPointError, ValueError, ZeroDivisionError,
                    OverflowError, Exception):
                caught.append(pin)
                break
    finally:
        oracle.use_library(None)
        oracle._lib = prev
    assert caught, "no pin caught mutant: " + name
