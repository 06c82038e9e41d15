"""The FGMRES-DR pins catch plausible mistakes in oracle/fgmresdr.py.

Each case copies the module source, plants one slip (on the CPU, in a
temporary directory), loads the copy, substitutes its functions for the
real ones for the duration of the case, and checks that a pin from
test_oracle_fgmresdr_pins fails.
"""
import importlib.util
import os

import pytest

from oracle import fgmresdr
from tests import test_oracle_fgmresdr_pins as P

MUTANTS = {
    "largest_harmonic_ritz": ('order = np.argsort(np.abs(theta), kind="stable")[:k]',
                              'order = np.argsort(np.abs(theta), kind="stable")[::-1][:k]'),
    "hsq_shifted_rows": ("hsq = hb[:nz, :nz]", "hsq = hb[1:, :nz]"),
    "projection_without_conjugate": ("hnew = pk1.conj().T @ H[:j + 1, :j] @ pk[:j]",
                                     "hnew = pk1.T @ H[:j + 1, :j] @ pk[:j]"),
    "z_not_transformed": ("Z = list((zmat @ pk[:j]).T)", "Z = list(zmat[:, :k].T)"),
    "gram_schmidt_sign": ("w = w - H[i, j] * V[i]", "w = w + H[i, j] * V[i]"),
    "restart_rhs_from_c": ("cnew = pk1.conj().T @ cls", "cnew = pk1.conj().T @ c[:j + 1]"),
}

PINS = [
    P.test_harmonic_ritz_definition,
    P.test_fgmres_equals_fgcr_after_the_same_iterations,
    P.test_deflated_restart_keeps_the_arnoldi_relation,
    P.test_planted_small_eigenvalues_are_deflated,
    P.test_harmonic_ritz_values_approach_smallest_eigenvalues_of_m,
]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path, monkeypatch):
    old, new = MUTANTS[name]
    src = open(fgmresdr.__file__).read()
    assert src.count(old) == 1, name
    path = tmp_path / "fgmresdr_mut.py"
    path.write_text(src.replace(old, new))
    spec = importlib.util.spec_from_file_location("fgmresdr_mut", str(path))
    mut = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mut)
    monkeypatch.setattr(fgmresdr, "fgmres_dr", mut.fgmres_dr)
    monkeypatch.setattr(fgmresdr, "harmonic_ritz", mut.harmonic_ritz)
    caught = False
    for pin in PINS:
        try:
            pin()
        except Exception:
            caught = True
            break
    assert caught, "no pin caught mutant: " + name
