"""Pins of the oracle's flexible GMRES with deflated restarts (Sec. 7).

- Without deflation FGMRES(m) and FGCR(m) are the same method (the paper
  notes the equivalence): after the same number of iterations, with the
  same restarts, both hold the same minimal-residual iterate.
- Each GMRES iterate minimises |b - M x| over the Krylov space; a dense
  brute-force least-squares solve on a 2^4 lattice gives the same residuals.
- After a deflated restart the basis keeps M Z = V Hbar, V orthonormal,
  and the true residual equals V c.
- On a matrix with four planted small eigenvalues the deflated restarts
  find them (harmonic Ritz values) and cut the iteration count several
  times; on the lattice operator (2^4, dense spectrum) the kept harmonic
  Ritz values approach the smallest eigenvalues of M.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import fgmresdr

DIMS = (4, 4, 4, 4)


def _system(dims, kappa, csw=1.0, seed=3):
    U = synth.smooth_gauge(dims, 0.5, seed)
    A = oracle.clover(U, kappa, csw)
    b = synth.gaussian_spinor(dims, 0)
    return U, A, b


def test_fgmres_equals_fgcr_after_the_same_iterations():
    U, A, b = _system(DIMS, 0.13)
    for maxiter in (5, 8, 21):  # within a cycle, at a restart, two restarts later
        x1, it1, _, _ = oracle.fgmres_dr(U, A, 0.13, b, m=8, k=0, maxiter=maxiter)
        x2, it2, _, _ = oracle.fgcr(U, A, 0.13, b, nkrylov=8, maxiter=maxiter)
        assert it1 == it2 == maxiter
        assert np.linalg.norm(x1 - x2) / np.linalg.norm(x2) < 1e-9


def test_fgmres_equals_fgcr_with_a_fixed_linear_preconditioner():
    """With a fixed linear right preconditioner P (here 1 + kappa H) both
    search P K_j(M P, r0).  (SAP is not linear in r: its MR step lengths
    depend on r, so the two methods differ under it.)"""
    U, A, b = _system(DIMS, 0.13)

    def hopping(r):
        return r + 0.13 * oracle.hop(U, r)

    x1, it1, _, _ = oracle.fgmres_dr(U, A, 0.13, b, m=6, k=0, maxiter=9, prec=hopping)
    x2, it2, _, _ = oracle.fgcr(U, A, 0.13, b, nkrylov=6, maxiter=9, prec=hopping)
    assert np.linalg.norm(x1 - x2) / np.linalg.norm(x2) < 1e-9


def _dense(U, A, kappa, dims):
    n = int(np.prod(dims)) * 12
    M = np.zeros((n, n), dtype=complex)
    for i in range(n):
        e = np.zeros(n, dtype=complex)
        e[i] = 1.0
        M[:, i] = oracle.wilson_clover(U, A, kappa, e.reshape(dims + (4, 3))).reshape(-1)
    return M


def test_minimal_residual_against_brute_force():
    dims = (2, 2, 2, 2)
    kappa = 0.13
    U, A, b = _system(dims, kappa)
    M = _dense(U, A, kappa, dims)
    bv = b.reshape(-1)
    hist = []
    oracle.fgmres_dr(U, A, kappa, b, tol=1e-14, m=12, k=0, maxiter=12, history=hist)
    krylov = [bv]
    for j in range(1, 13):
        basis = np.linalg.qr(np.stack(krylov, axis=1))[0]
        y = np.linalg.lstsq(M @ basis, bv, rcond=None)[0]
        want = np.linalg.norm(bv - M @ basis @ y) / np.linalg.norm(bv)
        assert abs(hist[j - 1] - want) <= 1e-9 * max(want, 1e-12) + 1e-13, (j, hist[j - 1], want)
        krylov.append(M @ krylov[-1])


def test_deflated_restart_keeps_the_arnoldi_relation():
    kappa = 0.13
    U, A, b = _system(DIMS, kappa)
    shape = b.shape
    seen = []

    def check(V, Z, H, c, theta):
        MZ = np.stack([oracle.wilson_clover(U, A, kappa, Z[:, i].reshape(shape)).reshape(-1)
                       for i in range(Z.shape[1])], axis=1)
        seen.append((np.linalg.norm(MZ - V @ H) / np.linalg.norm(MZ),
                     np.linalg.norm(V.conj().T @ V - np.eye(V.shape[1]))))
        check.V, check.c = V, c

    def matvec(v):
        return oracle.wilson_clover(U, A, kappa, v.reshape(shape)).reshape(-1)

    # one deflated restart after the first cycle of 10; the iterate formed
    # at that restart is the one a run stopped after 10 iterations returns,
    # and its true residual b - M x must equal V c
    fgmresdr.fgmres_dr(matvec, b, 1e-10, 10, 4, 11, None, None, check)
    x, it, _, _ = fgmresdr.fgmres_dr(matvec, b, 1e-10, 10, 4, 10)
    assert len(seen) == 1 and it == 10
    rel, orth = seen[0]
    assert rel < 1e-12 and orth < 1e-12
    r = b.reshape(-1) - matvec(x)
    assert np.linalg.norm(r - check.V @ check.c) / np.linalg.norm(r) < 1e-10


def test_planted_small_eigenvalues_are_deflated():
    rng = np.random.default_rng(0)
    n = 300
    small = np.array([1e-3, 2e-3, 3e-3, 5e-3])
    ev = np.concatenate([small, np.linspace(1, 3, n - 4)]) * np.exp(1j * rng.uniform(-0.3, 0.3, n))
    Q = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))[0]
    Amat = Q @ np.diag(ev) @ Q.conj().T
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    seen = []
    _, it0, _, ok0 = fgmresdr.fgmres_dr(lambda v: Amat @ v, b, 1e-10, 15, 0, 5000)
    _, it4, _, ok4 = fgmresdr.fgmres_dr(lambda v: Amat @ v, b, 1e-10, 15, 4, 5000,
                                        on_restart=lambda V, Z, H, c, th: seen.append(th))
    assert ok0 and ok4
    assert it4 * 4 < it0
    got = np.sort(np.abs(seen[-1]))
    assert np.allclose(got, small, rtol=1e-3)


def test_harmonic_ritz_values_approach_smallest_eigenvalues_of_m():
    """2^4, kappa 0.16 (a small, nearly degenerate pair |lambda| = 0.2528
    from gamma5-hermiticity, next 0.2725): after the solve the kept
    harmonic Ritz values match them (the largest kept ones, not the
    smallest, or a wrong Hsq, would not)."""
    dims = (2, 2, 2, 2)
    kappa = 0.16
    U, A, b = _system(dims, kappa)
    M = _dense(U, A, kappa, dims)
    smallest = np.sort(np.abs(np.linalg.eigvals(M)))[:3]
    seen = []
    oracle.fgmres_dr(U, A, kappa, b, tol=1e-13, m=16, k=6, maxiter=3000,
                     on_restart=lambda V, Z, H, c, th: seen.append(th))
    assert len(seen) > 3
    got = np.sort(np.abs(seen[-1]))[:3]
    assert np.allclose(got, smallest, rtol=3e-3), (got, smallest)


def test_harmonic_ritz_definition():
    """theta, g satisfy Hbar^H Hbar g = theta Hsq^H g and are the smallest."""
    rng = np.random.default_rng(1)
    nz = 9
    hbar = np.triu(rng.standard_normal((nz + 1, nz)) + 1j * rng.standard_normal((nz + 1, nz)), -1)
    theta, g = fgmresdr.harmonic_ritz(hbar, nz, 3)
    hb, hsq = hbar, hbar[:nz]
    for i in range(3):
        lhs = hb.conj().T @ hb @ g[:, i]
        rhs = theta[i] * hsq.conj().T @ g[:, i]
        assert np.linalg.norm(lhs - rhs) < 1e-10 * np.linalg.norm(lhs)
    allv = np.linalg.eigvals(np.linalg.solve(hsq.conj().T, hb.conj().T @ hb))
    assert np.allclose(np.sort(np.abs(theta)), np.sort(np.abs(allv))[:3])


@pytest.mark.parametrize("k", [0, 3])
def test_converges_with_sap(k):
    U, A, b = _system(DIMS, 0.13)
    x, it, res, ok = oracle.fgmres_dr(U, A, 0.13, b, m=10, k=k,
                                      prec=lambda r: oracle.sap(U, A, 0.13, r, (2, 2, 2, 2), 2, 4))
    assert ok and res <= 1e-10
    assert oracle.true_residual(U, A, 0.13, b, x) <= 1e-10
