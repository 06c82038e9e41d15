"""The deflation step of FGMRES-DR (lqcd_harmonic_ritz, host code of the
library, no GPU) against the oracle's numpy definition, on Hessenberg
matrices from Arnoldi processes (the matrices the solver feeds it)."""
import numpy as np
import pytest

from oracle import fgmresdr


@pytest.fixture(scope="module")
def lq():
    from paper_1103_1363_gb300 import _build
    _build.build()
    from paper_1103_1363_gb300 import lqcd
    return lqcd


def arnoldi(A, m, rng):
    n = A.shape[0]
    V = np.zeros((n, m + 1), complex)
    H = np.zeros((m + 1, m), complex)
    v = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    V[:, 0] = v / np.linalg.norm(v)
    for j in range(m):
        w = A @ V[:, j]
        for _ in range(2):
            for i in range(j + 1):
                d = np.vdot(V[:, i], w)
                H[i, j] += d
                w -= d * V[:, i]
        H[j + 1, j] = np.linalg.norm(w)
        V[:, j + 1] = w / H[j + 1, j]
    return H


@pytest.mark.parametrize("m,k", [(12, 4), (70, 10), (120, 16)])
def test_matches_oracle_and_finds_planted_eigenvalues(lq, m, k):
    rng = np.random.default_rng(7)
    n = 400
    small = np.array([1e-3, 2e-3, 4e-3])
    ev = np.concatenate([small, np.linspace(0.5, 3, n - 3)]) * np.exp(1j * rng.uniform(-0.5, 0.5, n))
    Q = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))[0]
    H = arnoldi(Q @ np.diag(ev) @ Q.conj().T, m, rng)
    theta, g = lq.lqcd_harmonic_ritz(H, m, k)
    theta0, _ = fgmresdr.harmonic_ritz(H, m, k)
    assert np.allclose(np.sort(np.abs(theta)), np.sort(np.abs(theta0)), rtol=1e-8)
    hsq = H[:m]
    scale = np.linalg.norm(H, 2) ** 2
    for i in range(k):  # the defining equation (backward error vs |Hbar|^2), and unit vectors
        lhs = H.conj().T @ H @ g[:, i]
        assert np.linalg.norm(lhs - theta[i] * hsq.conj().T @ g[:, i]) < 1e-13 * scale
        assert abs(np.linalg.norm(g[:, i]) - 1) < 1e-12
    if m >= 70:  # a long Arnoldi run resolves the planted eigenvalues
        assert np.allclose(np.sort(np.abs(theta))[:3], small, rtol=1e-6)


def test_rejects_bad_arguments(lq):
    with pytest.raises(lq.LqcdError):
        lq.lqcd_harmonic_ritz(np.zeros((5, 4), complex), 4, 5)  # k > nz
    with pytest.raises(lq.LqcdError):
        lq.lqcd_harmonic_ritz(np.zeros((5, 4), complex), 4, 2)  # singular leading block
