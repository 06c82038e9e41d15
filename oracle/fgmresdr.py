"""Flexible GMRES with deflated restarts, FP64 (test infrastructure).

Sec. 7 of the paper improves SAP-FGMRES on hard systems by deflated
restarts (it cites Morgan, "GMRES with deflated restarting"): at a restart,
approximate eigenvectors of the smallest eigenvalues are kept in the Krylov
basis.  This is that method with the flexible basis of FGMRES (Saad): the
preconditioned vectors z_j = P(v_j) are stored, and every cycle keeps

    M Z_j = V_{j+1} Hbar_j,   V orthonormal,   r = V_{j+1} c - M Z_j y.

Steps, in the order the method takes them:
  1. Arnoldi: z_j = P(v_j), w = M z_j, w orthogonalised against v_0..v_j by
     modified Gram-Schmidt (the entries of column j of Hbar), v_{j+1} = w/|w|.
  2. y minimises |c - Hbar_j y| (a library least-squares solve); the cycle
     ends after m vectors or when that residual reaches tol |b|.
  3. x += Z_j y; the true residual decides convergence.
  4. Deflated restart (k > 0): the harmonic Ritz pairs of the preconditioned
     operator on span(V_j), Hbar^H Hbar g = theta Hsq^H g with Hsq the
     leading j x j block (a library eigensolver), the k of smallest
     |theta| give G_k; P_{k+1} is an orthonormal basis of [G_k; 0] followed
     by the residual coefficients c - Hbar y, and
       V <- V P_{k+1},  Z <- Z P_k,  Hbar <- P_{k+1}^H Hbar P_k,  c <- P_{k+1}^H (c - Hbar y).
     Without deflation (k = 0) the cycle restarts from the true residual.

Plain numpy on full-lattice complex128 vectors; the operator comes from
oracle.c.  Nothing here is shared with the CUDA library.
"""
from __future__ import annotations

import numpy as np


def _orthonormal_columns(a):
    """Orthonormal basis of the columns of a (modified Gram-Schmidt, twice)."""
    q = np.array(a, dtype=complex)
    for _ in range(2):
        for i in range(q.shape[1]):
            for j in range(i):
                q[:, i] -= np.vdot(q[:, j], q[:, i]) * q[:, j]
            q[:, i] /= np.linalg.norm(q[:, i])
    return q


def harmonic_ritz(hbar, nz, k):
    """The k harmonic Ritz pairs of smallest |theta| for M Z = V Hbar with
    Hbar of shape (nz + 1, nz): Hbar^H Hbar g = theta Hsq^H g, Hsq = Hbar[:nz].
    Returns (theta[k], G[nz, k]) with unit-norm columns."""
    hb = hbar[:nz + 1, :nz]
    hsq = hb[:nz, :nz]
    kmat = np.linalg.solve(hsq.conj().T, hb.conj().T @ hb)
    theta, g = np.linalg.eig(kmat)
    order = np.argsort(np.abs(theta), kind="stable")[:k]
    g = g[:, order]
    return theta[order], g / np.linalg.norm(g, axis=0)


def fgmres_dr(matvec, b, tol=1e-10, m=20, k=0, maxiter=100000, prec=None, history=None, on_restart=None):
    """Solve matvec(x) = b.  matvec and prec map flat complex128 vectors to
    flat vectors (prec None: identity).  Returns (x, iterations, true
    relative residual, converged).  history (a list) receives the
    least-squares residual |c - Hbar y|/|b| after every iteration;
    on_restart(V, Z, Hbar, c, theta) is called after each deflated restart
    with the new basis (for tests)."""
    if k >= m:
        raise ValueError("need k < m")
    bv = np.asarray(b, dtype=complex).reshape(-1)
    bn = np.linalg.norm(bv)
    apply_p = (lambda v: v.copy()) if prec is None else (lambda v: np.asarray(prec(v), dtype=complex).reshape(-1))
    x = np.zeros_like(bv)
    r = bv.copy()
    rn = np.linalg.norm(r)
    if rn == 0.0:
        return x, 0, 0.0, True
    V = [r / rn]
    Z = []
    H = np.zeros((m + 1, m), dtype=complex)
    c = np.zeros(m + 1, dtype=complex)
    c[0] = rn
    j = 0
    iters = 0
    while True:
        y = np.zeros(0, dtype=complex)
        while j < m and iters < maxiter:
            z = apply_p(V[j])
            w = matvec(z)
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            V.append(w / H[j + 1, j])
            Z.append(z)
            j += 1
            iters += 1
            y = np.linalg.lstsq(H[:j + 1, :j], c[:j + 1], rcond=None)[0]
            res = np.linalg.norm(c[:j + 1] - H[:j + 1, :j] @ y)
            if history is not None:
                history.append(res / bn)
            if res <= tol * bn:
                break
        if j > 0:
            x = x + np.stack(Z[:j], axis=1) @ y
        true = np.linalg.norm(bv - matvec(x)) / bn
        if true <= tol or iters >= maxiter or not np.isfinite(true):
            return x, iters, true, bool(true <= tol)
        cls = c[:j + 1] - H[:j + 1, :j] @ y
        if k > 0 and j > k:
            theta, gk = harmonic_ritz(H, j, k)
            pk = _orthonormal_columns(np.vstack([gk, np.zeros((1, k))]))
            pk1 = _orthonormal_columns(np.hstack([pk, cls[:, None]]))
            vmat = np.stack(V[:j + 1], axis=1)
            zmat = np.stack(Z[:j], axis=1)
            V = list((vmat @ pk1).T)
            Z = list((zmat @ pk[:j]).T)
            hnew = pk1.conj().T @ H[:j + 1, :j] @ pk[:j]
            cnew = pk1.conj().T @ cls
            H = np.zeros((m + 1, m), dtype=complex)
            c = np.zeros(m + 1, dtype=complex)
            H[:k + 1, :k] = hnew
            c[:k + 1] = cnew
            j = k
            if on_restart is not None:
                on_restart(np.stack(V, axis=1), np.stack(Z, axis=1), H[:k + 1, :k].copy(), c[:k + 1].copy(), theta)
        else:
            r = bv - matvec(x)
            rn = np.linalg.norm(r)
            V = [r / rn]
            Z = []
            H = np.zeros((m + 1, m), dtype=complex)
            c = np.zeros(m + 1, dtype=complex)
            c[0] = rn
            j = 0
