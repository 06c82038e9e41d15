"""Pins of the oracle's Schwarz alternating procedure (no GPU): exact block
solves leave no residual on the last-solved colour, the block solve agrees
with a dense LAPACK solve of the Dirichlet block matrix, SAP is gauge
covariant, and SAP-preconditioned FGCR converges."""
import itertools

import numpy as np

import oracle
import synth

DIMS = (4, 4, 4, 8)
BS = (2, 2, 2, 4)
KAPPA = 0.12


def block_mask(dims, bs, colour):
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    return ((x // bs[0] + y // bs[1] + z // bs[2] + t // bs[3]) % 2) == colour


def test_exact_block_solves_clear_last_colour():
    U = synth.smooth_gauge(DIMS, 0.5, 71)
    A = oracle.clover(U, KAPPA, 1.0)
    r = synth.gaussian_spinor(DIMS, 72)
    z = oracle.sap(U, A, KAPPA, r, BS, ncycle=1, nmr=300)
    res = r - oracle.wilson_clover(U, A, KAPPA, z)
    black = block_mask(DIMS, BS, 1)
    assert np.linalg.norm(res[black]) / np.linalg.norm(r) < 1e-12
    assert np.linalg.norm(res[~black]) / np.linalg.norm(r) > 1e-3  # the other colour is not solved


def test_block_solve_matches_dense_dirichlet_solve():
    """One half cycle with converged MR on colour 0 = M_B^{-1} r_B on every
    colour-0 block, M_B built densely from the operator restricted to B."""
    U = synth.haar_gauge(DIMS, 73)
    A = oracle.clover(U, KAPPA, 1.0)
    r = synth.gaussian_spinor(DIMS, 74)
    r0 = np.where(block_mask(DIMS, BS, 0)[..., None, None], r, 0)  # source only on colour 0
    z = oracle.sap(U, A, KAPPA, r0, BS, ncycle=1, nmr=400)
    # block at origin: sites with x<2, y<2, z<2, t<4
    sel = np.zeros(DIMS[::-1], bool)
    sel[:4, :2, :2, :2] = True
    idx = np.nonzero(sel.reshape(-1))[0]
    n = len(idx) * 12
    cols = []
    for j in range(n):
        e = np.zeros((np.prod(DIMS), 12), complex)
        e[idx[j // 12], j % 12] = 1
        out = oracle.wilson_clover(U, A, KAPPA, e.reshape(DIMS[::-1] + (4, 3))).reshape(-1, 12)
        cols.append(out[idx].reshape(-1))
    MB = np.stack(cols, axis=1)
    rb = r.reshape(-1, 12)[idx].reshape(-1)
    want = np.linalg.solve(MB, rb)
    got = z.reshape(-1, 12)[idx].reshape(-1)
    # colour-1 blocks see only a zero residual in the second half cycle, so
    # z on colour-0 blocks is exactly the first half cycle's block solve
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-10


def test_sap_gauge_covariant():
    U = synth.haar_gauge(DIMS, 75)
    G = synth.random_gauge_transform(DIMS, 76)
    Up = np.empty_like(U)
    for mu in range(4):
        Gf = np.roll(G, -1, axis=3 - mu)
        Up[..., mu, :, :] = G @ U[..., mu, :, :] @ np.swapaxes(Gf.conj(), -1, -2)
    r = synth.gaussian_spinor(DIMS, 77)
    gr = np.einsum("...ab,...sb->...sa", G, r)
    A, Ap = oracle.clover(U, KAPPA, 1.0), oracle.clover(Up, KAPPA, 1.0)
    z = oracle.sap(U, A, KAPPA, r, BS, ncycle=2, nmr=4)
    zp = oracle.sap(Up, Ap, KAPPA, gr, BS, ncycle=2, nmr=4)
    want = np.einsum("...ab,...sb->...sa", G, z)
    assert np.linalg.norm(zp - want) / np.linalg.norm(want) < 1e-12


def test_sap_fgcr_converges_faster_than_identity():
    U = synth.smooth_gauge(DIMS, 0.5, 78)
    A = oracle.clover(U, KAPPA, 1.0)
    b = synth.gaussian_spinor(DIMS, 79)
    _, it_id, res_id, ok_id = oracle.fgcr(U, A, KAPPA, b, nkrylov=16, maxiter=2000)
    x, it_s, res_s, ok_s = oracle.fgcr(U, A, KAPPA, b, nkrylov=16, maxiter=2000,
                                       prec=lambda r: oracle.sap(U, A, KAPPA, r, BS, ncycle=1, nmr=4))
    assert ok_id and ok_s and res_s <= 1e-10
    assert oracle.true_residual(U, A, KAPPA, b, x) <= 1e-10
    assert it_s < it_id
