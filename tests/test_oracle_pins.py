"""Pins of the FP64 CPU oracle against mathematics (no GPU).

Each test fixes a part of the oracle by something other than the oracle
itself: the Clifford algebra, the free-field momentum-space closed form,
gamma5-hermiticity, gauge covariance, a dense matrix built from an
independent element formula, a dense LAPACK solve, and the closed form of
the clover term in a constant abelian field.  A plausible slip (a dropped
term, a flipped sign, a transposed link, a wrong neighbour) fails at least
one of them.
"""
import itertools

import numpy as np
import pytest

import oracle
import synth

KAPPA = 0.12


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def site_index(dims, x, y, z, t):
    lx, ly, lz, lt = dims
    return ((t * lz + z) * ly + y) * lx + x


# ------------------------------------------------------------------ gamma table

def test_gamma_clifford_and_hermitian():
    g = [oracle.gamma(m) for m in range(4)]
    for m in range(4):
        assert np.allclose(g[m], g[m].conj().T)
        for n in range(4):
            assert np.allclose(g[m] @ g[n] + g[n] @ g[m], 2.0 * np.eye(4) * (m == n))
    g5 = oracle.gamma(4)
    # chiral basis: gamma_5 = diag(1, 1, -1, -1)
    assert np.allclose(g5, np.diag([1, 1, -1, -1]))
    assert np.allclose(g5, g[0] @ g[1] @ g[2] @ g[3])


def test_sigma_hand_values():
    """sigma_{mu nu} = (i/2)[g_mu, g_nu]; entries worked out by hand from the
    DeGrand-Rossi matrices (sigma_xy = i g_x g_y, etc.)."""
    assert np.allclose(oracle.sigma(0, 1), np.diag([1, -1, 1, -1]))
    assert np.allclose(oracle.sigma(2, 3), np.diag([-1, 1, 1, -1]))
    s03 = np.zeros((4, 4))
    s03[0, 1] = s03[1, 0] = -1
    s03[2, 3] = s03[3, 2] = 1
    assert np.allclose(oracle.sigma(0, 3), s03)
    for m, n in itertools.combinations(range(4), 2):
        s = oracle.sigma(m, n)
        assert np.allclose(s, s.conj().T)
        assert np.allclose(s @ oracle.gamma(4), oracle.gamma(4) @ s)  # block diagonal


# ---------------------------------------------------------- O-T1: free field

@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 4, 6, 8)])
def test_free_field_closed_form(dims):
    """Unit links: a plane wave e^{ipx} u obeys M psi = 2 kappa D(p) psi with
    D(p) = m + sum_mu [i g_mu sin p_mu + (1 - cos p_mu)], m = 1/(2 kappa) - 4,
    p_i = 2 pi n / L_i, p_t = (2n + 1) pi / L_t (antiperiodic).  The 12x12
    symbol is read off every momentum, and its eigenvalues are also checked
    against 2 kappa [m + sum(1 - cos p)] +- i 2 kappa sqrt(sum sin^2 p)."""
    kappa = 0.13
    m = 1.0 / (2 * kappa) - 4.0
    lx, ly, lz, lt = dims
    U = synth.unit_gauge(dims)
    g = [oracle.gamma(mu) for mu in range(4)]
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx),
                             indexing="ij")
    rng = np.random.default_rng(5)
    moms = list(itertools.product(range(lx), range(ly), range(lz), range(lt)))
    for (nx, ny, nz, nt) in [moms[i] for i in rng.choice(len(moms), 12, replace=False)]:
        p = np.array([2 * np.pi * nx / lx, 2 * np.pi * ny / ly, 2 * np.pi * nz / lz,
                      (2 * nt + 1) * np.pi / lt])
        phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
        Dp = (m + np.sum(1 - np.cos(p))) * np.eye(4, dtype=complex)
        for mu in range(4):
            Dp = Dp + 1j * np.sin(p[mu]) * g[mu]
        for s in range(4):
            for c in range(3):
                u = np.zeros((4, 3), complex)
                u[s, c] = 1
                psi = phase[..., None, None] * u
                out = oracle.wilson_clover(U, None, kappa, psi)
                want = phase[..., None, None] * (2 * kappa * np.einsum("ij,jc->ic", Dp, u))
                assert rel(out, want) < 1e-13
        ev = np.linalg.eigvals(2 * kappa * Dp)
        ev = ev[np.argsort(ev.imag)]
        a = 2 * kappa * (m + np.sum(1 - np.cos(p)))
        b = 2 * kappa * np.sqrt(np.sum(np.sin(p) ** 2))
        assert np.allclose(ev, np.array([a - 1j * b, a - 1j * b, a + 1j * b, a + 1j * b]),
                           atol=1e-13)


def test_free_field_clover_vanishes():
    U = synth.unit_gauge((4, 4, 4, 4))
    A = oracle.clover(U, 0.13, 1.7)
    assert np.allclose(A, np.broadcast_to(np.eye(12), A.shape), atol=1e-15)


# ------------------------------------------------- O-T2: gamma5-hermiticity

def _inner(a, b):
    return np.vdot(a.reshape(-1), b.reshape(-1))


def test_gamma5_hermiticity():
    dims = (4, 4, 4, 6)
    U = synth.haar_gauge(dims, 11)
    A = oracle.clover(U, KAPPA, 1.3)
    Ainv, bad = oracle.invert_site_matrices(A)
    assert bad == 0
    phi = synth.gaussian_spinor(dims, 1)
    psi = synth.gaussian_spinor(dims, 2)
    for AA in (None, A):
        lhs = _inner(phi, oracle.wilson_clover(U, AA, KAPPA, psi, dag=True))
        rhs = _inner(oracle.wilson_clover(U, AA, KAPPA, phi), psi)
        assert abs(lhs - rhs) / abs(rhs) < 1e-13
    lhs = _inner(phi, oracle.schur(U, A, Ainv, KAPPA, psi, dag=True))
    rhs = _inner(oracle.schur(U, A, Ainv, KAPPA, phi), psi)
    assert abs(lhs - rhs) / abs(rhs) < 1e-13
    # A itself is Hermitian and commutes with gamma5
    assert np.allclose(A, np.swapaxes(A.conj(), -1, -2), atol=1e-14)
    g5 = np.kron(oracle.gamma(4), np.eye(3))
    assert np.allclose(A @ g5, g5 @ A, atol=1e-14)


# ---------------------------------------------------- O-T3: gauge covariance

def test_gauge_covariance():
    """U'_mu(x) = g(x) U_mu(x) g(x+mu)^dag, psi' = g psi  =>  M[U'] psi' = g M[U] psi
    (hopping term, clover term, Schur complement and its dagger)."""
    dims = (4, 6, 4, 8)
    U = synth.haar_gauge(dims, 21)
    G = synth.random_gauge_transform(dims, 22)
    Up = np.empty_like(U)
    for mu in range(4):
        axis = 3 - mu  # canonical array axes are (t, z, y, x)
        Gf = np.roll(G, -1, axis=axis)  # g(x + mu)
        Up[..., mu, :, :] = G @ U[..., mu, :, :] @ np.swapaxes(Gf.conj(), -1, -2)
    psi = synth.gaussian_spinor(dims, 23)
    gpsi = np.einsum("...ab,...sb->...sa", G, psi)
    A = oracle.clover(U, KAPPA, 1.0)
    Ap = oracle.clover(Up, KAPPA, 1.0)
    out = oracle.wilson_clover(Up, Ap, KAPPA, gpsi)
    want = np.einsum("...ab,...sb->...sa", G, oracle.wilson_clover(U, A, KAPPA, psi))
    assert rel(out, want) < 1e-13
    Ai, _ = oracle.invert_site_matrices(A)
    Api, _ = oracle.invert_site_matrices(Ap)
    out = oracle.schur(Up, Ap, Api, KAPPA, gpsi, dag=True)
    want = np.einsum("...ab,...sb->...sa", G, oracle.schur(U, A, Ai, KAPPA, psi, dag=True))
    assert rel(out, want) < 1e-13
    # field strength transforms adjointly
    F = oracle.field_strength(U)
    Fp = oracle.field_strength(Up)
    want = G[..., None, :, :] @ F @ np.swapaxes(G.conj(), -1, -2)[..., None, :, :]
    assert np.abs(Fp - want).max() < 1e-13


# ------------------------------------- O-T4 / O-T7: dense brute force on tiny lattices

def dense_from_elements(U, A, kappa, dims, tanti=True):
    """M(x,s,a; y,r,b) written element by element from the definition:
    A(x)_{sa,rb} delta_xy - kappa [ (1-g_mu)_{sr} U_mu(x)_{ab} sign delta_{y,x+mu}
                                   + (1+g_mu)_{sr} conj(U_mu(x-mu)_{ba}) sign delta_{y,x-mu} ],
    accumulating (on extent-2 directions x+mu and x-mu coincide)."""
    lx, ly, lz, lt = dims
    V = lx * ly * lz * lt
    g = [oracle.gamma(mu) for mu in range(4)]
    M = np.zeros((V * 12, V * 12), complex)
    ext = (lx, ly, lz, lt)
    for t, z, y, x in itertools.product(range(lt), range(lz), range(ly), range(lx)):
        c = [x, y, z, t]
        i = site_index(dims, *c)
        M[12 * i:12 * i + 12, 12 * i:12 * i + 12] += (np.eye(12) if A is None
                                                       else A[t, z, y, x])
        for mu in range(4):
            f = list(c)
            f[mu] = (c[mu] + 1) % ext[mu]
            b = list(c)
            b[mu] = (c[mu] - 1) % ext[mu]
            sf = -1.0 if (tanti and mu == 3 and c[3] == lt - 1) else 1.0
            sb = -1.0 if (tanti and mu == 3 and c[3] == 0) else 1.0
            jf = site_index(dims, *f)
            jb = site_index(dims, *b)
            Uf = U[t, z, y, x, mu]
            Ub = U[b[3], b[2], b[1], b[0], mu]
            M[12 * i:12 * i + 12, 12 * jf:12 * jf + 12] -= kappa * sf * np.kron(
                np.eye(4) - g[mu], Uf)
            M[12 * i:12 * i + 12, 12 * jb:12 * jb + 12] -= kappa * sb * np.kron(
                np.eye(4) + g[mu], Ub.conj().T)
    return M


def dense_from_operator(apply, dims):
    lx, ly, lz, lt = dims
    n = lx * ly * lz * lt * 12
    cols = []
    for j in range(n):
        e = np.zeros(n, complex)
        e[j] = 1
        cols.append(apply(e.reshape(lt, lz, ly, lx, 4, 3)).reshape(-1))
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("dims,csw", [((2, 2, 2, 2), 0.0), ((2, 2, 2, 2), 1.0),
                                      ((2, 2, 2, 4), 1.0)])
def test_dense_brute_force(dims, csw):
    U = synth.haar_gauge(dims, 31)
    A = oracle.clover(U, KAPPA, csw) if csw else None
    Md = dense_from_elements(U, A, KAPPA, dims)
    Mo = dense_from_operator(lambda v: oracle.wilson_clover(U, A, KAPPA, v), dims)
    assert np.abs(Md - Mo).max() < 1e-14
    # gamma5 M gamma5 = M^dag, densely
    Mdag = dense_from_operator(lambda v: oracle.wilson_clover(U, A, KAPPA, v, dag=True), dims)
    assert np.abs(Mdag - Md.conj().T).max() < 1e-14


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 2, 4, 2)])
def test_dense_schur_complement(dims):
    """Mhat = M_oo - M_oe M_ee^{-1} M_eo from the dense matrix (LAPACK inverse)."""
    U = synth.haar_gauge(dims, 41)
    A = oracle.clover(U, KAPPA, 1.0)
    Ainv, _ = oracle.invert_site_matrices(A)
    Md = dense_from_elements(U, A, KAPPA, dims)
    lx, ly, lz, lt = dims
    par = np.array([(x + y + z + t) & 1 for t, z, y, x in
                    itertools.product(range(lt), range(lz), range(ly), range(lx))])
    idx = np.repeat(par, 12)
    o = np.where(idx == 1)[0]
    e = np.where(idx == 0)[0]
    S = Md[np.ix_(o, o)] - Md[np.ix_(o, e)] @ np.linalg.inv(Md[np.ix_(e, e)]) @ Md[np.ix_(e, o)]
    So = dense_from_operator(lambda v: oracle.schur(U, A, Ainv, KAPPA, v), dims)
    assert np.abs(So[np.ix_(o, o)] - S).max() < 1e-13
    assert np.abs(So[np.ix_(e, o)]).max() == 0.0


def test_clover_inverse_matches_lapack():
    dims = (4, 4, 4, 4)
    U = synth.haar_gauge(dims, 51)
    A = oracle.clover(U, 0.135, 1.5)
    Ainv, bad = oracle.invert_site_matrices(A)
    assert bad == 0
    assert np.abs(Ainv - np.linalg.inv(A)).max() < 1e-12


# ---------------------------------------------------------------- O-T6: clover

@pytest.mark.parametrize("mu,nu,k", [(0, 1, 1), (1, 3, 1), (2, 3, 3)])
def test_clover_constant_abelian_field(mu, nu, k):
    """U_nu(x) = exp(i theta x_mu T), T = diag(1,-1,0), theta = 2 pi k / L_mu, all
    other links 1: every plaquette in the mu-nu plane is exp(i theta T), so
    Fhat_{mu nu} = i sin(theta) T on every site, the other planes vanish, and
    A = 1 - kappa csw sin(theta) sigma_{mu nu} (x) T."""
    dims = (4, 4, 6, 8)
    L = dims[mu]
    theta = 2 * np.pi * k / L
    T = np.diag([1.0, -1.0, 0.0])
    U = synth.unit_gauge(dims)
    lt, lz, ly, lx = dims[3], dims[2], dims[1], dims[0]
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx),
                             indexing="ij")
    xm = [x, y, z, t][mu]
    ph = np.exp(1j * theta * xm)
    U[..., nu, 0, 0] = ph
    U[..., nu, 1, 1] = ph.conj()
    F = oracle.field_strength(U)
    planes = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
    for pidx, (a, b) in enumerate(planes):
        want = 1j * np.sin(theta) * T if (a, b) == (mu, nu) else np.zeros((3, 3))
        assert np.abs(F[..., pidx, :, :] - want).max() < 1e-14
    kappa, csw = 0.13, 1.1
    A = oracle.clover(U, kappa, csw)
    sig = oracle.sigma(mu, nu)
    want = np.eye(12) - kappa * csw * np.sin(theta) * np.kron(sig, T)
    assert np.abs(A - want).max() < 1e-14
    if (mu, nu) == (0, 1):
        # hand value: sigma_xy[0,0] = +1, T[0,0] = +1
        assert abs(A[0, 0, 0, 0, 0, 0] - (1 - kappa * csw * np.sin(theta))) < 1e-14


def test_clover_singular_at_kappa_csw_sin_theta_one():
    """In the constant abelian field A = 1 - kappa csw sin(theta) sigma (x) T
    has the eigenvalue 1 - kappa csw sin(theta) (sigma and T both have the
    eigenvalue 1), so csw = 1 / (kappa sin theta) makes every site's clover
    matrix singular; the oracle's inverse reports every site, and none at
    90 % of that csw."""
    dims = (4, 4, 6, 8)
    U = synth.constant_abelian_gauge(dims, 0, 1, 1)
    theta = 2 * np.pi / dims[0]
    kappa = 0.13
    csw = 1.0 / (kappa * np.sin(theta))
    _, bad = oracle.invert_site_matrices(oracle.clover(U, kappa, csw))
    assert bad == int(np.prod(dims))
    _, bad = oracle.invert_site_matrices(oracle.clover(U, kappa, 0.9 * csw))
    assert bad == 0


def test_field_strength_properties():
    dims = (4, 4, 4, 4)
    U = synth.smooth_gauge(dims, 0.5, 61)
    F = oracle.field_strength(U)
    assert np.abs(F + np.swapaxes(F.conj(), -1, -2)).max() < 1e-15  # anti-Hermitian
    assert np.abs(np.trace(F, axis1=-2, axis2=-1)).max() < 1e-15  # traceless


# ---------------------------------------------------------- O-T5: solvers

def test_solvers_against_dense_solve():
    """CGNR, even-odd CG and FGCR against a dense LAPACK solve on 4^4."""
    dims = (4, 4, 4, 4)
    U = synth.haar_gauge(dims, 1)
    b = synth.gaussian_spinor(dims, 0)
    for csw in (0.0, 1.0):
        A = oracle.clover(U, KAPPA, csw) if csw else None
        Md = dense_from_operator(lambda v: oracle.wilson_clover(U, A, KAPPA, v), dims)
        xd = np.linalg.solve(Md, b.reshape(-1)).reshape(b.shape)
        sv = np.linalg.svd(Md, compute_uv=False)
        cond = sv[0] / sv[-1]
        x, it, res, ok = oracle.cgnr(U, A, KAPPA, b, maxiter=2000)
        assert ok and res <= 1e-10
        assert rel(x, xd) <= cond * 1e-10
        if A is not None:
            Ai, _ = oracle.invert_site_matrices(A)
        else:
            Ai = None
        x, it, res, ok = oracle.eo_cg(U, A, Ai, KAPPA, b, maxiter=2000)
        assert ok and res <= 1e-10
        assert rel(x, xd) <= cond * 1e-10
        x, it, res, ok = oracle.fgcr(U, A, KAPPA, b, nkrylov=8, maxiter=2000)
        assert ok and res <= 1e-10
        assert rel(x, xd) <= cond * 1e-10


def test_true_residual_definition():
    dims = (4, 4, 4, 4)
    U = synth.haar_gauge(dims, 1)
    b = synth.gaussian_spinor(dims, 0)
    x = synth.gaussian_spinor(dims, 3)
    r = b - oracle.wilson_clover(U, None, KAPPA, x)
    assert abs(oracle.true_residual(U, None, KAPPA, b, x)
               - np.linalg.norm(r) / np.linalg.norm(b)) < 1e-14
