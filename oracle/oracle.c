/*
 * FP64 CPU oracle for the even-odd preconditioned Wilson(-clover) Dirac
 * operator and its Krylov solvers.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA library; the two meet only through
 * the seeded inputs of the ``synth`` module.
 *
 * Everything here is written for a reader checking it by eye against the
 * definitions: plain loops over sites, full 4x4 gamma matrices (no spin
 * projection tricks), full 12x12 clover matrices per site, textbook CG and
 * flexible GCR.  C99 ``double complex`` throughout.
 *
 * Definitions (the paper states the problem M phi = b, M^dag M phi = b in
 * Sec. 3, Eq. (1), and solves it with CG on the normal equations and on the
 * even-odd Schur complement in Sec. 5; the operator itself is the standard
 * Wilson / Sheikholeslami-Wohlert one that the paper takes as known):
 *
 *   H psi(x) = sum_mu (1 - g_mu) U_mu(x) psi(x+mu) + (1 + g_mu) U_mu(x-mu)^dag psi(x-mu)
 *   A(x)     = 1 + i kappa csw sum_{mu<nu} sigma_{mu nu} Fhat_{mu nu}(x)
 *   M        = A - kappa H
 *   Mhat     = A_oo - kappa^2 H_oe A_ee^{-1} H_eo      (odd-site Schur complement)
 *
 * with DeGrand-Rossi (chiral) gamma matrices, sigma_{mu nu} = (i/2)[g_mu, g_nu],
 * Fhat = (Q - Q^dag)/8 made traceless, Q the sum of the four plaquette leaves
 * in the mu-nu plane, periodic boundaries in x, y, z and a factor -1 on every
 * fermion hop across the t boundary when t_antiperiodic is set.
 *
 * Layouts (canonical): site s = ((t*Lz + z)*Ly + y)*Lx + x with
 * dims = {Lx, Ly, Lz, Lt}; spinor psi[s][spin][colour]; gauge U[s][mu][a][b];
 * clover A[s][12][12] with row/column index spin*3 + colour.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* ------------------------------------------------------------------ lattice */

static long volume(const int d[4]) { return (long)d[0] * d[1] * d[2] * d[3]; }

static void coords(const int d[4], long s, int c[4])
{
    c[0] = (int)(s % d[0]); s /= d[0];
    c[1] = (int)(s % d[1]); s /= d[1];
    c[2] = (int)(s % d[2]); s /= d[2];
    c[3] = (int)s;
}

static long site_index(const int d[4], const int c[4])
{
    return ((long)(c[3] * d[2] + c[2]) * d[1] + c[1]) * d[0] + c[0];
}

static int parity_of(const int c[4]) { return (c[0] + c[1] + c[2] + c[3]) & 1; }

/* neighbour x + dir*mu_hat (dir = +1 or -1), periodic wrap */
static long neighbour(const int d[4], const int c[4], int mu, int dir)
{
    int n[4] = {c[0], c[1], c[2], c[3]};
    n[mu] = (n[mu] + dir + d[mu]) % d[mu];
    return site_index(d, n);
}

/* fermion boundary factor of the hop from x to x + dir*mu_hat */
static double hop_sign(const int d[4], const int c[4], int mu, int dir, int tanti)
{
    if (!tanti || mu != 3) return 1.0;
    if (dir > 0 && c[3] == d[3] - 1) return -1.0;
    if (dir < 0 && c[3] == 0) return -1.0;
    return 1.0;
}

/* ------------------------------------------------------------ gamma algebra */

/* DeGrand-Rossi basis, mu = 0..3 for x, y, z, t; mu = 4 gives gamma_5. */
void oracle_gamma(int mu, cplx g[4][4])
{
    memset(g, 0, 16 * sizeof(cplx));
    switch (mu) {
    case 0:
        g[0][3] = I;  g[1][2] = I;  g[2][1] = -I; g[3][0] = -I; break;
    case 1:
        g[0][3] = -1; g[1][2] = 1;  g[2][1] = 1;  g[3][0] = -1; break;
    case 2:
        g[0][2] = I;  g[1][3] = -I; g[2][0] = -I; g[3][1] = I;  break;
    case 3:
        g[0][2] = 1;  g[1][3] = 1;  g[2][0] = 1;  g[3][1] = 1;  break;
    default: {
        /* gamma_5 = g_x g_y g_z g_t, formed by matrix products */
        cplx a[4][4], b[4][4], t[4][4];
        oracle_gamma(0, a);
        for (int m = 1; m < 4; ++m) {
            oracle_gamma(m, b);
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j) {
                    cplx acc = 0;
                    for (int k = 0; k < 4; ++k) acc += a[i][k] * b[k][j];
                    t[i][j] = acc;
                }
            memcpy(a, t, sizeof(a));
        }
        memcpy(g, a, sizeof(a));
    }
    }
}

/* sigma_{mu nu} = (i/2) (g_mu g_nu - g_nu g_mu) */
void oracle_sigma(int mu, int nu, cplx s[4][4])
{
    cplx a[4][4], b[4][4];
    oracle_gamma(mu, a);
    oracle_gamma(nu, b);
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            cplx ab = 0, ba = 0;
            for (int k = 0; k < 4; ++k) { ab += a[i][k] * b[k][j]; ba += b[i][k] * a[k][j]; }
            s[i][j] = 0.5 * I * (ab - ba);
        }
}

/* --------------------------------------------------------- small matrices */

static void mat3_mul(const cplx *a, const cplx *b, cplx *c) /* c = a b */
{
    cplx t[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            cplx acc = 0;
            for (int k = 0; k < 3; ++k) acc += a[3 * i + k] * b[3 * k + j];
            t[3 * i + j] = acc;
        }
    memcpy(c, t, sizeof(t));
}

static void mat3_dag(const cplx *a, cplx *c)
{
    cplx t[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) t[3 * i + j] = conj(a[3 * j + i]);
    memcpy(c, t, sizeof(t));
}

static const cplx *link(const cplx *U, long s, int mu) { return U + (s * 4 + mu) * 9; }

/* -------------------------------------------------------- hopping term H */

/*
 * Contribution of one hop to out(x): out += sign * (1 + pm*g_mu) * V * psi(y)
 * where V is the colour matrix (U_mu(x) forward, U_mu(x-mu)^dag backward),
 * pm = -1 forward and +1 backward.  The spin matrix is the full 4x4 one.
 */
static void add_hop(cplx out[4][3], const cplx gmu[4][4], double pm, const cplx *V,
                    const cplx *psi, double sign)
{
    cplx vpsi[4][3]; /* colour rotation of every spin component */
    for (int s = 0; s < 4; ++s)
        for (int a = 0; a < 3; ++a) {
            cplx acc = 0;
            for (int b = 0; b < 3; ++b) acc += V[3 * a + b] * psi[3 * s + b];
            vpsi[s][a] = acc;
        }
    for (int s = 0; s < 4; ++s)
        for (int a = 0; a < 3; ++a) {
            cplx acc = 0;
            for (int r = 0; r < 4; ++r) {
                cplx proj = (s == r ? 1.0 : 0.0) + pm * gmu[s][r];
                acc += proj * vpsi[r][a];
            }
            out[s][a] += sign * acc;
        }
}

static void hop_site(const int d[4], int tanti, const cplx *U, const cplx *in, long x,
                     cplx out[4][3])
{
    int c[4];
    coords(d, x, c);
    memset(out, 0, 12 * sizeof(cplx));
    for (int mu = 0; mu < 4; ++mu) {
        cplx g[4][4], Vd[9];
        oracle_gamma(mu, g);
        long xf = neighbour(d, c, mu, +1);
        long xb = neighbour(d, c, mu, -1);
        /* forward: (1 - g_mu) U_mu(x) psi(x + mu) */
        add_hop(out, g, -1.0, link(U, x, mu), in + 12 * xf, hop_sign(d, c, mu, +1, tanti));
        /* backward: (1 + g_mu) U_mu(x - mu)^dag psi(x - mu) */
        mat3_dag(link(U, xb, mu), Vd);
        add_hop(out, g, +1.0, Vd, in + 12 * xb, hop_sign(d, c, mu, -1, tanti));
    }
}

/* out = H in over the whole lattice */
void oracle_hop(const int d[4], int tanti, const cplx *U, const cplx *in, cplx *out)
{
    long V = volume(d);
#pragma omp parallel for schedule(static)
    for (long x = 0; x < V; ++x) hop_site(d, tanti, U, in, x, (cplx(*)[3])(out + 12 * x));
}

/* out[i] = (H in)(sites[i]) for a list of sites (sampled checks on big lattices) */
void oracle_hop_sites(const int d[4], int tanti, const cplx *U, const cplx *in,
                      const long *sites, long n, cplx *out)
{
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) hop_site(d, tanti, U, in, sites[i], (cplx(*)[3])(out + 12 * i));
}

/* -------------------------------------------------------------- clover */

/* The four plaquette leaves in the mu-nu plane at x, all circulating the
 * same way (mu then nu), summed into Q. */
static void clover_leaves(const int d[4], const cplx *U, long x, int mu, int nu, cplx Q[9])
{
    int c[4], cm[4], cn[4];
    coords(d, x, c);
    long xpm = neighbour(d, c, mu, +1), xmm = neighbour(d, c, mu, -1);
    long xpn = neighbour(d, c, nu, +1), xmn = neighbour(d, c, nu, -1);
    coords(d, xmm, cm);
    coords(d, xmn, cn);
    long xmm_pn = neighbour(d, cm, nu, +1); /* x - mu + nu */
    long xmm_mn = neighbour(d, cm, nu, -1); /* x - mu - nu */
    long xmn_pm = neighbour(d, cn, mu, +1); /* x + mu - nu */
    cplx t[9], a[9], L[9];
    memset(Q, 0, 9 * sizeof(cplx));
    /* U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag */
    mat3_mul(link(U, x, mu), link(U, xpm, nu), t);
    mat3_dag(link(U, xpn, mu), a); mat3_mul(t, a, t);
    mat3_dag(link(U, x, nu), a);   mat3_mul(t, a, L);
    for (int i = 0; i < 9; ++i) Q[i] += L[i];
    /* U_nu(x) U_mu(x-mu+nu)^dag U_nu(x-mu)^dag U_mu(x-mu) */
    mat3_dag(link(U, xmm_pn, mu), a); mat3_mul(link(U, x, nu), a, t);
    mat3_dag(link(U, xmm, nu), a);    mat3_mul(t, a, t);
    mat3_mul(t, link(U, xmm, mu), L);
    for (int i = 0; i < 9; ++i) Q[i] += L[i];
    /* U_mu(x-mu)^dag U_nu(x-mu-nu)^dag U_mu(x-mu-nu) U_nu(x-nu) */
    mat3_dag(link(U, xmm, mu), t);
    mat3_dag(link(U, xmm_mn, nu), a); mat3_mul(t, a, t);
    mat3_mul(t, link(U, xmm_mn, mu), t);
    mat3_mul(t, link(U, xmn, nu), L);
    for (int i = 0; i < 9; ++i) Q[i] += L[i];
    /* U_nu(x-nu)^dag U_mu(x-nu) U_nu(x+mu-nu) U_mu(x)^dag */
    mat3_dag(link(U, xmn, nu), t);
    mat3_mul(t, link(U, xmn, mu), t);
    mat3_mul(t, link(U, xmn_pm, nu), t);
    mat3_dag(link(U, x, mu), a); mat3_mul(t, a, L);
    for (int i = 0; i < 9; ++i) Q[i] += L[i];
}

static const int PLANES[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};

/* F[s][plane][3][3], planes ordered (x,y),(x,z),(x,t),(y,z),(y,t),(z,t):
 * Fhat = (Q - Q^dag)/8 with its trace removed. */
void oracle_field_strength(const int d[4], const cplx *U, cplx *F)
{
    long V = volume(d);
#pragma omp parallel for schedule(static)
    for (long x = 0; x < V; ++x)
        for (int p = 0; p < 6; ++p) {
            cplx Q[9], *f = F + (x * 6 + p) * 9;
            clover_leaves(d, U, x, PLANES[p][0], PLANES[p][1], Q);
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) f[3 * i + j] = (Q[3 * i + j] - conj(Q[3 * j + i])) / 8.0;
            cplx tr = (f[0] + f[4] + f[8]) / 3.0;
            f[0] -= tr; f[4] -= tr; f[8] -= tr;
        }
}

/* A[s][12][12] = 1 + i kappa csw sum_{mu<nu} sigma_{mu nu} (x) Fhat_{mu nu}(x) */
void oracle_clover(const int d[4], const cplx *U, double kappa, double csw, cplx *A)
{
    long V = volume(d);
    cplx *F = malloc(sizeof(cplx) * 54 * V);
    oracle_field_strength(d, U, F);
    cplx sig[6][4][4];
    for (int p = 0; p < 6; ++p) oracle_sigma(PLANES[p][0], PLANES[p][1], sig[p]);
#pragma omp parallel for schedule(static)
    for (long x = 0; x < V; ++x) {
        cplx *a = A + x * 144;
        for (int i = 0; i < 144; ++i) a[i] = 0;
        for (int i = 0; i < 12; ++i) a[13 * i] = 1.0;
        for (int p = 0; p < 6; ++p) {
            const cplx *f = F + (x * 6 + p) * 9;
            for (int s = 0; s < 4; ++s)
                for (int r = 0; r < 4; ++r)
                    for (int ca = 0; ca < 3; ++ca)
                        for (int cb = 0; cb < 3; ++cb)
                            a[(s * 3 + ca) * 12 + r * 3 + cb] +=
                                I * kappa * csw * sig[p][s][r] * f[3 * ca + cb];
        }
    }
    free(F);
}

/* Gauss-Jordan inversion with partial pivoting of nsites n x n matrices.
 * Returns the number of matrices whose largest available pivot fell below
 * 1e-12 (their output is left as NaN). */
int oracle_invert_site_matrices(long nsites, int n, const cplx *A, cplx *Ainv)
{
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (long x = 0; x < nsites; ++x) {
        cplx *m = malloc(sizeof(cplx) * n * 2 * n);
        const cplx *a = A + x * n * n;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < 2 * n; ++j)
                m[i * 2 * n + j] = j < n ? a[i * n + j] : (j - n == i ? 1.0 : 0.0);
        int ok = 1;
        for (int col = 0; col < n && ok; ++col) {
            int piv = col;
            for (int i = col + 1; i < n; ++i)
                if (cabs(m[i * 2 * n + col]) > cabs(m[piv * 2 * n + col])) piv = i;
            if (cabs(m[piv * 2 * n + col]) < 1e-12) { ok = 0; break; }
            if (piv != col)
                for (int j = 0; j < 2 * n; ++j) {
                    cplx t = m[col * 2 * n + j];
                    m[col * 2 * n + j] = m[piv * 2 * n + j];
                    m[piv * 2 * n + j] = t;
                }
            cplx inv = 1.0 / m[col * 2 * n + col];
            for (int j = 0; j < 2 * n; ++j) m[col * 2 * n + j] *= inv;
            for (int i = 0; i < n; ++i) {
                if (i == col) continue;
                cplx f = m[i * 2 * n + col];
                if (f == 0) continue;
                for (int j = 0; j < 2 * n; ++j) m[i * 2 * n + j] -= f * m[col * 2 * n + j];
            }
        }
        cplx *o = Ainv + x * n * n;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) o[i * n + j] = ok ? m[i * 2 * n + n + j] : NAN;
        bad += !ok;
        free(m);
    }
    return bad;
}

/* out(x) = A(x) in(x) for per-site 12x12 matrices */
void oracle_apply_site_matrices(long nsites, const cplx *A, const cplx *in, cplx *out)
{
#pragma omp parallel for schedule(static)
    for (long x = 0; x < nsites; ++x) {
        const cplx *a = A + x * 144, *v = in + 12 * x;
        cplx t[12];
        for (int i = 0; i < 12; ++i) {
            cplx acc = 0;
            for (int j = 0; j < 12; ++j) acc += a[12 * i + j] * v[j];
            t[i] = acc;
        }
        memcpy(out + 12 * x, t, sizeof(t));
    }
}

/* ----------------------------------------------------- Wilson-clover M */

void oracle_gamma5(long nsites, const cplx *in, cplx *out)
{
    cplx g5[4][4];
    oracle_gamma(4, g5);
#pragma omp parallel for schedule(static)
    for (long x = 0; x < nsites; ++x) {
        cplx t[12];
        for (int s = 0; s < 4; ++s)
            for (int a = 0; a < 3; ++a) {
                cplx acc = 0;
                for (int r = 0; r < 4; ++r) acc += g5[s][r] * in[12 * x + 3 * r + a];
                t[3 * s + a] = acc;
            }
        memcpy(out + 12 * x, t, sizeof(t));
    }
}

/* out = M in = A in - kappa H in; A == NULL means A = 1 (csw = 0) */
void oracle_wilson_clover(const int d[4], int tanti, const cplx *U, const cplx *A, double kappa,
                          const cplx *in, cplx *out)
{
    long V = volume(d);
    cplx *h = malloc(sizeof(cplx) * 12 * V);
    oracle_hop(d, tanti, U, in, h);
    if (A) oracle_apply_site_matrices(V, A, in, out);
    else memcpy(out, in, sizeof(cplx) * 12 * V);
    for (long i = 0; i < 12 * V; ++i) out[i] -= kappa * h[i];
    free(h);
}

/* out = M^dag in, using M^dag = g5 M g5 (gamma5-hermiticity) */
void oracle_wilson_clover_dag(const int d[4], int tanti, const cplx *U, const cplx *A,
                              double kappa, const cplx *in, cplx *out)
{
    long V = volume(d);
    cplx *t = malloc(sizeof(cplx) * 12 * V);
    oracle_gamma5(V, in, t);
    oracle_wilson_clover(d, tanti, U, A, kappa, t, out);
    oracle_gamma5(V, out, out);
    free(t);
}

/* zero the spinor on every site whose parity differs from `keep` */
static void restrict_parity(const int d[4], cplx *v, int keep)
{
    long V = volume(d);
    for (long x = 0; x < V; ++x) {
        int c[4];
        coords(d, x, c);
        if (parity_of(c) != keep) memset(v + 12 * x, 0, 12 * sizeof(cplx));
    }
}

/*
 * Odd-site Schur complement on full-lattice arrays (even sites of `in` are
 * ignored, even sites of `out` are zero):
 *   out_o = A_oo in_o - kappa^2 H_oe A_ee^{-1} H_eo in_o
 * A == NULL means A = 1.
 */
void oracle_schur(const int d[4], int tanti, const cplx *U, const cplx *A, const cplx *Ainv,
                  double kappa, const cplx *in, cplx *out)
{
    long V = volume(d);
    cplx *po = malloc(sizeof(cplx) * 12 * V), *te = malloc(sizeof(cplx) * 12 * V);
    cplx *uo = malloc(sizeof(cplx) * 12 * V);
    memcpy(po, in, sizeof(cplx) * 12 * V);
    restrict_parity(d, po, 1);
    oracle_hop(d, tanti, U, po, te); /* H_eo p_o lands on even sites */
    restrict_parity(d, te, 0);
    if (Ainv) oracle_apply_site_matrices(V, Ainv, te, te);
    oracle_hop(d, tanti, U, te, uo); /* H_oe (...) lands on odd sites */
    restrict_parity(d, uo, 1);
    if (A) oracle_apply_site_matrices(V, A, po, out);
    else memcpy(out, po, sizeof(cplx) * 12 * V);
    for (long i = 0; i < 12 * V; ++i) out[i] -= kappa * kappa * uo[i];
    restrict_parity(d, out, 1);
    free(po); free(te); free(uo);
}

/* out = Mhat^dag in = g5 Mhat g5 in */
void oracle_schur_dag(const int d[4], int tanti, const cplx *U, const cplx *A, const cplx *Ainv,
                      double kappa, const cplx *in, cplx *out)
{
    long V = volume(d);
    cplx *t = malloc(sizeof(cplx) * 12 * V);
    oracle_gamma5(V, in, t);
    oracle_schur(d, tanti, U, A, Ainv, kappa, t, out);
    oracle_gamma5(V, out, out);
    free(t);
}

/* ------------------------------------------------------------- BLAS-1 */

static double norm2(long n, const cplx *v)
{
    double s = 0;
    for (long i = 0; i < n; ++i) s += creal(v[i]) * creal(v[i]) + cimag(v[i]) * cimag(v[i]);
    return s;
}

static cplx cdot(long n, const cplx *a, const cplx *b) /* <a, b> = sum conj(a) b */
{
    cplx s = 0;
    for (long i = 0; i < n; ++i) s += conj(a[i]) * b[i];
    return s;
}

/* true relative residual |b - M x| / |b| of the full operator */
double oracle_true_residual(const int d[4], int tanti, const cplx *U, const cplx *A, double kappa,
                            const cplx *b, const cplx *x)
{
    long n = 12 * volume(d);
    cplx *r = malloc(sizeof(cplx) * n);
    oracle_wilson_clover(d, tanti, U, A, kappa, x, r);
    for (long i = 0; i < n; ++i) r[i] = b[i] - r[i];
    double res = sqrt(norm2(n, r) / norm2(n, b));
    free(r);
    return res;
}

/* ------------------------------------------------------------------ CG */

/*
 * Conjugate gradient (Hestenes-Stiefel) on a Hermitian positive-definite
 * operator K = O^dag O, starting from x (in/out).  `op(ctx, in, out, dag)`
 * applies O (dag = 0) or O^dag (dag = 1).  Iterates until the recursive
 * residual of the normal equations drops below `inner_tol` relative to
 * |O^dag b|, or until maxiter.  Returns the number of iterations.
 */
typedef void (*op_fn)(void *ctx, const cplx *in, cplx *out, int dag);

static int cg_normal(op_fn op, void *ctx, long n, const cplx *b, cplx *x, double inner_tol,
                     int maxiter)
{
    cplx *r = malloc(sizeof(cplx) * n), *p = malloc(sizeof(cplx) * n);
    cplx *q = malloc(sizeof(cplx) * n), *s = malloc(sizeof(cplx) * n);
    /* r = O^dag (b - O x) */
    op(ctx, x, q, 0);
    for (long i = 0; i < n; ++i) q[i] = b[i] - q[i];
    op(ctx, q, r, 1);
    op(ctx, b, s, 1);
    double target = inner_tol * inner_tol * norm2(n, s);
    memcpy(p, r, sizeof(cplx) * n);
    double rr = norm2(n, r);
    int k = 0;
    while (k < maxiter && rr > target) {
        op(ctx, p, q, 0);              /* q = O p */
        double alpha = rr / norm2(n, q); /* <p, O^dag O p> = |O p|^2 */
        op(ctx, q, s, 1);              /* s = O^dag O p */
        for (long i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * s[i]; }
        double rr_new = norm2(n, r);
        double beta = rr_new / rr;
        rr = rr_new;
        for (long i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
        ++k;
    }
    free(r); free(p); free(q); free(s);
    return k;
}

struct full_ctx { const int *d; int tanti; const cplx *U, *A; double kappa; };

static void full_op(void *vctx, const cplx *in, cplx *out, int dag)
{
    struct full_ctx *c = vctx;
    if (dag) oracle_wilson_clover_dag(c->d, c->tanti, c->U, c->A, c->kappa, in, out);
    else oracle_wilson_clover(c->d, c->tanti, c->U, c->A, c->kappa, in, out);
}

/*
 * CG on the normal equations of the full operator (CGNR), x0 = 0.  The stop
 * test is the true residual |b - M x|/|b| <= tol; the normal-equation
 * residual only triggers that check (at tol/10, tightened if the check
 * fails).  Returns 0 on convergence, 1 otherwise; *iters and *true_res out.
 */
int oracle_cgnr(const int d[4], int tanti, const cplx *U, const cplx *A, double kappa,
                const cplx *b, cplx *x, double tol, int maxiter, int *iters, double *true_res)
{
    long n = 12 * volume(d);
    struct full_ctx c = {d, tanti, U, A, kappa};
    memset(x, 0, sizeof(cplx) * n);
    int total = 0, idle = 0;
    double inner = tol * 0.1, res = 1.0;
    while (total < maxiter) {
        int k = cg_normal(full_op, &c, n, b, x, inner, maxiter - total);
        total += k;
        res = oracle_true_residual(d, tanti, U, A, kappa, b, x);
        if (res <= tol || isnan(res)) break;
        if (k == 0 && ++idle > 3) break; /* no further progress possible */
        inner *= 0.1;
    }
    *iters = total;
    *true_res = res;
    return res <= tol ? 0 : 1;
}

struct schur_ctx { const int *d; int tanti; const cplx *U, *A, *Ainv; double kappa; };

static void schur_op(void *vctx, const cplx *in, cplx *out, int dag)
{
    struct schur_ctx *c = vctx;
    if (dag) oracle_schur_dag(c->d, c->tanti, c->U, c->A, c->Ainv, c->kappa, in, out);
    else oracle_schur(c->d, c->tanti, c->U, c->A, c->Ainv, c->kappa, in, out);
}

/*
 * Even-odd preconditioned solve of M x = b (full-lattice b, x):
 *   bhat_o = b_o + kappa H_oe A_ee^{-1} b_e
 *   CG on Mhat^dag Mhat x_o = Mhat^dag bhat_o
 *   x_e    = A_ee^{-1} (b_e + kappa H_eo x_o)
 * Stop test: true residual of the full system <= tol.  A/Ainv NULL = no clover.
 */
int oracle_eo_cg(const int d[4], int tanti, const cplx *U, const cplx *A, const cplx *Ainv,
                 double kappa, const cplx *b, cplx *x, double tol, int maxiter, int *iters,
                 double *true_res)
{
    long V = volume(d), n = 12 * V;
    cplx *be = malloc(sizeof(cplx) * n), *bo = malloc(sizeof(cplx) * n);
    cplx *bhat = malloc(sizeof(cplx) * n), *t = malloc(sizeof(cplx) * n);
    cplx *xo = calloc(n, sizeof(cplx));
    memcpy(be, b, sizeof(cplx) * n); restrict_parity(d, be, 0);
    memcpy(bo, b, sizeof(cplx) * n); restrict_parity(d, bo, 1);
    /* bhat_o */
    if (Ainv) oracle_apply_site_matrices(V, Ainv, be, t); else memcpy(t, be, sizeof(cplx) * n);
    oracle_hop(d, tanti, U, t, bhat);
    restrict_parity(d, bhat, 1);
    for (long i = 0; i < n; ++i) bhat[i] = bo[i] + kappa * bhat[i];
    struct schur_ctx c = {d, tanti, U, A, Ainv, kappa};
    int total = 0, idle = 0;
    double inner = tol * 0.1, res = 1.0;
    while (total < maxiter) {
        int k = cg_normal(schur_op, &c, n, bhat, xo, inner, maxiter - total);
        total += k;
        /* reconstruct x_e and test the full system */
        oracle_hop(d, tanti, U, xo, t);
        restrict_parity(d, t, 0);
        for (long i = 0; i < n; ++i) t[i] = be[i] + kappa * t[i];
        if (Ainv) oracle_apply_site_matrices(V, Ainv, t, t);
        restrict_parity(d, t, 0);
        for (long i = 0; i < n; ++i) x[i] = t[i] + xo[i];
        res = oracle_true_residual(d, tanti, U, A, kappa, b, x);
        if (res <= tol || isnan(res)) break;
        if (k == 0 && ++idle > 3) break;
        inner *= 0.1;
    }
    *iters = total;
    *true_res = res;
    free(be); free(bo); free(bhat); free(t); free(xo);
    return res <= tol ? 0 : 1;
}

/* Run a fixed number of CG iterations on the Schur normal equations from
 * x_o = 0 (used to time the oracle and to make training pairs).  b is the
 * odd-site right-hand side bhat (even sites ignored); x_o returned. */
void oracle_schur_cg_iters(const int d[4], int tanti, const cplx *U, const cplx *A,
                           const cplx *Ainv, double kappa, const cplx *bhat, cplx *xo, int niter)
{
    long n = 12 * volume(d);
    struct schur_ctx c = {d, tanti, U, A, Ainv, kappa};
    cplx *bo = malloc(sizeof(cplx) * n);
    memcpy(bo, bhat, sizeof(cplx) * n);
    restrict_parity(d, bo, 1);
    memset(xo, 0, sizeof(cplx) * n);
    cg_normal(schur_op, &c, n, bo, xo, 0.0, niter);
    free(bo);
}

/* Run a fixed number of CGNR iterations on the full operator from x = 0. */
void oracle_cgnr_iters(const int d[4], int tanti, const cplx *U, const cplx *A, double kappa,
                       const cplx *b, cplx *x, int niter)
{
    long n = 12 * volume(d);
    struct full_ctx c = {d, tanti, U, A, kappa};
    memset(x, 0, sizeof(cplx) * n);
    cg_normal(full_op, &c, n, b, x, 0.0, niter);
}

/* ---------------------------------------------- gauge-equivariant network */

/*
 * Parallel-transport convolution layer (hops h = 0 .. 8):
 *   out(x)[co][s] = sum_h sum_{ci, r} W_h[co*4+s][ci*4+r] (T_h in)(x)[ci][r]
 * with colour carried along by the transport
 *   T_0 psi(x)      = psi(x)
 *   T_{2mu+1} psi(x) = U_mu(x) psi(x+mu)             (times the fermion t sign)
 *   T_{2mu+2} psi(x) = U_mu(x-mu)^dag psi(x-mu)       (times the fermion t sign)
 * Field layout: in[s][ci][spin][colour], out[s][co][spin][colour];
 * W[h][4*cout][4*cin] complex.
 */
static void transport(const int d[4], int tanti, const cplx *U, int nch, const cplx *in, long x,
                      int h, cplx *res /* [nch][4][3] */)
{
    int c[4];
    coords(d, x, c);
    if (h == 0) { memcpy(res, in + x * nch * 12, sizeof(cplx) * nch * 12); return; }
    int mu = (h - 1) / 2, fwd = ((h - 1) % 2) == 0;
    long y = neighbour(d, c, mu, fwd ? +1 : -1);
    double sg = hop_sign(d, c, mu, fwd ? +1 : -1, tanti);
    cplx V[9];
    if (fwd) memcpy(V, link(U, x, mu), sizeof(V));
    else mat3_dag(link(U, y, mu), V);
    const cplx *v = in + y * nch * 12;
    for (int k = 0; k < nch * 4; ++k)
        for (int a = 0; a < 3; ++a) {
            cplx acc = 0;
            for (int b = 0; b < 3; ++b) acc += V[3 * a + b] * v[3 * k + b];
            res[3 * k + a] = sg * acc;
        }
}

/* adjoint of T_h: T_{2mu+1}^dag = T_{2mu+2} and vice versa, T_0^dag = T_0 */
static int adjoint_hop(int h) { return h == 0 ? 0 : (h % 2 == 1 ? h + 1 : h - 1); }

void oracle_net_layer(const int d[4], int tanti, const cplx *U, int cin, int cout, const cplx *W,
                      const cplx *in, cplx *out)
{
    long V = volume(d);
    int nin = 4 * cin, nout = 4 * cout;
#pragma omp parallel
    {
        cplx *tr = malloc(sizeof(cplx) * nin * 3);
#pragma omp for schedule(static)
        for (long x = 0; x < V; ++x) {
            cplx *o = out + x * nout * 3;
            memset(o, 0, sizeof(cplx) * nout * 3);
            for (int h = 0; h < 9; ++h) {
                transport(d, tanti, U, cin, in, x, h, tr);
                const cplx *w = W + (long)h * nout * nin;
                for (int i = 0; i < nout; ++i)
                    for (int j = 0; j < nin; ++j)
                        for (int a = 0; a < 3; ++a) o[3 * i + a] += w[i * nin + j] * tr[3 * j + a];
            }
        }
        free(tr);
    }
}

/*
 * Adjoint layer (gradient with respect to the input):
 *   gin = sum_h T_h^dag W_h^dag gout
 * computed as, for each site x, sum_h T_{adj(h)} applied to the field
 * W_h^dag gout, which is the definition of the adjoint of a sum of
 * (site-local matrix) x (transport) terms.
 */
void oracle_net_layer_adj(const int d[4], int tanti, const cplx *U, int cin, int cout,
                          const cplx *W, const cplx *gout, cplx *gin)
{
    long V = volume(d);
    int nin = 4 * cin, nout = 4 * cout;
    cplx *wg = malloc(sizeof(cplx) * V * nin * 3);
    memset(gin, 0, sizeof(cplx) * V * nin * 3);
    for (int h = 0; h < 9; ++h) {
        const cplx *w = W + (long)h * nout * nin;
#pragma omp parallel for schedule(static)
        for (long x = 0; x < V; ++x) {
            const cplx *g = gout + x * nout * 3;
            cplx *o = wg + x * nin * 3;
            for (int j = 0; j < nin; ++j)
                for (int a = 0; a < 3; ++a) {
                    cplx acc = 0;
                    for (int i = 0; i < nout; ++i) acc += conj(w[i * nin + j]) * g[3 * i + a];
                    o[3 * j + a] = acc;
                }
        }
        int ha = adjoint_hop(h);
#pragma omp parallel
        {
            cplx *tr = malloc(sizeof(cplx) * nin * 3);
#pragma omp for schedule(static)
            for (long x = 0; x < V; ++x) {
                transport(d, tanti, U, cin, wg, x, ha, tr);
                for (int k = 0; k < nin * 3; ++k) gin[x * nin * 3 + k] += tr[k];
            }
            free(tr);
        }
    }
    free(wg);
}

/*
 * Weight gradient: for a real loss L with G_out = dL/dRe(out) + i dL/dIm(out),
 *   G_{W_h}[i][j] = sum_x sum_colour G_out(x)[i][a] conj((T_h in)(x)[j][a])
 * which equals dL/dRe(W) + i dL/dIm(W) (= 2 dL/dconj(W)).
 */
void oracle_net_layer_wgrad(const int d[4], int tanti, const cplx *U, int cin, int cout,
                            const cplx *in, const cplx *gout, cplx *gW)
{
    long V = volume(d);
    int nin = 4 * cin, nout = 4 * cout;
    memset(gW, 0, sizeof(cplx) * 9 * nout * nin);
    cplx *tr = malloc(sizeof(cplx) * nin * 3);
    for (int h = 0; h < 9; ++h) {
        cplx *gw = gW + (long)h * nout * nin;
        for (long x = 0; x < V; ++x) {
            transport(d, tanti, U, cin, in, x, h, tr);
            const cplx *g = gout + x * nout * 3;
            for (int i = 0; i < nout; ++i)
                for (int j = 0; j < nin; ++j) {
                    cplx acc = 0;
                    for (int a = 0; a < 3; ++a) acc += g[3 * i + a] * conj(tr[3 * j + a]);
                    gw[i * nin + j] += acc;
                }
        }
    }
    free(tr);
}

/* ----------------------------------------------------------------- SAP */

/*
 * Schwarz alternating procedure as a preconditioner (Sec. 5): the lattice is
 * divided into non-overlapping blocks of extent bs[mu] (every lattice extent
 * a multiple of bs[mu] with an even number >= 2 of blocks per direction), and
 * the blocks are coloured like a checkerboard by the parity of the sum of
 * their block coordinates.  Starting from z = 0, each of ncycle cycles
 * solves on all colour-0 blocks, updates the residual, solves on all
 * colour-1 blocks and updates the residual.  A block solve is nmr iterations
 * of minimal residual (MR) on the block operator with Dirichlet boundary
 * conditions, M_B = P_B M P_B (P_B restricts to the block), starting from 0:
 *   q = M_B rho;  alpha = <q, rho> / <q, q>;  delta += alpha rho;  rho -= alpha q.
 * Output z approximates M^{-1} r.
 */
static int block_colour(const int d[4], const int bs[4], const int c[4])
{
    (void)d;
    return (c[0] / bs[0] + c[1] / bs[1] + c[2] / bs[2] + c[3] / bs[3]) & 1;
}

static long block_id(const int d[4], const int bs[4], const int c[4])
{
    const int nb0 = d[0] / bs[0], nb1 = d[1] / bs[1], nb2 = d[2] / bs[2];
    return ((long)(c[3] / bs[3] * nb2 + c[2] / bs[2]) * nb1 + c[1] / bs[1]) * nb0 + c[0] / bs[0];
}

void oracle_sap(const int d[4], int tanti, const cplx *U, const cplx *A, double kappa, const int bs[4],
                int ncycle, int nmr, const cplx *r, cplx *z)
{
    long V = volume(d), n = 12 * V;
    long nblocks = V / ((long)bs[0] * bs[1] * bs[2] * bs[3]);
    long *bid = malloc(sizeof(long) * V);
    int *col = malloc(sizeof(int) * V);
    for (long x = 0; x < V; ++x) {
        int c[4];
        coords(d, x, c);
        bid[x] = block_id(d, bs, c);
        col[x] = block_colour(d, bs, c);
    }
    cplx *rho = malloc(sizeof(cplx) * n), *q = malloc(sizeof(cplx) * n), *t = malloc(sizeof(cplx) * n);
    cplx *blk = malloc(sizeof(cplx) * n);
    memset(z, 0, sizeof(cplx) * n);
    for (int cy = 0; cy < ncycle; ++cy)
        for (int colour = 0; colour < 2; ++colour) {
            /* residual of the current z */
            oracle_wilson_clover(d, tanti, U, A, kappa, z, t);
            for (long i = 0; i < n; ++i) rho[i] = r[i] - t[i];
            for (long b = 0; b < nblocks; ++b) {
                /* is this block of the colour being solved? */
                int is_col = -1;
                for (long x = 0; x < V && is_col < 0; ++x)
                    if (bid[x] == b) is_col = col[x] == colour;
                if (!is_col) continue;
                /* rho_B and delta on the block */
                memset(blk, 0, sizeof(cplx) * n);
                for (long x = 0; x < V; ++x)
                    if (bid[x] == b) memcpy(blk + 12 * x, rho + 12 * x, 12 * sizeof(cplx));
                cplx *delta = t;
                memset(delta, 0, sizeof(cplx) * n);
                for (int it = 0; it < nmr; ++it) {
                    oracle_wilson_clover(d, tanti, U, A, kappa, blk, q); /* blk is zero off the block */
                    for (long x = 0; x < V; ++x)
                        if (bid[x] != b) memset(q + 12 * x, 0, 12 * sizeof(cplx));
                    cplx qr = cdot(n, q, blk);
                    double qq = norm2(n, q);
                    if (qq == 0.0) break;
                    cplx alpha = qr / qq;
                    for (long i = 0; i < n; ++i) { delta[i] += alpha * blk[i]; blk[i] -= alpha * q[i]; }
                }
                for (long x = 0; x < V; ++x)
                    if (bid[x] == b)
                        for (int k = 0; k < 12; ++k) z[12 * x + k] += delta[12 * x + k];
            }
        }
    free(bid); free(col); free(rho); free(q); free(t); free(blk);
}

/* ---------------------------------------------------------------- FGCR */

/*
 * Flexible GCR(k) with right preconditioning on the full operator M
 * (Sec. 5: FGCR stores two vectors per iteration, so it is restarted;
 * mixed precision is iterative refinement at the restart - here all FP64).
 * Per iteration: z_k = P(r), w_k = M z_k, w_k and z_k orthogonalised against
 * the previous w_j by modified Gram-Schmidt, x += a z_k, r -= a w_k with
 * a = <w_k, r>/<w_k, w_k>.  At each restart r = b - M x is recomputed.
 * `prec(pctx, r, z)` applies the preconditioner; NULL means identity.
 * Stops when |b - M x|/|b| <= tol.  Returns 0 on convergence.
 */
typedef void (*prec_fn)(void *pctx, const cplx *r, cplx *z);

int oracle_fgcr(const int d[4], int tanti, const cplx *U, const cplx *A, double kappa,
                const cplx *b, cplx *x, double tol, int nkrylov, int maxiter, prec_fn prec,
                void *pctx, int *iters, double *true_res)
{
    long n = 12 * volume(d);
    cplx *r = malloc(sizeof(cplx) * n);
    cplx *z = malloc(sizeof(cplx) * n * nkrylov), *w = malloc(sizeof(cplx) * n * nkrylov);
    double *ww = malloc(sizeof(double) * nkrylov);
    memset(x, 0, sizeof(cplx) * n);
    double bn = sqrt(norm2(n, b));
    int total = 0;
    double res = 1.0;
    while (total < maxiter) {
        oracle_wilson_clover(d, tanti, U, A, kappa, x, r);
        for (long i = 0; i < n; ++i) r[i] = b[i] - r[i];
        res = sqrt(norm2(n, r)) / bn;
        if (res <= tol || isnan(res)) break;
        for (int k = 0; k < nkrylov && total < maxiter; ++k) {
            cplx *zk = z + n * k, *wk = w + n * k;
            if (prec) prec(pctx, r, zk); else memcpy(zk, r, sizeof(cplx) * n);
            oracle_wilson_clover(d, tanti, U, A, kappa, zk, wk);
            for (int j = 0; j < k; ++j) {
                cplx *wj = w + n * j, *zj = z + n * j;
                cplx c = cdot(n, wj, wk) / ww[j];
                for (long i = 0; i < n; ++i) { wk[i] -= c * wj[i]; zk[i] -= c * zj[i]; }
            }
            ww[k] = norm2(n, wk);
            cplx a = cdot(n, wk, r) / ww[k];
            for (long i = 0; i < n; ++i) { x[i] += a * zk[i]; r[i] -= a * wk[i]; }
            ++total;
            if (sqrt(norm2(n, r)) / bn <= tol * 0.5) break;
        }
    }
    oracle_wilson_clover(d, tanti, U, A, kappa, x, r);
    for (long i = 0; i < n; ++i) r[i] = b[i] - r[i];
    res = sqrt(norm2(n, r)) / bn;
    *iters = total;
    *true_res = res;
    free(r); free(z); free(w); free(ww);
    return res <= tol ? 0 : 1;
}

/* Threads an OpenMP loop of this library runs on (1 without OpenMP): the
 * core count a timed oracle run reports. */
int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of later OpenMP loops (timing on a given number of cores; no
 * effect on any result beyond the summation order of the reductions). */
void oracle_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
