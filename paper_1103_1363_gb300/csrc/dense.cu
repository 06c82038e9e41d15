// Host-only dense complex linear algebra for the Krylov solvers (see
// dense.h).  Compiled by nvcc as plain host code.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <numeric>

#include "dense.h"
#include "internal.h"

namespace lqcd {
namespace dense {

#define A_(a, i, j, ld) (a)[(size_t)(i) + (size_t)(j) * (ld)]

// ------------------------------------------------------------ least squares

void Lsq::reset(const cd* c, int rows)
{
    ncol_ = 0;
    nrow_ = rows;
    u_.clear();
    unorm2_.clear();
    r_.clear();
    g_.assign(c, c + rows);
}

void Lsq::add_column(const cd* col, int rows)
{
    if (rows > nrow_) {
        g_.resize(rows, cd(0.0, 0.0));
        nrow_ = rows;
    }
    std::vector<cd> v(col, col + rows);
    v.resize(nrow_, cd(0.0, 0.0));
    for (int j = 0; j < ncol_; ++j) {  // earlier reflectors
        if (unorm2_[j] == 0.0) continue;
        const std::vector<cd>& u = u_[j];
        cd s(0.0, 0.0);
        for (size_t i = 0; i < u.size(); ++i) s += std::conj(u[i]) * v[j + i];
        const cd f = 2.0 * s / unorm2_[j];
        for (size_t i = 0; i < u.size(); ++i) v[j + i] -= f * u[i];
    }
    const int j = ncol_;
    double tail = 0.0;
    for (int i = j + 1; i < nrow_; ++i) tail += std::norm(v[i]);
    std::vector<cd> rcol(v.begin(), v.begin() + j + 1);
    std::vector<cd> u;
    double un2 = 0.0;
    if (tail > 0.0) {
        const cd alpha = v[j];
        const double xn = std::sqrt(std::norm(alpha) + tail);
        const double aa = std::abs(alpha);
        const cd beta = aa > 0.0 ? -(alpha / aa) * xn : cd(-xn, 0.0);
        u.assign(v.begin() + j, v.end());
        u[0] = alpha - beta;
        for (const cd& e : u) un2 += std::norm(e);
        rcol[j] = beta;
        cd s(0.0, 0.0);
        for (size_t i = 0; i < u.size(); ++i) s += std::conj(u[i]) * g_[j + i];
        const cd f = 2.0 * s / un2;
        for (size_t i = 0; i < u.size(); ++i) g_[j + i] -= f * u[i];
    }
    u_.push_back(u);
    unorm2_.push_back(un2);
    r_.push_back(rcol);
    ++ncol_;
}

double Lsq::residual() const
{
    double s = 0.0;
    for (int i = ncol_; i < nrow_; ++i) s += std::norm(g_[i]);
    return std::sqrt(s);
}

std::vector<cd> Lsq::solve() const
{
    std::vector<cd> y(ncol_);
    for (int i = ncol_ - 1; i >= 0; --i) {
        cd s = g_[i];
        for (int c = i + 1; c < ncol_; ++c) s -= r_[c][i] * y[c];
        y[i] = r_[i][i] != cd(0.0, 0.0) ? s / r_[i][i] : cd(0.0, 0.0);
    }
    return y;
}

// ------------------------------------------------------- orthonormalisation

void orthonormalize(int rows, int cols, cd* a, int lda)
{
    for (int pass = 0; pass < 2; ++pass)
        for (int i = 0; i < cols; ++i) {
            for (int j = 0; j < i; ++j) {
                cd s(0.0, 0.0);
                for (int r = 0; r < rows; ++r) s += std::conj(A_(a, r, j, lda)) * A_(a, r, i, lda);
                for (int r = 0; r < rows; ++r) A_(a, r, i, lda) -= s * A_(a, r, j, lda);
            }
            double n = 0.0;
            for (int r = 0; r < rows; ++r) n += std::norm(A_(a, r, i, lda));
            n = std::sqrt(n);
            if (n > 0.0)
                for (int r = 0; r < rows; ++r) A_(a, r, i, lda) /= n;
        }
}

// ---------------------------------------------------------- eigenproblem

namespace {

// a = Q h Q^H with h upper Hessenberg (Householder reflections); q = Q.
void hessenberg(int n, cd* a, cd* q)
{
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) A_(q, i, j, n) = i == j ? cd(1.0, 0.0) : cd(0.0, 0.0);
    std::vector<cd> u(n);
    for (int j = 0; j + 2 < n; ++j) {
        const int len = n - j - 1;
        double tail = 0.0;
        for (int i = 1; i < len; ++i) tail += std::norm(A_(a, j + 1 + i, j, n));
        if (tail == 0.0) continue;
        const cd alpha = A_(a, j + 1, j, n);
        const double xn = std::sqrt(std::norm(alpha) + tail);
        const double aa = std::abs(alpha);
        const cd beta = aa > 0.0 ? -(alpha / aa) * xn : cd(-xn, 0.0);
        for (int i = 0; i < len; ++i) u[i] = A_(a, j + 1 + i, j, n);
        u[0] = alpha - beta;
        double un2 = 0.0;
        for (int i = 0; i < len; ++i) un2 += std::norm(u[i]);
        // from the left on rows j+1.., columns j..
        for (int c = j; c < n; ++c) {
            cd s(0.0, 0.0);
            for (int i = 0; i < len; ++i) s += std::conj(u[i]) * A_(a, j + 1 + i, c, n);
            const cd f = 2.0 * s / un2;
            for (int i = 0; i < len; ++i) A_(a, j + 1 + i, c, n) -= f * u[i];
        }
        // from the right on columns j+1.. of a and of q
        for (int pass = 0; pass < 2; ++pass) {
            cd* m = pass == 0 ? a : q;
            for (int r = 0; r < n; ++r) {
                cd s(0.0, 0.0);
                for (int i = 0; i < len; ++i) s += A_(m, r, j + 1 + i, n) * u[i];
                const cd f = 2.0 * s / un2;
                for (int i = 0; i < len; ++i) A_(m, r, j + 1 + i, n) -= f * std::conj(u[i]);
            }
        }
        A_(a, j + 1, j, n) = beta;
        for (int i = 1; i < len; ++i) A_(a, j + 1 + i, j, n) = cd(0.0, 0.0);
    }
}

// Givens rotation G = [c s; -conj(s) c] (c real) with G [x; y] = [r; 0].
void givens(cd x, cd y, double& c, cd& s)
{
    const double ax = std::abs(x), ay = std::abs(y);
    if (ay == 0.0) {
        c = 1.0;
        s = cd(0.0, 0.0);
        return;
    }
    if (ax == 0.0) {
        c = 0.0;
        s = cd(1.0, 0.0);
        return;
    }
    const double rho = std::hypot(ax, ay);
    c = ax / rho;
    s = (x / ax) * std::conj(y) / rho;
}

// Schur form of an upper Hessenberg h by shifted QR (Wilkinson shifts,
// Givens sweeps); q accumulates the unitary factor.  False on no convergence.
bool schur(int n, cd* h, cd* q)
{
    double hnorm = 0.0;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i <= std::min(j + 1, n - 1); ++i) hnorm = std::max(hnorm, std::abs(A_(h, i, j, n)));
    if (hnorm == 0.0) return true;
    const double eps = DBL_EPSILON;
    int hi = n - 1, iter = 0, total = 0;
    while (hi > 0) {
        int l = hi;
        while (l > 0) {
            double s = std::abs(A_(h, l - 1, l - 1, n)) + std::abs(A_(h, l, l, n));
            if (s == 0.0) s = hnorm;
            if (std::abs(A_(h, l, l - 1, n)) <= eps * s) {
                A_(h, l, l - 1, n) = cd(0.0, 0.0);
                break;
            }
            --l;
        }
        if (l == hi) {  // h[hi, hi] has converged
            --hi;
            iter = 0;
            continue;
        }
        if (++total > 60 * n) return false;
        ++iter;
        cd mu;
        if (iter % 11 == 0) {  // exceptional shift
            mu = A_(h, hi, hi, n) + cd(0.75 * std::abs(A_(h, hi, hi - 1, n)), 0.0);
        } else {
            const cd a = A_(h, hi - 1, hi - 1, n), b = A_(h, hi - 1, hi, n);
            const cd c = A_(h, hi, hi - 1, n), d = A_(h, hi, hi, n);
            const cd tr2 = 0.5 * (a + d);
            const cd disc = std::sqrt(tr2 * tr2 - (a * d - b * c));
            const cd m1 = tr2 + disc, m2 = tr2 - disc;
            mu = std::abs(m1 - d) < std::abs(m2 - d) ? m1 : m2;
        }
        for (int k = l; k < hi; ++k) {
            const cd x = k == l ? A_(h, l, l, n) - mu : A_(h, k, k - 1, n);
            const cd y = k == l ? A_(h, l + 1, l, n) : A_(h, k + 1, k - 1, n);
            double c;
            cd s;
            givens(x, y, c, s);
            for (int j = std::max(l, k - 1); j < n; ++j) {  // rows k, k+1
                const cd t1 = A_(h, k, j, n), t2 = A_(h, k + 1, j, n);
                A_(h, k, j, n) = c * t1 + s * t2;
                A_(h, k + 1, j, n) = -std::conj(s) * t1 + c * t2;
            }
            const int rmax = std::min(k + 2, hi);
            for (int r = 0; r <= rmax; ++r) {  // columns k, k+1
                const cd t1 = A_(h, r, k, n), t2 = A_(h, r, k + 1, n);
                A_(h, r, k, n) = c * t1 + std::conj(s) * t2;
                A_(h, r, k + 1, n) = -s * t1 + c * t2;
            }
            for (int r = 0; r < n; ++r) {
                const cd t1 = A_(q, r, k, n), t2 = A_(q, r, k + 1, n);
                A_(q, r, k, n) = c * t1 + std::conj(s) * t2;
                A_(q, r, k + 1, n) = -s * t1 + c * t2;
            }
            if (k > l) A_(h, k + 1, k - 1, n) = cd(0.0, 0.0);
        }
    }
    return true;
}

}  // namespace

bool harmonic_ritz(int nz, const cd* hbar, int ldh, int k, cd* theta, cd* g)
{
    const int n = nz;
    // A = Hbar^H Hbar, then K = Hsq^{-H} A by elimination with partial pivoting
    std::vector<cd> A((size_t)n * n), L((size_t)n * n), K((size_t)n * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            cd s(0.0, 0.0);
            for (int r = 0; r <= nz; ++r) s += std::conj(A_(hbar, r, i, ldh)) * A_(hbar, r, j, ldh);
            A_(A.data(), i, j, n) = s;
            A_(L.data(), i, j, n) = std::conj(A_(hbar, j, i, ldh));  // Hsq^H
        }
    K = A;
    double lnorm = 0.0;
    for (const cd& e : L) lnorm = std::max(lnorm, std::abs(e));
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (std::abs(A_(L.data(), r, col, n)) > std::abs(A_(L.data(), piv, col, n))) piv = r;
        if (!(std::abs(A_(L.data(), piv, col, n)) > 1e-14 * lnorm)) return false;
        if (piv != col) {
            for (int j = 0; j < n; ++j) {
                std::swap(A_(L.data(), piv, j, n), A_(L.data(), col, j, n));
                std::swap(A_(K.data(), piv, j, n), A_(K.data(), col, j, n));
            }
        }
        const cd d = A_(L.data(), col, col, n);
        for (int r = col + 1; r < n; ++r) {
            const cd f = A_(L.data(), r, col, n) / d;
            if (f == cd(0.0, 0.0)) continue;
            for (int j = col; j < n; ++j) A_(L.data(), r, j, n) -= f * A_(L.data(), col, j, n);
            for (int j = 0; j < n; ++j) A_(K.data(), r, j, n) -= f * A_(K.data(), col, j, n);
        }
    }
    for (int col = n - 1; col >= 0; --col) {
        const cd d = A_(L.data(), col, col, n);
        for (int j = 0; j < n; ++j) {
            cd s = A_(K.data(), col, j, n);
            for (int c = col + 1; c < n; ++c) s -= A_(L.data(), col, c, n) * A_(K.data(), c, j, n);
            A_(K.data(), col, j, n) = s / d;
        }
    }
    // eigenvalues and vectors of K: Hessenberg form, Schur form
    std::vector<cd> Q((size_t)n * n);
    hessenberg(n, K.data(), Q.data());
    if (!schur(n, K.data(), Q.data())) return false;
    std::vector<int> idx(n);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
        return std::abs(A_(K.data(), a, a, n)) < std::abs(A_(K.data(), b, b, n));
    });
    double tnorm = 0.0;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i <= j; ++i) tnorm = std::max(tnorm, std::abs(A_(K.data(), i, j, n)));
    const double small = DBL_EPSILON * std::max(tnorm, 1e-300);
    std::vector<cd> u(n);
    for (int e = 0; e < k; ++e) {
        const int i = idx[e];
        const cd lam = A_(K.data(), i, i, n);
        theta[e] = lam;
        std::fill(u.begin(), u.end(), cd(0.0, 0.0));
        u[i] = cd(1.0, 0.0);
        for (int r = i - 1; r >= 0; --r) {  // (T - lam) u = 0 above row i
            cd s(0.0, 0.0);
            for (int c = r + 1; c <= i; ++c) s += A_(K.data(), r, c, n) * u[c];
            cd den = A_(K.data(), r, r, n) - lam;
            if (std::abs(den) < small) den = cd(small, 0.0);
            u[r] = -s / den;
        }
        double nrm = 0.0;
        for (int r = 0; r < n; ++r) {
            cd s(0.0, 0.0);
            for (int c = 0; c <= i; ++c) s += A_(Q.data(), r, c, n) * u[c];
            A_(g, r, e, n) = s;
            nrm += std::norm(s);
        }
        nrm = std::sqrt(nrm);
        for (int r = 0; r < n; ++r) A_(g, r, e, n) /= nrm;
    }
    return true;
}

#undef A_

}  // namespace dense
}  // namespace lqcd

extern "C" lqcd_status lqcd_harmonic_ritz(int nz, const double* hbar, int ldh, int k, double* theta, double* g)
{
    using namespace lqcd;
    if (!hbar || !theta || !g || nz < 1 || nz > 256 || k < 1 || k > nz || ldh < nz + 1)
        return fail(LQCD_ERR_INVALID, "lqcd_harmonic_ritz: bad argument");
    try {
        if (!dense::harmonic_ritz(nz, reinterpret_cast<const dense::cd*>(hbar), ldh, k,
                                  reinterpret_cast<dense::cd*>(theta), reinterpret_cast<dense::cd*>(g)))
            return fail(LQCD_ERR_BREAKDOWN, "lqcd_harmonic_ritz: singular leading block or no convergence");
    } catch (...) {
        return fail(LQCD_ERR_NOMEM, "lqcd_harmonic_ritz: host allocation failed");
    }
    return LQCD_OK;
}
