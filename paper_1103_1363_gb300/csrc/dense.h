// Small dense complex linear algebra on the host for the Krylov solvers:
// an incremental Householder least-squares solver (GMRES's min |c - Hbar y|),
// Gram-Schmidt orthonormalisation, and the harmonic Ritz pairs of the
// deflated restart.  Matrices are column-major: a[i + j * ld].
#pragma once

#include <complex>
#include <vector>

namespace lqcd {
namespace dense {

typedef std::complex<double> cd;

// min |c - H y| with H growing by one column at a time (each new column
// may also add rows below the previous ones).  Keeps the Householder
// reflectors, the triangle R and Q^H c.
class Lsq {
public:
    void reset(const cd* c, int rows);
    // append column col[0..rows-1]; rows >= the current row count
    void add_column(const cd* col, int rows);
    int columns() const { return ncol_; }
    double residual() const;       // |c - H y| at the minimiser
    std::vector<cd> solve() const; // the minimiser y (R y = (Q^H c)[0..ncol-1])

private:
    int ncol_ = 0, nrow_ = 0;
    std::vector<std::vector<cd>> u_;  // reflector j acts on rows j..; u_[j] has nrow at creation - j entries
    std::vector<double> unorm2_;      // |u_j|^2 (0: identity)
    std::vector<std::vector<cd>> r_;  // column j of R, rows 0..j
    std::vector<cd> g_;               // Q^H c (rows 0..nrow-1)
};

// Orthonormal columns in place (modified Gram-Schmidt, two passes).
void orthonormalize(int rows, int cols, cd* a, int lda);

// Harmonic Ritz pairs of M Z = V Hbar, Hbar (nz + 1) x nz with leading
// dimension ldh: Hbar^H Hbar g = theta Hsq^H g, the k of smallest |theta|.
// theta[k], g[nz * k] (unit columns).  False if Hsq is singular or the QR
// iteration does not converge.
bool harmonic_ritz(int nz, const cd* hbar, int ldh, int k, cd* theta, cd* g);

}  // namespace dense
}  // namespace lqcd
