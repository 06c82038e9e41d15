// Clover term A(x) = 1 + i kappa csw sum_{mu<nu} sigma_{mu nu} Fhat_{mu nu}(x):
// build from the four-leaf field strength, invert, round to every held
// precision, and apply.  Build and inversion run in FP64 (the FP64 residual
// of the mixed-precision solver needs A to FP64 accuracy).  The leaf
// products are per-site SU(3) matrix products, the memory-bound kernel the
// paper uses as its example of the information-flow model (Sec. 3, Eq. (3)).
#include "internal.h"

namespace lqcd {

// 3x3 complex matrices as 18 doubles, row-major, (re, im) interleaved.
__device__ __forceinline__ void m3_mul(const double* a, const double* b, double* out)  // out = a b
{
    double t[18];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            double re = 0, im = 0;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const double ar = a[2 * (3 * i + k)], ai = a[2 * (3 * i + k) + 1];
                const double br = b[2 * (3 * k + j)], bi = b[2 * (3 * k + j) + 1];
                re += ar * br - ai * bi;
                im += ar * bi + ai * br;
            }
            t[2 * (3 * i + j)] = re;
            t[2 * (3 * i + j) + 1] = im;
        }
#pragma unroll
    for (int k = 0; k < 18; ++k) out[k] = t[k];
}

__device__ __forceinline__ void m3_dag(const double* a, double* out)
{
    double t[18];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            t[2 * (3 * i + j)] = a[2 * (3 * j + i)];
            t[2 * (3 * i + j) + 1] = -a[2 * (3 * j + i) + 1];
        }
#pragma unroll
    for (int k = 0; k < 18; ++k) out[k] = t[k];
}

__device__ __forceinline__ void link_at(const Geom& g, const void* gauge, const int c[4], int mu, double u[18])
{
    const int full = full_index(g, c);
    const int par = (c[0] + c[1] + c[2] + c[3]) & 1;
    GaugeIO<P64, 18>::load(gauge, g.stride, par, mu, full >> 1, u);
}

__device__ __forceinline__ void shifted(const Geom& g, const int c[4], int mu, int d, int out[4])
{
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
    out[mu] = (out[mu] + d + g.L[mu]) % g.L[mu];
}

// Sum of the four plaquette leaves in the mu-nu plane, all circulating mu -> nu.
__device__ void leaves(const Geom& g, const void* gauge, const int c[4], int mu, int nu, double Q[18])
{
    int pm[4], mm[4], pn[4], mn[4], mm_pn[4], mm_mn[4], pm_mn[4];
    shifted(g, c, mu, +1, pm);
    shifted(g, c, mu, -1, mm);
    shifted(g, c, nu, +1, pn);
    shifted(g, c, nu, -1, mn);
    shifted(g, mm, nu, +1, mm_pn);
    shifted(g, mm, nu, -1, mm_mn);
    shifted(g, pm, nu, -1, pm_mn);
    double a[18], b[18], t[18];
#pragma unroll
    for (int k = 0; k < 18; ++k) Q[k] = 0;
    // U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
    link_at(g, gauge, c, mu, a);
    link_at(g, gauge, pm, nu, b);
    m3_mul(a, b, t);
    link_at(g, gauge, pn, mu, a);
    m3_dag(a, a);
    m3_mul(t, a, t);
    link_at(g, gauge, c, nu, a);
    m3_dag(a, a);
    m3_mul(t, a, t);
#pragma unroll
    for (int k = 0; k < 18; ++k) Q[k] += t[k];
    // U_nu(x) U_mu(x-mu+nu)^dag U_nu(x-mu)^dag U_mu(x-mu)
    link_at(g, gauge, c, nu, a);
    link_at(g, gauge, mm_pn, mu, b);
    m3_dag(b, b);
    m3_mul(a, b, t);
    link_at(g, gauge, mm, nu, a);
    m3_dag(a, a);
    m3_mul(t, a, t);
    link_at(g, gauge, mm, mu, a);
    m3_mul(t, a, t);
#pragma unroll
    for (int k = 0; k < 18; ++k) Q[k] += t[k];
    // U_mu(x-mu)^dag U_nu(x-mu-nu)^dag U_mu(x-mu-nu) U_nu(x-nu)
    link_at(g, gauge, mm, mu, a);
    m3_dag(a, a);
    link_at(g, gauge, mm_mn, nu, b);
    m3_dag(b, b);
    m3_mul(a, b, t);
    link_at(g, gauge, mm_mn, mu, a);
    m3_mul(t, a, t);
    link_at(g, gauge, mn, nu, a);
    m3_mul(t, a, t);
#pragma unroll
    for (int k = 0; k < 18; ++k) Q[k] += t[k];
    // U_nu(x-nu)^dag U_mu(x-nu) U_nu(x+mu-nu) U_mu(x)^dag
    link_at(g, gauge, mn, nu, a);
    m3_dag(a, a);
    link_at(g, gauge, mn, mu, b);
    m3_mul(a, b, t);
    link_at(g, gauge, pm_mn, nu, a);
    m3_mul(t, a, t);
    link_at(g, gauge, c, mu, a);
    m3_dag(a, a);
    m3_mul(t, a, t);
#pragma unroll
    for (int k = 0; k < 18; ++k) Q[k] += t[k];
}

// sigma_{mu nu} restricted to the two chiral blocks of the DeGrand-Rossi
// basis (upper: spins 0,1; lower: spins 2,3), planes xy, xz, xt, yz, yt, zt.
// Entries are (re, im) of the 2x2 block, row-major.  Worked out from
// sigma = (i/2)[g_mu, g_nu]; every sigma_{mu nu} commutes with g5 here.
__constant__ double SIGMA_BLK[6][2][8] = {
    {{1, 0, 0, 0, 0, 0, -1, 0}, {1, 0, 0, 0, 0, 0, -1, 0}},    // xy: diag(1,-1), diag(1,-1)
    {{0, 0, 0, -1, 0, 1, 0, 0}, {0, 0, 0, -1, 0, 1, 0, 0}},    // xz: [[0,-i],[i,0]] both
    {{0, 0, -1, 0, -1, 0, 0, 0}, {0, 0, 1, 0, 1, 0, 0, 0}},    // xt: [[0,-1],[-1,0]], [[0,1],[1,0]]
    {{0, 0, 1, 0, 1, 0, 0, 0}, {0, 0, 1, 0, 1, 0, 0, 0}},      // yz: [[0,1],[1,0]] both
    {{0, 0, 0, -1, 0, 1, 0, 0}, {0, 0, 0, 1, 0, -1, 0, 0}},    // yt: [[0,-i],[i,0]], [[0,i],[-i,0]]
    {{-1, 0, 0, 0, 0, 0, 1, 0}, {1, 0, 0, 0, 0, 0, -1, 0}},    // zt: diag(-1,1), diag(1,-1)
};

// Pack a 6x6 Hermitian block m[r][s][re/im] into 36 reals.
__device__ __forceinline__ void pack_herm6(const double m[6][6][2], double c[36])
{
#pragma unroll
    for (int r = 0; r < 6; ++r) c[r] = m[r][r][0];
    int k = 6;
#pragma unroll
    for (int r = 1; r < 6; ++r)
#pragma unroll
        for (int s = 0; s < r; ++s) {
            c[k++] = m[r][s][0];
            c[k++] = m[r][s][1];
        }
}

__device__ __forceinline__ void unpack_herm6(const double c[36], double m[6][6][2])
{
    for (int r = 0; r < 6; ++r) {
        m[r][r][0] = c[r];
        m[r][r][1] = 0.0;
    }
    int k = 6;
    for (int r = 1; r < 6; ++r)
        for (int s = 0; s < r; ++s) {
            m[r][s][0] = c[k];
            m[r][s][1] = c[k + 1];
            m[s][r][0] = c[k];
            m[s][r][1] = -c[k + 1];
            k += 2;
        }
}

// One thread per site of parity blockIdx.y: A blocks in FP64.
__global__ void clover_build_kernel(Geom g, const void* gauge, double kc, char* A64, size_t par_bytes)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int par = blockIdx.y;
    if (i >= g.Vh) return;
    int c[4];
    cb_coords(g, i, par, c);
    double blk[2][6][6][2];
    for (int b = 0; b < 2; ++b)
        for (int r = 0; r < 6; ++r)
            for (int s = 0; s < 6; ++s) {
                blk[b][r][s][0] = (r == s) ? 1.0 : 0.0;
                blk[b][r][s][1] = 0.0;
            }
    const int PL[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
    for (int p = 0; p < 6; ++p) {
        double Q[18], F[18];
        leaves(g, gauge, c, PL[p][0], PL[p][1], Q);
        // Fhat = (Q - Q^dag) / 8, traceless
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                F[2 * (3 * a + b)] = (Q[2 * (3 * a + b)] - Q[2 * (3 * b + a)]) * 0.125;
                F[2 * (3 * a + b) + 1] = (Q[2 * (3 * a + b) + 1] + Q[2 * (3 * b + a) + 1]) * 0.125;
            }
        const double tri = (F[1] + F[9] + F[17]) / 3.0;  // trace is imaginary
        F[1] -= tri;
        F[9] -= tri;
        F[17] -= tri;
        // block += i kc sigma (x) F
        for (int b = 0; b < 2; ++b)
            for (int s = 0; s < 2; ++s)
                for (int r = 0; r < 2; ++r) {
                    const double sr = SIGMA_BLK[p][b][2 * (2 * s + r)], si = SIGMA_BLK[p][b][2 * (2 * s + r) + 1];
                    if (sr == 0.0 && si == 0.0) continue;
                    for (int a = 0; a < 3; ++a)
                        for (int cc = 0; cc < 3; ++cc) {
                            const double fr = F[2 * (3 * a + cc)], fi = F[2 * (3 * a + cc) + 1];
                            const double zr = sr * fr - si * fi, zi = sr * fi + si * fr;
                            blk[b][3 * s + a][3 * r + cc][0] += -kc * zi;
                            blk[b][3 * s + a][3 * r + cc][1] += kc * zr;
                        }
                }
    }
    for (int b = 0; b < 2; ++b) {
        double pk[36];
        pack_herm6(blk[b], pk);
        CloverIO<P64>::store_block(A64 + par * par_bytes, g.stride, i, b, pk);
    }
}

// One thread per (site, chiral block) of parity blockIdx.y: Gauss-Jordan
// inversion with partial pivoting in FP64.
__global__ void clover_invert_kernel(Geom g, const char* A64, char* Ainv64, size_t par_bytes, int* errw)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int par = blockIdx.y;
    if (t >= 2 * g.Vh) return;
    const int i = t >> 1, b = t & 1;
    double pk[36], m[6][6][2], inv[6][6][2];
    CloverIO<P64>::load_block(A64 + par * par_bytes, g.stride, i, b, pk);
    unpack_herm6(pk, m);
    for (int r = 0; r < 6; ++r)
        for (int s = 0; s < 6; ++s) {
            inv[r][s][0] = (r == s) ? 1.0 : 0.0;
            inv[r][s][1] = 0.0;
        }
    bool ok = true;
    for (int col = 0; col < 6; ++col) {
        int piv = col;
        double best = hypot(m[col][col][0], m[col][col][1]);
        for (int r = col + 1; r < 6; ++r) {
            const double v = hypot(m[r][col][0], m[r][col][1]);
            if (v > best) { best = v; piv = r; }
        }
        if (best < 1e-12) { ok = false; break; }
        if (piv != col)
            for (int s = 0; s < 6; ++s)
                for (int q = 0; q < 2; ++q) {
                    double tmp = m[col][s][q]; m[col][s][q] = m[piv][s][q]; m[piv][s][q] = tmp;
                    tmp = inv[col][s][q]; inv[col][s][q] = inv[piv][s][q]; inv[piv][s][q] = tmp;
                }
        // scale the pivot row by 1 / m[col][col]
        const double pr = m[col][col][0], pi = m[col][col][1];
        const double den = pr * pr + pi * pi;
        const double ir = pr / den, ii = -pi / den;
        for (int s = 0; s < 6; ++s) {
            double xr = m[col][s][0], xi = m[col][s][1];
            m[col][s][0] = xr * ir - xi * ii;
            m[col][s][1] = xr * ii + xi * ir;
            xr = inv[col][s][0]; xi = inv[col][s][1];
            inv[col][s][0] = xr * ir - xi * ii;
            inv[col][s][1] = xr * ii + xi * ir;
        }
        for (int r = 0; r < 6; ++r) {
            if (r == col) continue;
            const double fr = m[r][col][0], fi = m[r][col][1];
            for (int s = 0; s < 6; ++s) {
                m[r][s][0] -= fr * m[col][s][0] - fi * m[col][s][1];
                m[r][s][1] -= fr * m[col][s][1] + fi * m[col][s][0];
                inv[r][s][0] -= fr * inv[col][s][0] - fi * inv[col][s][1];
                inv[r][s][1] -= fr * inv[col][s][1] + fi * inv[col][s][0];
            }
        }
    }
    if (!ok) atomicOr(errw, ERRW_CLOVER_SINGULAR);
    pack_herm6(inv, pk);
    CloverIO<P64>::store_block(Ainv64 + par * par_bytes, g.stride, i, b, pk);
}

// FP64 clover -> precision P, both parities (blockIdx.y).
template <int P>
__global__ void clover_round_kernel(Geom g, const char* src, size_t src_pb, char* dst, size_t dst_pb)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int par = blockIdx.y;
    if (i >= g.Vh) return;
    double a[36], b[36];
    CloverIO<P64>::load_block(src + par * src_pb, g.stride, i, 0, a);
    CloverIO<P64>::load_block(src + par * src_pb, g.stride, i, 1, b);
    if constexpr (P == P32) {
        float fa[36], fb[36];
        for (int k = 0; k < 36; ++k) { fa[k] = (float)a[k]; fb[k] = (float)b[k]; }
        CloverIO<P32>::store_block(dst + par * dst_pb, g.stride, i, 0, fa);
        CloverIO<P32>::store_block(dst + par * dst_pb, g.stride, i, 1, fb);
    } else {
        float f[72];
        for (int k = 0; k < 36; ++k) { f[k] = (float)a[k]; f[36 + k] = (float)b[k]; }
        CloverIO<P>::store_all(dst + par * dst_pb, g.stride, i, f);
    }
}

lqcd_status clover_build(lqcd_ctx* c, double kappa, double csw)
{
    const int block = 64;
    dim3 grid((c->g.Vh + block - 1) / block, 2);
    const size_t pb64 = c->clov_parity_bytes(P64);
    clover_build_kernel<<<grid, block, 0, c->stream>>>(c->g, c->gauge[P64], kappa * csw,
                                                       static_cast<char*>(c->clov[P64]), pb64);
    LQ_CUDA(cudaGetLastError());
    c->launches++;
    dim3 grid2((2 * c->g.Vh + block - 1) / block, 2);
    clover_invert_kernel<<<grid2, block, 0, c->stream>>>(c->g, static_cast<const char*>(c->clov[P64]),
                                                         static_cast<char*>(c->clovinv[P64]), pb64, c->errw);
    LQ_CUDA(cudaGetLastError());
    c->launches++;
    for (int P = P32; P <= PB16; ++P) {
        if (!c->holds(P)) continue;
        const size_t pb = c->clov_parity_bytes(P);
        for (int which = 0; which < 2; ++which) {
            const char* src = static_cast<const char*>(which ? c->clovinv[P64] : c->clov[P64]);
            char* dst = static_cast<char*>(which ? c->clovinv[P] : c->clov[P]);
            switch (P) {
            case P32: clover_round_kernel<P32><<<grid, block, 0, c->stream>>>(c->g, src, pb64, dst, pb); break;
            case P16: clover_round_kernel<P16><<<grid, block, 0, c->stream>>>(c->g, src, pb64, dst, pb); break;
            default: clover_round_kernel<PB16><<<grid, block, 0, c->stream>>>(c->g, src, pb64, dst, pb); break;
            }
            LQ_CUDA(cudaGetLastError());
            c->launches++;
        }
    }
    return LQCD_OK;
}

// out = Cl in for one parity, Cl = A or A^{-1} stored in PG, spinors in PS.
template <int PG, int PS>
__global__ void clover_apply_kernel(Geom g, char* out, const char* in, const char* cl, size_t rb)
{
    typedef typename RealT<PS>::type R;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int rhs = blockIdx.y;
    if (i >= g.Vh) return;
    R v[24], w[24];
    SpinorIO<PS>::load(in + rhs * rb, g.stride, i, v);
    clover_apply_site<PG>(cl, g.stride, i, v, w);
    SpinorIO<PS>::store(out + rhs * rb, g.stride, i, w);
}

lqcd_status clover_apply_launch(lqcd_ctx* c, void* out, const void* in, int parity, int inverse, int mode, int nrhs,
                                size_t rb)
{
    const int block = 128;
    dim3 grid((c->g.Vh + block - 1) / block, nrhs);
    const int pg = mode_pg(mode);
    const char* cl = static_cast<const char*>(inverse ? c->clovinv[pg] : c->clov[pg]) + parity * c->clov_parity_bytes(pg);
    char* o = static_cast<char*>(out);
    const char* i = static_cast<const char*>(in);
    switch (mode) {
    case P64: clover_apply_kernel<P64, P64><<<grid, block, 0, c->stream>>>(c->g, o, i, cl, rb); break;
    case P32: clover_apply_kernel<P32, P32><<<grid, block, 0, c->stream>>>(c->g, o, i, cl, rb); break;
    case P16: clover_apply_kernel<P16, P16><<<grid, block, 0, c->stream>>>(c->g, o, i, cl, rb); break;
    case PB16: clover_apply_kernel<PB16, PB16><<<grid, block, 0, c->stream>>>(c->g, o, i, cl, rb); break;
    case MODE_F16_LINKS: clover_apply_kernel<P16, P32><<<grid, block, 0, c->stream>>>(c->g, o, i, cl, rb); break;
    case MODE_BF16_LINKS: clover_apply_kernel<PB16, P32><<<grid, block, 0, c->stream>>>(c->g, o, i, cl, rb); break;
    case MODE_F16_SPINORS: clover_apply_kernel<P32, P16><<<grid, block, 0, c->stream>>>(c->g, o, i, cl, rb); break;
    case MODE_BF16_SPINORS: clover_apply_kernel<P32, PB16><<<grid, block, 0, c->stream>>>(c->g, o, i, cl, rb); break;
    default: return fail(LQCD_ERR_INVALID, "clover apply: bad precision mode");
    }
    LQ_CUDA(cudaGetLastError());
    c->launches++;
    return LQCD_OK;
}

}  // namespace lqcd
