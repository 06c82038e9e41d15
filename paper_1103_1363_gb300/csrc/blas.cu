// Site-wise vector updates of the solvers, fused with their reductions.
// Every kernel streams whole 24-real sites through registers in the
// compute precision; sums are accumulated per thread in FP64 and reduced
// deterministically (block partials, last block adds them in order).
// These are the data-parallel site-wise operations the paper splits over
// cores (Sec. 4); on the GPU the grid is the split.
#include "internal.h"

namespace lqcd {

static inline int blas_grid(const lqcd_ctx* c, int block)
{
    int nb = (c->g.Vh + block - 1) / block;
    const int cap = 4 * 152;
    return nb < cap ? nb : cap;
}

// nf = 1: one parity field; nf = 2: a full field (even then odd).
template <int P>
__global__ void norm2_kernel(Geom g, const char* x, size_t rb, int nf, double* partials, size_t part_rs,
                             unsigned* tickets, double* red)
{
    typedef typename RealT<P>::type R;
    const int rhs = blockIdx.y;
    const size_t fb = spinor_field_bytes(P, g.stride);
    double n = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.Vh; i += gridDim.x * blockDim.x)
        for (int f = 0; f < nf; ++f) {
            R v[24];
            SpinorIO<P>::load(x + rhs * rb + f * fb, g.stride, i, v);
            R s = 0;
#pragma unroll
            for (int k = 0; k < 24; ++k) s += v[k] * v[k];
            n += (double)s;
        }
    double vv[1] = {n};
    block_reduce_finalize<1>(vv, partials + rhs * part_rs, tickets + rhs, red + rhs * SC_PER_RHS);
}

template <int P>
__global__ void xmy_norm_kernel(Geom g, char* out, const char* b, const char* a, size_t rb, int nf,
                                double* partials, size_t part_rs, unsigned* tickets, double* red)
{
    typedef typename RealT<P>::type R;
    const int rhs = blockIdx.y;
    const size_t fb = spinor_field_bytes(P, g.stride);
    double n = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.Vh; i += gridDim.x * blockDim.x)
        for (int f = 0; f < nf; ++f) {
            R vb[24], va[24];
            SpinorIO<P>::load(b + rhs * rb + f * fb, g.stride, i, vb);
            SpinorIO<P>::load(a + rhs * rb + f * fb, g.stride, i, va);
            R s = 0;
#pragma unroll
            for (int k = 0; k < 24; ++k) {
                vb[k] -= va[k];
                s += vb[k] * vb[k];
            }
            n += (double)s;
            SpinorIO<P>::store(out + rhs * rb + f * fb, g.stride, i, vb);
        }
    double vv[1] = {n};
    block_reduce_finalize<1>(vv, partials + rhs * part_rs, tickets + rhs, red + rhs * SC_PER_RHS);
}

// p = r + beta p, beta = (scal[num] + scal[num + 1]) / (scal[den] + scal[den + 1])
// (the two slots hold the even- and odd-parity parts of |r|^2)
template <int PP, int PR>
__global__ void cg_p_kernel(Geom g, char* p, size_t p_rb, const char* r, size_t r_rb, int nf, const double* scal,
                            int num, int den, const int* skip)
{
    typedef typename RealT<PP>::type RP;
    typedef typename RealT<PR>::type RR;
    const int rhs = blockIdx.y;
    if (skip && skip[rhs]) return;
    const double* sc = scal + rhs * SC_PER_RHS;
    const double bden = sc[den] + sc[den + 1];  // 0 once the residual has vanished
    const RR beta = bden > 0.0 ? (RR)((sc[num] + sc[num + 1]) / bden) : (RR)0;
    const size_t fp = spinor_field_bytes(PP, g.stride), fr = spinor_field_bytes(PR, g.stride);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.Vh; i += gridDim.x * blockDim.x)
        for (int f = 0; f < nf; ++f) {
            RP vp[24];
            RR vr[24];
            SpinorIO<PP>::load(p + rhs * p_rb + f * fp, g.stride, i, vp);
            SpinorIO<PR>::load(r + rhs * r_rb + f * fr, g.stride, i, vr);
#pragma unroll
            for (int k = 0; k < 24; ++k) vp[k] = (RP)(vr[k] + beta * (RR)vp[k]);
            SpinorIO<PP>::store(p + rhs * p_rb + f * fp, g.stride, i, vp);
        }
}

// xhi += xlo; xlo = 0
template <int PL>
__global__ void accum_x_kernel(Geom g, char* xhi, size_t hi_rb, char* xlo, size_t lo_rb, int nf)
{
    typedef typename RealT<PL>::type RL;
    const int rhs = blockIdx.y;
    const size_t fh = spinor_field_bytes(P64, g.stride), fl = spinor_field_bytes(PL, g.stride);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.Vh; i += gridDim.x * blockDim.x)
        for (int f = 0; f < nf; ++f) {
            double vh[24];
            RL vl[24];
            SpinorIO<P64>::load(xhi + rhs * hi_rb + f * fh, g.stride, i, vh);
            SpinorIO<PL>::load(xlo + rhs * lo_rb + f * fl, g.stride, i, vl);
#pragma unroll
            for (int k = 0; k < 24; ++k) {
                vh[k] += (double)vl[k];
                vl[k] = 0;
            }
            SpinorIO<P64>::store(xhi + rhs * hi_rb + f * fh, g.stride, i, vh);
            SpinorIO<PL>::store(xlo + rhs * lo_rb + f * fl, g.stride, i, vl);
        }
}

template <int P>
__global__ void zero_kernel(Geom g, char* x, size_t rb, int nf)
{
    typedef typename RealT<P>::type R;
    const int rhs = blockIdx.y;
    const size_t fb = spinor_field_bytes(P, g.stride);
    R v[24];
#pragma unroll
    for (int k = 0; k < 24; ++k) v[k] = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.Vh; i += gridDim.x * blockDim.x)
        for (int f = 0; f < nf; ++f) SpinorIO<P>::store(x + rhs * rb + f * fb, g.stride, i, v);
}

__global__ void copy_scalar_kernel(double* scal, int dst, int src, int nrhs)
{
    const int r = threadIdx.x;
    if (r < nrhs) scal[r * SC_PER_RHS + dst] = scal[r * SC_PER_RHS + src];
}

#define LQ_SWITCH_P(P, CALL)                 \
    switch (P) {                             \
    case P64: { constexpr int PT = P64; CALL; break; }  \
    case P32: { constexpr int PT = P32; CALL; break; }  \
    case P16: { constexpr int PT = P16; CALL; break; }  \
    default: { constexpr int PT = PB16; CALL; break; }  \
    }

lqcd_status blas_norm2(lqcd_ctx* c, const void* x, int P, int nrhs, size_t rb, int nf, int slot)
{
    const int block = 256;
    dim3 grid(blas_grid(c, block), nrhs);
    LQ_SWITCH_P(P, (norm2_kernel<PT><<<grid, block, 0, c->stream>>>(c->g, static_cast<const char*>(x), rb, nf,
                                                                     c->partials, c->part_rs, c->tickets,
                                                                     c->scal + slot)));
    LQ_CUDA(cudaGetLastError());
    c->launches++;
    return LQCD_OK;
}

lqcd_status blas_xmy_norm(lqcd_ctx* c, void* out, const void* b, const void* a, int P, int nrhs, size_t rb, int nf,
                          int slot)
{
    const int block = 256;
    dim3 grid(blas_grid(c, block), nrhs);
    LQ_SWITCH_P(P, (xmy_norm_kernel<PT><<<grid, block, 0, c->stream>>>(
                       c->g, static_cast<char*>(out), static_cast<const char*>(b), static_cast<const char*>(a), rb,
                       nf, c->partials, c->part_rs, c->tickets, c->scal + slot)));
    LQ_CUDA(cudaGetLastError());
    c->launches++;
    return LQCD_OK;
}

lqcd_status blas_cg_p_update(lqcd_ctx* c, void* p, int Pp, const void* r, int Pr, int nrhs, size_t p_rb,
                             size_t r_rb, int nf, int s_num, int s_den)
{
    const int block = 256;
    dim3 grid(blas_grid(c, block), nrhs);
    char* pp = static_cast<char*>(p);
    const char* rr = static_cast<const char*>(r);
    if (Pr == P64) {
        if (Pp != P64) return fail(LQCD_ERR_INVALID, "cg_p_update: FP64 r needs FP64 p");
        cg_p_kernel<P64, P64><<<grid, block, 0, c->stream>>>(c->g, pp, p_rb, rr, r_rb, nf, c->scal, s_num, s_den,
                                                             c->skip);
    } else {
        LQ_SWITCH_P(Pp, (cg_p_kernel<PT, P32><<<grid, block, 0, c->stream>>>(c->g, pp, p_rb, rr, r_rb, nf, c->scal,
                                                                               s_num, s_den, c->skip)));
    }
    LQ_CUDA(cudaGetLastError());
    c->launches++;
    return LQCD_OK;
}

lqcd_status blas_accumulate_x(lqcd_ctx* c, void* xhi, const void* xlo, int Plo, int nrhs, size_t hi_rb, size_t lo_rb,
                              int nf)
{
    const int block = 256;
    dim3 grid(blas_grid(c, block), nrhs);
    char* h = static_cast<char*>(xhi);
    char* l = const_cast<char*>(static_cast<const char*>(xlo));
    LQ_SWITCH_P(Plo, (accum_x_kernel<PT><<<grid, block, 0, c->stream>>>(c->g, h, hi_rb, l, lo_rb, nf)));
    LQ_CUDA(cudaGetLastError());
    c->launches++;
    return LQCD_OK;
}

lqcd_status blas_zero(lqcd_ctx* c, void* x, int P, int nrhs, size_t rb, int nf)
{
    const int block = 256;
    dim3 grid(blas_grid(c, block), nrhs);
    LQ_SWITCH_P(P, (zero_kernel<PT><<<grid, block, 0, c->stream>>>(c->g, static_cast<char*>(x), rb, nf)));
    LQ_CUDA(cudaGetLastError());
    c->launches++;
    return LQCD_OK;
}

lqcd_status blas_copy_scalar(lqcd_ctx* c, int dst, int src, int nrhs)
{
    copy_scalar_kernel<<<1, 32 * ((nrhs + 31) / 32), 0, c->stream>>>(c->scal, dst, src, nrhs);
    LQ_CUDA(cudaGetLastError());
    c->launches++;
    return LQCD_OK;
}

}  // namespace lqcd
