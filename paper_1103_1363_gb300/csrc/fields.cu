// Layout and precision conversions: canonical FP64 spinors and links to the
// parity-split structure-of-arrays fields of every precision, and back.
#include "internal.h"

namespace lqcd {

// Canonical spinor of rhs r: canon + r * canon_rb bytes, site s at 24 doubles.
template <int P>
__global__ void pack_kernel(Geom g, int par, const double* __restrict__ canon, size_t canon_rb, char* out,
                            size_t out_rb)
{
    typedef typename RealT<P>::type R;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int rhs = blockIdx.y;
    if (i >= g.Vh) return;
    int c[4];
    cb_coords(g, i, par, c);
    const double* src = reinterpret_cast<const double*>(reinterpret_cast<const char*>(canon) + rhs * canon_rb) +
                        (size_t)full_index(g, c) * 24;
    R v[24];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        double2 d = reinterpret_cast<const double2*>(src)[k];
        v[2 * k] = (R)d.x;
        v[2 * k + 1] = (R)d.y;
    }
    SpinorIO<P>::store(out + rhs * out_rb, g.stride, i, v);
}

template <int P>
__global__ void unpack_kernel(Geom g, int par, double* canon, size_t canon_rb, const char* in, size_t in_rb)
{
    typedef typename RealT<P>::type R;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int rhs = blockIdx.y;
    if (i >= g.Vh) return;
    int c[4];
    cb_coords(g, i, par, c);
    double* dst = reinterpret_cast<double*>(reinterpret_cast<char*>(canon) + rhs * canon_rb) +
                  (size_t)full_index(g, c) * 24;
    R v[24];
    SpinorIO<P>::load(in + rhs * in_rb, g.stride, i, v);
#pragma unroll
    for (int k = 0; k < 12; ++k) reinterpret_cast<double2*>(dst)[k] = make_double2((double)v[2 * k], (double)v[2 * k + 1]);
}

// FP64 internal field of parity par = canonical a - b (b may be null: 0).
__global__ void pack_difference_kernel(Geom g, int par, const double* __restrict__ a, const double* __restrict__ b,
                                       size_t canon_rb, char* out, size_t out_rb)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int rhs = blockIdx.y;
    if (i >= g.Vh) return;
    int c[4];
    cb_coords(g, i, par, c);
    const size_t off = rhs * canon_rb / sizeof(double) + (size_t)full_index(g, c) * 24;
    double v[24];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const double2 p = reinterpret_cast<const double2*>(a + off)[k];
        const double2 q = b ? reinterpret_cast<const double2*>(b + off)[k] : make_double2(0.0, 0.0);
        v[2 * k] = p.x - q.x;
        v[2 * k + 1] = p.y - q.y;
    }
    SpinorIO<P64>::store(out + rhs * out_rb, g.stride, i, v);
}

// FP64 internal field of parity par -> canonical FP32 complex spinor.
__global__ void unpack_f32_kernel(Geom g, int par, float* canon, size_t canon_rb, const char* in, size_t in_rb)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int rhs = blockIdx.y;
    if (i >= g.Vh) return;
    int c[4];
    cb_coords(g, i, par, c);
    float4* dst = reinterpret_cast<float4*>(reinterpret_cast<char*>(canon) + rhs * canon_rb) +
                  (size_t)full_index(g, c) * 6;
    double v[24];
    SpinorIO<P64>::load(in + rhs * in_rb, g.stride, i, v);
#pragma unroll
    for (int k = 0; k < 6; ++k)
        dst[k] = make_float4((float)v[4 * k], (float)v[4 * k + 1], (float)v[4 * k + 2], (float)v[4 * k + 3]);
}

// One thread per (checkerboard site, parity, mu) with t0 <= t < t1; the
// canonical slice starts at site (t0, 0, 0, 0).
template <int P, int RECON>
__global__ void gauge_pack_kernel(Geom g, const double* __restrict__ slice, int t0, int t1, char* out)
{
    typedef typename RealT<P>::type R;
    const int per_t = g.Vh / g.L[3];
    const int n = per_t * (t1 - t0);
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int par = blockIdx.y, mu = blockIdx.z;
    if (idx >= n) return;
    const int i = idx + t0 * per_t;  // checkerboard index (t is the slowest coordinate)
    int c[4];
    cb_coords(g, i, par, c);
    const long s = (long)full_index(g, c) - (long)t0 * per_t * 2;
    const double* src = slice + ((size_t)s * 4 + mu) * 18;
    R u[18];
#pragma unroll
    for (int k = 0; k < 18; ++k) u[k] = (R)src[k];
    GaugeIO<P, RECON>::store(out, g.stride, par, mu, i, u);
}

template <int PIN, int POUT>
__global__ void convert_kernel(Geom g, char* out, size_t out_rb, const char* in, size_t in_rb, int nfield,
                               double* partials, size_t part_rs, unsigned* tickets, double* red, size_t red_rs)
{
    typedef typename RealT<PIN>::type RI;
    typedef typename RealT<POUT>::type RO;
    const int rhs = blockIdx.y;
    double nrm = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.Vh; i += gridDim.x * blockDim.x) {
        for (int f = 0; f < nfield; ++f) {
            RI v[24];
            RO w[24];
            SpinorIO<PIN>::load(in + rhs * in_rb + f * spinor_field_bytes(PIN, g.stride), g.stride, i, v);
#pragma unroll
            for (int k = 0; k < 24; ++k) {
                w[k] = (RO)v[k];
                nrm += (double)v[k] * (double)v[k];
            }
            SpinorIO<POUT>::store(out + rhs * out_rb + f * spinor_field_bytes(POUT, g.stride), g.stride, i, w);
        }
    }
    if (partials) {
        double v[1] = {nrm};
        block_reduce_finalize<1>(v, partials + rhs * part_rs, tickets + rhs, red + rhs * red_rs);
    }
}

static int grid_for(const lqcd_ctx* c, int block)
{
    int n = (c->g.Vh + block - 1) / block;
    return n;
}

lqcd_status pack_spinor(lqcd_ctx* c, void* internal, const double* canon, int parity, int P, int nrhs,
                        size_t internal_rb, size_t canon_rb)
{
    const int block = 128;
    for (int par = 0; par < 2; ++par) {
        if (parity >= 0 && par != parity) continue;
        char* out = static_cast<char*>(internal) + (parity < 0 ? par * c->field_bytes(P) : 0);
        dim3 grid(grid_for(c, block), nrhs);
        switch (P) {
        case P64: pack_kernel<P64><<<grid, block, 0, c->stream>>>(c->g, par, canon, canon_rb, out, internal_rb); break;
        case P32: pack_kernel<P32><<<grid, block, 0, c->stream>>>(c->g, par, canon, canon_rb, out, internal_rb); break;
        case P16: pack_kernel<P16><<<grid, block, 0, c->stream>>>(c->g, par, canon, canon_rb, out, internal_rb); break;
        default: pack_kernel<PB16><<<grid, block, 0, c->stream>>>(c->g, par, canon, canon_rb, out, internal_rb); break;
        }
        LQ_CUDA(cudaGetLastError());
        c->launches++;
    }
    return LQCD_OK;
}

lqcd_status unpack_spinor(lqcd_ctx* c, double* canon, const void* internal, int parity, int P, int nrhs,
                          size_t internal_rb, size_t canon_rb)
{
    const int block = 128;
    for (int par = 0; par < 2; ++par) {
        if (parity >= 0 && par != parity) continue;
        const char* in = static_cast<const char*>(internal) + (parity < 0 ? par * c->field_bytes(P) : 0);
        dim3 grid(grid_for(c, block), nrhs);
        switch (P) {
        case P64: unpack_kernel<P64><<<grid, block, 0, c->stream>>>(c->g, par, canon, canon_rb, in, internal_rb); break;
        case P32: unpack_kernel<P32><<<grid, block, 0, c->stream>>>(c->g, par, canon, canon_rb, in, internal_rb); break;
        case P16: unpack_kernel<P16><<<grid, block, 0, c->stream>>>(c->g, par, canon, canon_rb, in, internal_rb); break;
        default: unpack_kernel<PB16><<<grid, block, 0, c->stream>>>(c->g, par, canon, canon_rb, in, internal_rb); break;
        }
        LQ_CUDA(cudaGetLastError());
        c->launches++;
    }
    return LQCD_OK;
}

lqcd_status pack_difference(lqcd_ctx* c, void* internal, const double* a, const double* b, int nrhs,
                            size_t internal_rb, size_t canon_rb)
{
    const int block = 128;
    for (int par = 0; par < 2; ++par) {
        char* out = static_cast<char*>(internal) + par * c->field_bytes(P64);
        dim3 grid(grid_for(c, block), nrhs);
        pack_difference_kernel<<<grid, block, 0, c->stream>>>(c->g, par, a, b, canon_rb, out, internal_rb);
        LQ_CUDA(cudaGetLastError());
        c->launches++;
    }
    return LQCD_OK;
}

lqcd_status unpack_spinor_f32(lqcd_ctx* c, float* canon, const void* internal, int nrhs, size_t internal_rb,
                              size_t canon_rb)
{
    const int block = 128;
    for (int par = 0; par < 2; ++par) {
        const char* in = static_cast<const char*>(internal) + par * c->field_bytes(P64);
        dim3 grid(grid_for(c, block), nrhs);
        unpack_f32_kernel<<<grid, block, 0, c->stream>>>(c->g, par, canon, canon_rb, in, internal_rb);
        LQ_CUDA(cudaGetLastError());
        c->launches++;
    }
    return LQCD_OK;
}

lqcd_status gauge_pack(lqcd_ctx* c, const double* slice, int t0, int t1, int P)
{
    const int block = 128;
    const int n = c->g.Vh / c->g.L[3] * (t1 - t0);
    dim3 grid((n + block - 1) / block, 2, 4);
    char* out = static_cast<char*>(c->gauge[P]);
    const int rc = c->recon_of(P);
#define LQ_G(PP, RC) gauge_pack_kernel<PP, RC><<<grid, block, 0, c->stream>>>(c->g, slice, t0, t1, out)
    if (P == P64) LQ_G(P64, 18);
    else if (P == P32) { if (rc == 12) LQ_G(P32, 12); else LQ_G(P32, 18); }
    else if (P == P16) { if (rc == 12) LQ_G(P16, 12); else LQ_G(P16, 18); }
    else { if (rc == 12) LQ_G(PB16, 12); else LQ_G(PB16, 18); }
#undef LQ_G
    LQ_CUDA(cudaGetLastError());
    c->launches++;
    return LQCD_OK;
}

template <int PIN>
static cudaError_t convert_out(lqcd_ctx* c, dim3 grid, int block, char* out, int Pout, size_t out_rb,
                               const char* in, size_t in_rb, int nfield, double* red, size_t red_rs)
{
    double* part = red ? c->partials : nullptr;
#define LQ_C(PO) convert_kernel<PIN, PO><<<grid, block, 0, c->stream>>>(c->g, out, out_rb, in, in_rb, nfield, part, c->part_rs, c->tickets, red, red_rs)
    switch (Pout) {
    case P64: LQ_C(P64); break;
    case P32: LQ_C(P32); break;
    case P16: LQ_C(P16); break;
    default: LQ_C(PB16); break;
    }
#undef LQ_C
    return cudaGetLastError();
}

// Convert nrhs fields (nf = 1: one parity, nf = 2: full) between precisions;
// with norm_slot >= 0 also write |in|^2 (FP64) to scal[rhs][norm_slot].
lqcd_status convert_field(lqcd_ctx* c, void* out, int Pout, const void* in, int Pin, int nrhs, size_t out_rb,
                          size_t in_rb, int nf, int norm_slot)
{
    const int block = 256;
    int nb = (c->g.Vh + block - 1) / block;
    if (nb > 4 * 152) nb = 4 * 152;
    dim3 grid(nb, nrhs);
    char* o = static_cast<char*>(out);
    const char* i = static_cast<const char*>(in);
    double* red = norm_slot >= 0 ? c->scal + norm_slot : nullptr;
    cudaError_t e;
    switch (Pin) {
    case P64: e = convert_out<P64>(c, grid, block, o, Pout, out_rb, i, in_rb, nf, red, SC_PER_RHS); break;
    case P32: e = convert_out<P32>(c, grid, block, o, Pout, out_rb, i, in_rb, nf, red, SC_PER_RHS); break;
    case P16: e = convert_out<P16>(c, grid, block, o, Pout, out_rb, i, in_rb, nf, red, SC_PER_RHS); break;
    default: e = convert_out<PB16>(c, grid, block, o, Pout, out_rb, i, in_rb, nf, red, SC_PER_RHS); break;
    }
    LQ_CUDA(e);
    c->launches++;
    return LQCD_OK;
}

}  // namespace lqcd
