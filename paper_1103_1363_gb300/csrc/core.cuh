// Core device types of the GB300 Wilson-clover library: precisions, the
// structure-of-arrays field layouts, SU(3) link storage with third-row
// reconstruction, per-site-norm half-precision spinors, and deterministic
// block/grid reductions.
//
// Layout rule (all fields): one array per parity, site index i fastest,
// 16-byte (or 8-byte) vectors per "chunk": element (chunk k, site i) lives at
// base[k * stride + i].  A warp therefore reads 32 consecutive vectors per
// chunk: fully coalesced 512-byte transactions.  The paper's kernel packs
// colour/spin/complex per site for 128-bit SIMD registers (Sec. 5); on a GPU
// the SIMD lanes are the threads, so the site index is the fast one.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace lqcd {

enum Prec { P64 = 0, P32 = 1, P16 = 2, PB16 = 3 };

template <int P> struct RealT { typedef float type; };
template <> struct RealT<P64> { typedef double type; };

// Accumulation precision of the CG vectors r, x for an inner precision P.
template <int P> struct AccumP { enum { value = (P == P64) ? P64 : P32 }; };
__host__ __device__ inline int AccumPrec(int P) { return P == P64 ? P64 : P32; }

// A precision mode selects the storage of the operator's coefficients
// (links and clover, "pg") and of the spinor fields ("ps").  Modes 0-3 store
// both in the same precision; modes 4 and 5 store links and clover in FP16 /
// BF16 and every spinor field in FP32.  The arithmetic is FP64 for mode 0
// and FP32 otherwise.
// Mode 6 is not used.
enum { MODE_F16_LINKS = 4, MODE_BF16_LINKS = 5, MODE_F16_SPINORS = 7, MODE_BF16_SPINORS = 8, NMODES = 9 };
__host__ __device__ inline bool valid_mode(int m) { return m >= 0 && m < NMODES && m != 6; }
__host__ __device__ inline int mode_pg(int m)
{
    switch (m) {
    case MODE_F16_LINKS: return P16;
    case MODE_BF16_LINKS: return PB16;
    case MODE_F16_SPINORS:
    case MODE_BF16_SPINORS: return P32;
    default: return m;
    }
}
__host__ __device__ inline int mode_ps(int m)
{
    switch (m) {
    case MODE_F16_LINKS:
    case MODE_BF16_LINKS: return P32;
    case MODE_F16_SPINORS: return P16;
    case MODE_BF16_SPINORS: return PB16;
    default: return m;
    }
}

// Lattice geometry of one context, passed by value to every kernel.
struct Geom {
    int L[4];    // Lx, Ly, Lz, Lt
    int Lxh;     // Lx / 2
    int Vh;      // sites per parity
    int stride;  // Vh rounded up to a multiple of 128
    int tanti;   // antiperiodic fermion boundary in t
    int part;    // bit mu: the global lattice is cut along mu; hops across the local boundary use faces
    int tfirst;  // this sub-domain holds the global t = 0 slice (fermion sign on its backward t faces)
    int tlast;   // ... the global t = Lt - 1 slice (sign on its forward t faces)
};

// ----------------------------------------------------------------- helpers

__device__ __forceinline__ float2 h2f(uint32_t u, int isbf)
{
    if (isbf) {
        __nv_bfloat162 b = *reinterpret_cast<__nv_bfloat162*>(&u);
        return __bfloat1622float2(b);
    }
    __half2 h = *reinterpret_cast<__half2*>(&u);
    return __half22float2(h);
}

__device__ __forceinline__ uint32_t f2h(float a, float b, int isbf)
{
    uint32_t u;
    if (isbf) {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        u = *reinterpret_cast<uint32_t*>(&h);
    } else {
        __half2 h = __floats2half2_rn(a, b);
        u = *reinterpret_cast<uint32_t*>(&h);
    }
    return u;
}

// ------------------------------------------------------------ spinor fields
// 24 reals per site: index 2*(spin*3 + colour) + {0: re, 1: im}.

template <int P> struct SpinorIO;

template <> struct SpinorIO<P64> {
    static constexpr int bytes_per_site = 192;
    __device__ __forceinline__ static void load(const void* base, int stride, int i, double v[24])
    {
        const double2* p = static_cast<const double2*>(base);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            double2 c = __ldg(p + (size_t)k * stride + i);
            v[2 * k] = c.x;
            v[2 * k + 1] = c.y;
        }
    }
    __device__ __forceinline__ static void store(void* base, int stride, int i, const double v[24])
    {
        double2* p = static_cast<double2*>(base);
#pragma unroll
        for (int k = 0; k < 12; ++k) p[(size_t)k * stride + i] = make_double2(v[2 * k], v[2 * k + 1]);
    }
};

template <> struct SpinorIO<P32> {
    static constexpr int bytes_per_site = 96;
    __device__ __forceinline__ static void load(const void* base, int stride, int i, float v[24])
    {
        const float4* p = static_cast<const float4*>(base);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            float4 c = __ldg(p + (size_t)k * stride + i);
            v[4 * k] = c.x;
            v[4 * k + 1] = c.y;
            v[4 * k + 2] = c.z;
            v[4 * k + 3] = c.w;
        }
    }
    __device__ __forceinline__ static void store(void* base, int stride, int i, const float v[24])
    {
        float4* p = static_cast<float4*>(base);
#pragma unroll
        for (int k = 0; k < 6; ++k)
            p[(size_t)k * stride + i] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
    }
};

// Half precision with a per-site FP32 norm n = max |v_i|; stored q_i = v_i / n.
template <int ISBF> struct SpinorHalfIO {
    static constexpr int bytes_per_site = 52;
    __device__ __forceinline__ static void load(const void* base, int stride, int i, float v[24])
    {
        const uint4* p = static_cast<const uint4*>(base);
        const float n = __ldg(reinterpret_cast<const float*>(p + (size_t)3 * stride) + i);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint4 c = __ldg(p + (size_t)k * stride + i);
            float2 a = h2f(c.x, ISBF), b = h2f(c.y, ISBF), d = h2f(c.z, ISBF), e = h2f(c.w, ISBF);
            v[8 * k + 0] = a.x * n; v[8 * k + 1] = a.y * n;
            v[8 * k + 2] = b.x * n; v[8 * k + 3] = b.y * n;
            v[8 * k + 4] = d.x * n; v[8 * k + 5] = d.y * n;
            v[8 * k + 6] = e.x * n; v[8 * k + 7] = e.y * n;
        }
    }
    __device__ __forceinline__ static void store(void* base, int stride, int i, const float v[24])
    {
        uint4* p = static_cast<uint4*>(base);
        float n = 0.f;
#pragma unroll
        for (int k = 0; k < 24; ++k) n = fmaxf(n, fabsf(v[k]));
        // a site whose largest component is subnormal (below 2^-126) is stored
        // as zero: 1/n would overflow to infinity and make the site NaN (NaN
        // itself still propagates, for the solvers' breakdown checks)
        if (n < 1.17549435e-38f) n = 0.f;
        const float s = n > 0.f ? 1.f / n : 0.f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint4 c;
            c.x = f2h(v[8 * k + 0] * s, v[8 * k + 1] * s, ISBF);
            c.y = f2h(v[8 * k + 2] * s, v[8 * k + 3] * s, ISBF);
            c.z = f2h(v[8 * k + 4] * s, v[8 * k + 5] * s, ISBF);
            c.w = f2h(v[8 * k + 6] * s, v[8 * k + 7] * s, ISBF);
            p[(size_t)k * stride + i] = c;
        }
        reinterpret_cast<float*>(p + (size_t)3 * stride)[i] = n;
    }
};
template <> struct SpinorIO<P16> : SpinorHalfIO<0> {};
template <> struct SpinorIO<PB16> : SpinorHalfIO<1> {};

__host__ __device__ inline size_t spinor_field_bytes(int P, int stride)
{
    return (size_t)stride * (P == P64 ? 192 : P == P32 ? 96 : 52);
}

// ------------------------------------------------------------- gauge links
// Copy layout [parity][mu][chunk][stride].  A link is 9 complex entries
// u[2*(3a+b)+{re,im}]; recon-12 stores rows 0 and 1 and rebuilds row 2 as
// conj(row0 x row1), valid because every link is in SU(3).  The fermion
// boundary sign is applied by the kernel, never folded into the link.

template <class R>
__device__ __forceinline__ void reconstruct_row2(R u[18])
{
    // u2b = conj( eps_{b c d} u0c u1d )
#define RE(a, b) u[2 * (3 * (a) + (b))]
#define IM(a, b) u[2 * (3 * (a) + (b)) + 1]
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        const int c = (b + 1) % 3, d = (b + 2) % 3;
        // u0c u1d - u0d u1c, one multiply-add per real product
        R re = RE(0, c) * RE(1, d);
        re -= IM(0, c) * IM(1, d);
        re -= RE(0, d) * RE(1, c);
        re += IM(0, d) * IM(1, c);
        R im = RE(0, c) * IM(1, d);
        im += IM(0, c) * RE(1, d);
        im -= RE(0, d) * IM(1, c);
        im -= IM(0, d) * RE(1, c);
        RE(2, b) = re;
        IM(2, b) = -im;
    }
#undef RE
#undef IM
}

template <int P, int RECON> struct GaugeIO;

template <int RECON> struct GaugeIO<P64, RECON> {
    static constexpr int nchunk = RECON == 12 ? 6 : 9;
    static constexpr int bytes_per_link = nchunk * 16;
    __device__ __forceinline__ static void load(const void* base, int stride, int par, int mu, int i,
                                                double u[18])
    {
        const double2* p = static_cast<const double2*>(base) + (size_t)((par * 4 + mu) * nchunk) * stride + i;
#pragma unroll
        for (int k = 0; k < nchunk; ++k) {
            double2 c = __ldg(p + (size_t)k * stride);
            u[2 * k] = c.x;
            u[2 * k + 1] = c.y;
        }
        if (RECON == 12) reconstruct_row2(u);
    }
    __device__ __forceinline__ static void store(void* base, int stride, int par, int mu, int i,
                                                 const double u[18])
    {
        double2* p = static_cast<double2*>(base) + (size_t)((par * 4 + mu) * nchunk) * stride + i;
#pragma unroll
        for (int k = 0; k < nchunk; ++k) p[(size_t)k * stride] = make_double2(u[2 * k], u[2 * k + 1]);
    }
};

template <> struct GaugeIO<P32, 18> {
    static constexpr int nchunk = 9;
    static constexpr int bytes_per_link = 72;
    __device__ __forceinline__ static void load(const void* base, int stride, int par, int mu, int i, float u[18])
    {
        const float2* p = static_cast<const float2*>(base) + (size_t)((par * 4 + mu) * 9) * stride + i;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            float2 c = __ldg(p + (size_t)k * stride);
            u[2 * k] = c.x;
            u[2 * k + 1] = c.y;
        }
    }
    __device__ __forceinline__ static void store(void* base, int stride, int par, int mu, int i, const float u[18])
    {
        float2* p = static_cast<float2*>(base) + (size_t)((par * 4 + mu) * 9) * stride + i;
#pragma unroll
        for (int k = 0; k < 9; ++k) p[(size_t)k * stride] = make_float2(u[2 * k], u[2 * k + 1]);
    }
};

template <> struct GaugeIO<P32, 12> {
    static constexpr int nchunk = 3;
    static constexpr int bytes_per_link = 48;
    __device__ __forceinline__ static void load(const void* base, int stride, int par, int mu, int i, float u[18])
    {
        const float4* p = static_cast<const float4*>(base) + (size_t)((par * 4 + mu) * 3) * stride + i;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float4 c = __ldg(p + (size_t)k * stride);
            u[4 * k] = c.x;
            u[4 * k + 1] = c.y;
            u[4 * k + 2] = c.z;
            u[4 * k + 3] = c.w;
        }
        reconstruct_row2(u);
    }
    __device__ __forceinline__ static void store(void* base, int stride, int par, int mu, int i, const float u[18])
    {
        float4* p = static_cast<float4*>(base) + (size_t)((par * 4 + mu) * 3) * stride + i;
#pragma unroll
        for (int k = 0; k < 3; ++k) p[(size_t)k * stride] = make_float4(u[4 * k], u[4 * k + 1], u[4 * k + 2], u[4 * k + 3]);
    }
};

// Half-precision links: |U_ab| <= 1, so no norm is needed.
template <int ISBF, int RECON> struct GaugeHalfIO {
    // recon-12: 3 chunks of uint2 (two complex each); recon-18: 9 chunks of one half2
    static constexpr int nchunk = RECON == 12 ? 3 : 9;
    static constexpr int bytes_per_link = RECON == 12 ? 24 : 36;
    __device__ __forceinline__ static void load(const void* base, int stride, int par, int mu, int i, float u[18])
    {
        if (RECON == 12) {
            const uint2* p = static_cast<const uint2*>(base) + (size_t)((par * 4 + mu) * 3) * stride + i;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                uint2 c = __ldg(p + (size_t)k * stride);
                float2 a = h2f(c.x, ISBF), b = h2f(c.y, ISBF);
                u[4 * k] = a.x; u[4 * k + 1] = a.y; u[4 * k + 2] = b.x; u[4 * k + 3] = b.y;
            }
            reconstruct_row2(u);
        } else {
            const uint32_t* p = static_cast<const uint32_t*>(base) + (size_t)((par * 4 + mu) * 9) * stride + i;
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                float2 a = h2f(__ldg(p + (size_t)k * stride), ISBF);
                u[2 * k] = a.x; u[2 * k + 1] = a.y;
            }
        }
    }
    __device__ __forceinline__ static void store(void* base, int stride, int par, int mu, int i, const float u[18])
    {
        if (RECON == 12) {
            uint2* p = static_cast<uint2*>(base) + (size_t)((par * 4 + mu) * 3) * stride + i;
#pragma unroll
            for (int k = 0; k < 3; ++k)
                p[(size_t)k * stride] = make_uint2(f2h(u[4 * k], u[4 * k + 1], ISBF), f2h(u[4 * k + 2], u[4 * k + 3], ISBF));
        } else {
            uint32_t* p = static_cast<uint32_t*>(base) + (size_t)((par * 4 + mu) * 9) * stride + i;
#pragma unroll
            for (int k = 0; k < 9; ++k) p[(size_t)k * stride] = f2h(u[2 * k], u[2 * k + 1], ISBF);
        }
    }
};
template <int RECON> struct GaugeIO<P16, RECON> : GaugeHalfIO<0, RECON> {};
template <int RECON> struct GaugeIO<PB16, RECON> : GaugeHalfIO<1, RECON> {};

__host__ __device__ inline size_t gauge_link_bytes(int P, int recon)
{
    if (P == P64) return recon == 12 ? 96 : 144;
    if (P == P32) return recon == 12 ? 48 : 72;
    return recon == 12 ? 24 : 36;
}

// ------------------------------------------------------------- clover term
// Per site two 6x6 Hermitian blocks (chirality +: spins 0,1; -: spins 2,3),
// 36 reals each: the 6 real diagonal entries, then the 15 complex entries
// below the diagonal in row order (1,0),(2,0),(2,1),(3,0),...,(5,4).
// Row/column index within a block is (spin - 2*block)*3 + colour.
// Layout [parity][chunk][stride]: F64 36 x double2, F32 18 x float4,
// F16/BF16 9 x uint4.

template <int P> struct CloverIO;

template <> struct CloverIO<P64> {
    static constexpr int bytes_per_site = 576;
    __device__ __forceinline__ static void load_block(const void* base, int stride, int i, int blk, double c[36])
    {
        const double2* p = static_cast<const double2*>(base) + (size_t)(18 * blk) * stride + i;
#pragma unroll
        for (int k = 0; k < 18; ++k) {
            double2 v = __ldg(p + (size_t)k * stride);
            c[2 * k] = v.x;
            c[2 * k + 1] = v.y;
        }
    }
    __device__ __forceinline__ static void store_block(void* base, int stride, int i, int blk, const double c[36])
    {
        double2* p = static_cast<double2*>(base) + (size_t)(18 * blk) * stride + i;
#pragma unroll
        for (int k = 0; k < 18; ++k) p[(size_t)k * stride] = make_double2(c[2 * k], c[2 * k + 1]);
    }
};

template <> struct CloverIO<P32> {
    static constexpr int bytes_per_site = 288;
    __device__ __forceinline__ static void load_block(const void* base, int stride, int i, int blk, float c[36])
    {
        const float4* p = static_cast<const float4*>(base) + (size_t)(9 * blk) * stride + i;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            float4 v = __ldg(p + (size_t)k * stride);
            c[4 * k] = v.x; c[4 * k + 1] = v.y; c[4 * k + 2] = v.z; c[4 * k + 3] = v.w;
        }
    }
    __device__ __forceinline__ static void store_block(void* base, int stride, int i, int blk, const float c[36])
    {
        float4* p = static_cast<float4*>(base) + (size_t)(9 * blk) * stride + i;
#pragma unroll
        for (int k = 0; k < 9; ++k) p[(size_t)k * stride] = make_float4(c[4 * k], c[4 * k + 1], c[4 * k + 2], c[4 * k + 3]);
    }
};

// Half-precision clover: 72 halves per site as 9 uint4; block b occupies
// halves 36b .. 36b+35, i.e. uint4 chunks straddle the block boundary, so
// both blocks are read together.
template <int ISBF> struct CloverHalfIO {
    static constexpr int bytes_per_site = 144;
    __device__ __forceinline__ static void load_all(const void* base, int stride, int i, float c[72])
    {
        const uint4* p = static_cast<const uint4*>(base) + i;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            uint4 v = __ldg(p + (size_t)k * stride);
            float2 a = h2f(v.x, ISBF), b = h2f(v.y, ISBF), d = h2f(v.z, ISBF), e = h2f(v.w, ISBF);
            c[8 * k] = a.x; c[8 * k + 1] = a.y; c[8 * k + 2] = b.x; c[8 * k + 3] = b.y;
            c[8 * k + 4] = d.x; c[8 * k + 5] = d.y; c[8 * k + 6] = e.x; c[8 * k + 7] = e.y;
        }
    }
    __device__ __forceinline__ static void store_all(void* base, int stride, int i, const float c[72])
    {
        uint4* p = static_cast<uint4*>(base) + i;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            uint4 v;
            v.x = f2h(c[8 * k], c[8 * k + 1], ISBF);
            v.y = f2h(c[8 * k + 2], c[8 * k + 3], ISBF);
            v.z = f2h(c[8 * k + 4], c[8 * k + 5], ISBF);
            v.w = f2h(c[8 * k + 6], c[8 * k + 7], ISBF);
            p[(size_t)k * stride] = v;
        }
    }
};
template <> struct CloverIO<P16> : CloverHalfIO<0> {};
template <> struct CloverIO<PB16> : CloverHalfIO<1> {};

__host__ __device__ inline size_t clover_site_bytes(int P)
{
    return P == P64 ? 576 : P == P32 ? 288 : 144;
}

// out = C v for one packed 6x6 Hermitian block (36 reals), v and out 6 complex.
template <class R>
__device__ __forceinline__ void hermitian6_apply(const R c[36], const R v[12], R out[12])
{
#pragma unroll
    for (int r = 0; r < 6; ++r) {
        out[2 * r] = c[r] * v[2 * r];
        out[2 * r + 1] = c[r] * v[2 * r + 1];
    }
    int k = 6;
#pragma unroll
    for (int r = 1; r < 6; ++r) {
#pragma unroll
        for (int s = 0; s < r; ++s) {
            const R lr = c[k], li = c[k + 1];  // L[r][s]; C[s][r] = conj(L[r][s])
            k += 2;
            // one multiply-add per real product
            out[2 * r] += lr * v[2 * s];
            out[2 * r] -= li * v[2 * s + 1];
            out[2 * r + 1] += lr * v[2 * s + 1];
            out[2 * r + 1] += li * v[2 * s];
            out[2 * s] += lr * v[2 * r];
            out[2 * s] += li * v[2 * r + 1];
            out[2 * s + 1] += lr * v[2 * r + 1];
            out[2 * s + 1] -= li * v[2 * r];
        }
    }
}

// Full-site clover application in the compute precision of P.
template <int P>
__device__ __forceinline__ void clover_apply_site(const void* base, int stride, int i,
                                                  const typename RealT<P>::type in[24],
                                                  typename RealT<P>::type out[24])
{
    typedef typename RealT<P>::type R;
    if constexpr (P == P64 || P == P32) {
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            R c[36];
            CloverIO<P>::load_block(base, stride, i, b, c);
            hermitian6_apply<R>(c, in + 12 * b, out + 12 * b);
        }
    } else {
        float c[72];
        CloverIO<P>::load_all(base, stride, i, c);
        hermitian6_apply<float>(c, in, out);
        hermitian6_apply<float>(c + 36, in + 12, out + 12);
    }
}

// ------------------------------------------------------------- reductions
// Deterministic two-stage sum: every block reduces its threads' values
// (warp shuffles, then shared memory), writes one partial, and the last
// block to finish (atomic ticket) adds the partials in block order.  The
// result never depends on scheduling.

// Block bidx of the nblk blocks that reduce into `result`.
template <int NV>
__device__ __forceinline__ void block_reduce_finalize(double (&v)[NV], double* partials, unsigned* ticket,
                                                      double* result, int bidx, int nblk)
{
    __shared__ double sm[32][NV];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sm[warp][k] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double s = 0.0;
            for (int w = 0; w < nwarps; ++w) s += sm[w][k];
            partials[(size_t)bidx * NV + k] = s;
        }
        __threadfence();
        const unsigned t = atomicAdd(ticket, 1u);
        last = (t == (unsigned)nblk - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const volatile double* vp = partials;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double x = 0.0;
        for (int b = threadIdx.x; b < nblk; b += blockDim.x) x += vp[(size_t)b * NV + k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sm[warp][k] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double s = 0.0;
            for (int w = 0; w < nwarps; ++w) s += sm[w][k];
            result[k] = s;
        }
        *ticket = 0u;  // ready for the next launch on this slot
    }
}

template <int NV>
__device__ __forceinline__ void block_reduce_finalize(double (&v)[NV], double* partials, unsigned* ticket,
                                                      double* result)
{
    block_reduce_finalize<NV>(v, partials, ticket, result, (int)blockIdx.x, (int)gridDim.x);
}

// --------------------------------------------------------------- geometry

// Coordinates of checkerboard site i of parity par.
__device__ __forceinline__ void cb_coords(const Geom& g, int i, int par, int c[4])
{
    int xh = i % g.Lxh;
    int r = i / g.Lxh;
    c[1] = r % g.L[1];
    r /= g.L[1];
    c[2] = r % g.L[2];
    c[3] = r / g.L[2];
    c[0] = 2 * xh + ((c[1] + c[2] + c[3] + par) & 1);
}

__device__ __forceinline__ int full_index(const Geom& g, const int c[4])
{
    return ((c[3] * g.L[2] + c[2]) * g.L[1] + c[1]) * g.L[0] + c[0];
}

}  // namespace lqcd
