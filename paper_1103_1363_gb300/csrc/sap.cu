// Schwarz alternating procedure (SAP) preconditioner, the paper's
// preconditioner inside FGCR (Sec. 5).  The lattice is cut into
// non-overlapping blocks coloured like a checkerboard.  One cycle solves
// approximately on every block of colour 0 (nmr minimal-residual iterations
// of the block operator with Dirichlet boundaries), updates the residual,
// then does the same on the blocks of colour 1.
//
// On the Cell the block solve ran out of the SPE local store; here one CTA
// owns one block and keeps the block residual rho in shared memory (float4
// planes [6][V_B], so that lanes touch consecutive words).  The MR scalars
// are CTA-wide reductions.
//
// Residual update without a full operator application (the paper's scheme:
// after one colour, the residual changes on those blocks and on the inner
// border of the others).  Each launch writes, on the sites it solves, the
// final block residual (rho_out), the correction delta (dlt) and z += delta.
// The next launch (other colour) starts from rho_out on its own sites and
// adds the hops that reach them from the neighbouring blocks' delta:
// rho(x) += kappa sum_{y outside the block} hop(x <- y) delta(y).  Reads of
// dlt are at sites of the other colour and writes at sites of the launch's
// colour, so the gather needs no atomics.
//
// Blocks of at most SAP_THREADS sites run one site per thread with q and
// delta in registers and the block's links staged in shared memory once per
// block solve; larger blocks (up to 1024 sites, e.g. the paper's 8x4x8x4)
// stride over the sites with q in shared memory, delta accumulated in dlt
// and the links read through L1/L2.
#include <cmath>
#include <cstring>

#include "internal.h"

namespace lqcd {

enum { SAP_THREADS = 256, SAP_MAX_SITES = 1024 };

struct SapArgs {
    Geom g;
    int bs[4];          // block extents
    int nb[4];          // blocks per direction
    int vol;            // sites per block
    int colour;         // blocks with (sum of block coordinates) % 2 == colour are solved
    int nmr;            // MR iterations per block
    int has_prev;       // add the border hops of dlt (0 in the very first launch)
    const void* gauge;  // FP32 links
    const char* clov;   // FP32 clover A, parity p at clov + p * clov_pb; nullptr: A = 1
    size_t clov_pb;
    float kappa;
    const char* rho_in; // residual on the solved sites before the neighbours' last correction
    char* rho_out;      // final block residual on the solved sites (may equal rho_in)
    char* dlt;          // corrections: read at other-colour sites, written at solved sites
    char* z;            // z += delta on the solved sites
    size_t fb;          // bytes of one FP32 parity field (full field: even, then odd at + fb)
};

struct SapSite {
    int c[4];  // global coordinates
    int l[4];  // coordinates inside the block
    int par, cb;
};

__device__ __forceinline__ SapSite sap_site(const SapArgs& a, const int bc[4], int l)
{
    SapSite s;
    s.l[0] = l % a.bs[0];
    l /= a.bs[0];
    s.l[1] = l % a.bs[1];
    l /= a.bs[1];
    s.l[2] = l % a.bs[2];
    s.l[3] = l / a.bs[2];
#pragma unroll
    for (int m = 0; m < 4; ++m) s.c[m] = bc[m] * a.bs[m] + s.l[m];
    s.par = (s.c[0] + s.c[1] + s.c[2] + s.c[3]) & 1;
    s.cb = full_index(a.g, s.c) >> 1;
    return s;
}

__device__ __forceinline__ void smem_load(const float4* base, int vol, int l, float v[24])
{
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const float4 t = base[k * vol + l];
        v[4 * k] = t.x;
        v[4 * k + 1] = t.y;
        v[4 * k + 2] = t.z;
        v[4 * k + 3] = t.w;
    }
}

__device__ __forceinline__ void smem_store(float4* base, int vol, int l, const float v[24])
{
#pragma unroll
    for (int k = 0; k < 6; ++k) base[k * vol + l] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
}

// acc += the block-restricted hops of direction MU at site s (local index l):
// (1 - g) U_mu(x) rho(x + mu) if x + mu is in the block, and
// (1 + g) U_mu(x - mu)^dag rho(x - mu) if x - mu is.  A block never wraps
// around the lattice (at least two blocks per direction), so no boundary
// phase enters inside it.
template <int RECON, int MU>
__device__ __forceinline__ void sap_hop(const SapArgs& a, const float4* rs, const SapSite& s, int l, int lstride,
                                        float acc[24])
{
    float v[24], h[12], u[18], w[12];
    if (s.l[MU] + 1 < a.bs[MU]) {
        smem_load(rs, a.vol, l + lstride, v);
        project<MU, -1>(v, h);
        GaugeIO<P32, RECON>::load(a.gauge, a.g.stride, s.par, MU, s.cb, u);
        su3_mul_half<false, true>(u, h, w);
        accumulate<MU, -1>(acc, w);
    }
    if (s.l[MU] > 0) {
        int cc[4] = {s.c[0], s.c[1], s.c[2], s.c[3]};
        cc[MU] -= 1;
        smem_load(rs, a.vol, l - lstride, v);
        project<MU, +1>(v, h);
        GaugeIO<P32, RECON>::load(a.gauge, a.g.stride, 1 - s.par, MU, full_index(a.g, cc) >> 1, u);
        su3_mul_half<true, true>(u, h, w);
        accumulate<MU, +1>(acc, w);
    }
}

// The block's links in shared memory, [mu][plane][site]: recon-12 keeps rows
// 0 and 1 as three float4 planes (row 2 rebuilt on use), recon-18 all nine
// complex entries as float2 planes.  The link of x - mu that a backward hop
// needs is the forward link of a site inside the block.
template <int RECON> struct SmemLinks;
template <> struct SmemLinks<12> {
    static constexpr int bytes = 48;
    __device__ __forceinline__ static void store(char* base, int vol, int mu, int l, const float u[18])
    {
        float4* p = reinterpret_cast<float4*>(base) + mu * 3 * vol + l;
#pragma unroll
        for (int k = 0; k < 3; ++k) p[k * vol] = make_float4(u[4 * k], u[4 * k + 1], u[4 * k + 2], u[4 * k + 3]);
    }
    __device__ __forceinline__ static void load(const char* base, int vol, int mu, int l, float u[18])
    {
        const float4* p = reinterpret_cast<const float4*>(base) + mu * 3 * vol + l;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float4 t = p[k * vol];
            u[4 * k] = t.x;
            u[4 * k + 1] = t.y;
            u[4 * k + 2] = t.z;
            u[4 * k + 3] = t.w;
        }
        reconstruct_row2(u);
    }
};
template <> struct SmemLinks<18> {
    static constexpr int bytes = 72;
    __device__ __forceinline__ static void store(char* base, int vol, int mu, int l, const float u[18])
    {
        float2* p = reinterpret_cast<float2*>(base) + mu * 9 * vol + l;
#pragma unroll
        for (int k = 0; k < 9; ++k) p[k * vol] = make_float2(u[2 * k], u[2 * k + 1]);
    }
    __device__ __forceinline__ static void load(const char* base, int vol, int mu, int l, float u[18])
    {
        const float2* p = reinterpret_cast<const float2*>(base) + mu * 9 * vol + l;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const float2 t = p[k * vol];
            u[2 * k] = t.x;
            u[2 * k + 1] = t.y;
        }
    }
};

// sap_hop with the links taken from shared memory
template <int RECON, int MU>
__device__ __forceinline__ void sap_hop_staged(const SapArgs& a, const float4* rs, const char* lk, const SapSite& s,
                                               int l, int lstride, float acc[24])
{
    float v[24], h[12], u[18], w[12];
    if (s.l[MU] + 1 < a.bs[MU]) {
        smem_load(rs, a.vol, l + lstride, v);
        project<MU, -1>(v, h);
        SmemLinks<RECON>::load(lk, a.vol, MU, l, u);
        su3_mul_half<false, true>(u, h, w);
        accumulate<MU, -1>(acc, w);
    }
    if (s.l[MU] > 0) {
        smem_load(rs, a.vol, l - lstride, v);
        project<MU, +1>(v, h);
        SmemLinks<RECON>::load(lk, a.vol, MU, l - lstride, u);
        su3_mul_half<true, true>(u, h, w);
        accumulate<MU, +1>(acc, w);
    }
}

// acc += the hops of direction MU that reach site s from outside its block,
// applied to the neighbours' corrections (lattice wrap-around and the
// antiperiodic t phase included, as in the full operator).
template <int RECON, int MU>
__device__ __forceinline__ void sap_border_hop(const SapArgs& a, const SapSite& s, float acc[24])
{
    float v[24], h[12], u[18], w[12];
    const int L = a.g.L[MU];
    const char* other = a.dlt + (1 - s.par) * a.fb;
    if (s.l[MU] == a.bs[MU] - 1) {
        int cc[4] = {s.c[0], s.c[1], s.c[2], s.c[3]};
        cc[MU] = s.c[MU] == L - 1 ? 0 : s.c[MU] + 1;
        SpinorIO<P32>::load(other, a.g.stride, full_index(a.g, cc) >> 1, v);
        project<MU, -1>(v, h);
        if (MU == 3 && a.g.tanti && s.c[3] == L - 1) {
#pragma unroll
            for (int k = 0; k < 12; ++k) h[k] = -h[k];
        }
        GaugeIO<P32, RECON>::load(a.gauge, a.g.stride, s.par, MU, s.cb, u);
        su3_mul_half<false, true>(u, h, w);
        accumulate<MU, -1>(acc, w);
    }
    if (s.l[MU] == 0) {
        int cc[4] = {s.c[0], s.c[1], s.c[2], s.c[3]};
        cc[MU] = s.c[MU] == 0 ? L - 1 : s.c[MU] - 1;
        const int cbn = full_index(a.g, cc) >> 1;
        SpinorIO<P32>::load(other, a.g.stride, cbn, v);
        project<MU, +1>(v, h);
        if (MU == 3 && a.g.tanti && s.c[3] == 0) {
#pragma unroll
            for (int k = 0; k < 12; ++k) h[k] = -h[k];
        }
        GaugeIO<P32, RECON>::load(a.gauge, a.g.stride, 1 - s.par, MU, cbn, u);
        su3_mul_half<true, true>(u, h, w);
        accumulate<MU, +1>(acc, w);
    }
}

// rho = the current residual at site s: rho_in plus the border hops of the
// neighbouring blocks' last corrections.
template <int RECON>
__device__ __forceinline__ void sap_residual_site(const SapArgs& a, const SapSite& s, float rho[24])
{
    SpinorIO<P32>::load(a.rho_in + s.par * a.fb, a.g.stride, s.cb, rho);
    if (a.has_prev) {
        float acc[24];
#pragma unroll
        for (int k = 0; k < 24; ++k) acc[k] = 0.f;
        sap_border_hop<RECON, 0>(a, s, acc);
        sap_border_hop<RECON, 1>(a, s, acc);
        sap_border_hop<RECON, 2>(a, s, acc);
        sap_border_hop<RECON, 3>(a, s, acc);
#pragma unroll
        for (int k = 0; k < 24; ++k) rho[k] += a.kappa * acc[k];
    }
}

// q = M_B rho at site s (rho of the whole block in shared memory), with the
// site's contributions to |q|^2 and <q, rho>.
// lk: the block's links in shared memory, or nullptr to read them from the
// global FP32 copy.
template <int RECON, bool STAGED>
__device__ __forceinline__ void sap_block_op_site(const SapArgs& a, const float4* rs, const char* lk,
                                                  const SapSite& s, int l, const int ls[4], float q[24], float& qq,
                                                  float& qr_re, float& qr_im)
{
    float acc[24], rho[24];
#pragma unroll
    for (int k = 0; k < 24; ++k) acc[k] = 0.f;
    if (STAGED) {
        sap_hop_staged<RECON, 0>(a, rs, lk, s, l, ls[0], acc);
        sap_hop_staged<RECON, 1>(a, rs, lk, s, l, ls[1], acc);
        sap_hop_staged<RECON, 2>(a, rs, lk, s, l, ls[2], acc);
        sap_hop_staged<RECON, 3>(a, rs, lk, s, l, ls[3], acc);
    } else {
        sap_hop<RECON, 0>(a, rs, s, l, ls[0], acc);
        sap_hop<RECON, 1>(a, rs, s, l, ls[1], acc);
        sap_hop<RECON, 2>(a, rs, s, l, ls[2], acc);
        sap_hop<RECON, 3>(a, rs, s, l, ls[3], acc);
    }
    smem_load(rs, a.vol, l, rho);
    if (a.clov) {
        clover_apply_site<P32>(a.clov + s.par * a.clov_pb, a.g.stride, s.cb, rho, q);
    } else {
#pragma unroll
        for (int k = 0; k < 24; ++k) q[k] = rho[k];
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const float qa = q[2 * k] - a.kappa * acc[2 * k];
        const float qb = q[2 * k + 1] - a.kappa * acc[2 * k + 1];
        q[2 * k] = qa;
        q[2 * k + 1] = qb;
        qq += qa * qa + qb * qb;
        qr_re += qa * rho[2 * k] + qb * rho[2 * k + 1];  // <q, rho> = sum conj(q) rho
        qr_im += qa * rho[2 * k + 1] - qb * rho[2 * k];
    }
}

// CTA-wide sums of three values; every thread returns the same totals.
__device__ __forceinline__ void cta_sum3(float& a, float& b, float& c, float* red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (lane == 0) {
        red[3 * warp] = a;
        red[3 * warp + 1] = b;
        red[3 * warp + 2] = c;
    }
    __syncthreads();
    a = b = c = 0.f;
    for (int w = 0; w < nw; ++w) {
        a += red[3 * w];
        b += red[3 * w + 1];
        c += red[3 * w + 2];
    }
    __syncthreads();  // red may be overwritten by the next call
}

__device__ __forceinline__ bool sap_block_coords(const SapArgs& a, int bc[4])
{
    int b = blockIdx.x;
    bc[0] = b % a.nb[0];
    b /= a.nb[0];
    bc[1] = b % a.nb[1];
    b /= a.nb[1];
    bc[2] = b % a.nb[2];
    bc[3] = b / a.nb[2];
    return ((bc[0] + bc[1] + bc[2] + bc[3]) & 1) == a.colour;
}

// One site per thread (vol <= blockDim.x): q and delta in registers, the
// block's links staged in shared memory behind rho.
template <int RECON>
__global__ void __launch_bounds__(SAP_THREADS, 2) sap_block_kernel_one(const SapArgs a)
{
    extern __shared__ float4 sap_smem[];
    __shared__ float red[3 * (SAP_THREADS / 32)];
    float4* rs = sap_smem;                                     // block residual rho [6][vol]
    char* lk = reinterpret_cast<char*>(sap_smem + 6 * a.vol);  // links [4][planes][vol]
    int bc[4];
    if (!sap_block_coords(a, bc)) return;  // whole CTA
    const int ls[4] = {1, a.bs[0], a.bs[0] * a.bs[1], a.bs[0] * a.bs[1] * a.bs[2]};
    const int l = threadIdx.x;
    const bool live = l < a.vol;
    const SapSite s = sap_site(a, bc, live ? l : 0);
    float delta[24];
#pragma unroll
    for (int k = 0; k < 24; ++k) delta[k] = 0.f;
    if (live) {
        float rho[24], u[18];
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            GaugeIO<P32, RECON>::load(a.gauge, a.g.stride, s.par, mu, s.cb, u);
            SmemLinks<RECON>::store(lk, a.vol, mu, l, u);
        }
        sap_residual_site<RECON>(a, s, rho);
        smem_store(rs, a.vol, l, rho);
    }
    __syncthreads();
    for (int it = 0; it < a.nmr; ++it) {
        float q[24], qq = 0.f, qr_re = 0.f, qr_im = 0.f;
        if (live) sap_block_op_site<RECON, true>(a, rs, lk, s, l, ls, q, qq, qr_re, qr_im);
        cta_sum3(qq, qr_re, qr_im, red);  // also orders every read of rho before the update
        if (!(qq > 0.f)) break;           // same totals in every thread: uniform
        const float ar = qr_re / qq, ai = qr_im / qq;
        if (live) {  // delta += alpha rho, rho -= alpha q
            float rho[24];
            smem_load(rs, a.vol, l, rho);
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                const float rr = rho[2 * k], ri = rho[2 * k + 1];
                delta[2 * k] += ar * rr - ai * ri;
                delta[2 * k + 1] += ar * ri + ai * rr;
                rho[2 * k] = rr - (ar * q[2 * k] - ai * q[2 * k + 1]);
                rho[2 * k + 1] = ri - (ar * q[2 * k + 1] + ai * q[2 * k]);
            }
            smem_store(rs, a.vol, l, rho);
        }
        __syncthreads();
    }
    if (live) {
        float rho[24], zv[24];
        smem_load(rs, a.vol, l, rho);
        SpinorIO<P32>::store(a.rho_out + s.par * a.fb, a.g.stride, s.cb, rho);
        SpinorIO<P32>::store(a.dlt + s.par * a.fb, a.g.stride, s.cb, delta);
        char* zp = a.z + s.par * a.fb;
        SpinorIO<P32>::load(zp, a.g.stride, s.cb, zv);
#pragma unroll
        for (int k = 0; k < 24; ++k) zv[k] += delta[k];
        SpinorIO<P32>::store(zp, a.g.stride, s.cb, zv);
    }
}

// Threads stride over the block's sites: q in shared memory, delta
// accumulated in dlt at the solved sites.
template <int RECON>
__global__ void __launch_bounds__(SAP_THREADS) sap_block_kernel_strided(const SapArgs a)
{
    extern __shared__ float4 sap_smem[];
    __shared__ float red[3 * (SAP_THREADS / 32)];
    float4* rs = sap_smem;              // block residual rho [6][vol]
    float4* qs = sap_smem + 6 * a.vol;  // q = M_B rho      [6][vol]
    int bc[4];
    if (!sap_block_coords(a, bc)) return;  // whole CTA
    const int ls[4] = {1, a.bs[0], a.bs[0] * a.bs[1], a.bs[0] * a.bs[1] * a.bs[2]};
    const float zero[24] = {};
    for (int l = threadIdx.x; l < a.vol; l += blockDim.x) {
        const SapSite s = sap_site(a, bc, l);
        float rho[24];
        sap_residual_site<RECON>(a, s, rho);
        smem_store(rs, a.vol, l, rho);
    }
    __syncthreads();
    for (int l = threadIdx.x; l < a.vol; l += blockDim.x) {  // delta = 0 on the block
        const SapSite s = sap_site(a, bc, l);
        SpinorIO<P32>::store(a.dlt + s.par * a.fb, a.g.stride, s.cb, zero);
    }
    for (int it = 0; it < a.nmr; ++it) {
        float qq = 0.f, qr_re = 0.f, qr_im = 0.f;
        for (int l = threadIdx.x; l < a.vol; l += blockDim.x) {
            const SapSite s = sap_site(a, bc, l);
            float q[24];
            sap_block_op_site<RECON, false>(a, rs, nullptr, s, l, ls, q, qq, qr_re, qr_im);
            smem_store(qs, a.vol, l, q);
        }
        cta_sum3(qq, qr_re, qr_im, red);
        if (!(qq > 0.f)) break;
        const float ar = qr_re / qq, ai = qr_im / qq;
        for (int l = threadIdx.x; l < a.vol; l += blockDim.x) {
            const SapSite s = sap_site(a, bc, l);
            float rho[24], q[24], dv[24];
            smem_load(rs, a.vol, l, rho);
            smem_load(qs, a.vol, l, q);
            char* dp = a.dlt + s.par * a.fb;
            SpinorIO<P32>::load(dp, a.g.stride, s.cb, dv);
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                const float rr = rho[2 * k], ri = rho[2 * k + 1];
                dv[2 * k] += ar * rr - ai * ri;
                dv[2 * k + 1] += ar * ri + ai * rr;
                rho[2 * k] = rr - (ar * q[2 * k] - ai * q[2 * k + 1]);
                rho[2 * k + 1] = ri - (ar * q[2 * k + 1] + ai * q[2 * k]);
            }
            SpinorIO<P32>::store(dp, a.g.stride, s.cb, dv);
            smem_store(rs, a.vol, l, rho);
        }
        __syncthreads();
    }
    for (int l = threadIdx.x; l < a.vol; l += blockDim.x) {
        const SapSite s = sap_site(a, bc, l);
        float rho[24], dv[24], zv[24];
        smem_load(rs, a.vol, l, rho);
        SpinorIO<P32>::store(a.rho_out + s.par * a.fb, a.g.stride, s.cb, rho);
        SpinorIO<P32>::load(a.dlt + s.par * a.fb, a.g.stride, s.cb, dv);
        char* zp = a.z + s.par * a.fb;
        SpinorIO<P32>::load(zp, a.g.stride, s.cb, zv);
#pragma unroll
        for (int k = 0; k < 24; ++k) zv[k] += dv[k];
        SpinorIO<P32>::store(zp, a.g.stride, s.cb, zv);
    }
}

lqcd_status sap_check(const lqcd_ctx* c, const int bs[4])
{
    int vol = 1;
    for (int m = 0; m < 4; ++m) {
        if (bs[m] < 1 || c->g.L[m] % bs[m] != 0)
            return fail(LQCD_ERR_INVALID, "SAP: the block extents must divide the lattice extents");
        const int nb = c->g.L[m] / bs[m];
        if (nb < 2 || (nb & 1))
            return fail(LQCD_ERR_INVALID, "SAP: an even number (>= 2) of blocks per direction is needed");
        vol *= bs[m];
    }
    if (vol > SAP_MAX_SITES) return fail(LQCD_ERR_INVALID, "SAP: at most 1024 sites per block");
    if (!c->holds(P32)) return fail(LQCD_ERR_STATE, "SAP: the context must hold FP32 links (prec_mask)");
    return LQCD_OK;
}

lqcd_status sap_apply(lqcd_ctx* c, void* z, const void* r, const int bs[4], int ncycle, int nmr, char* rho_buf,
                      char* dlt_buf)
{
    LQ_TRY(sap_check(c, bs));
    const size_t fb = c->field_bytes(P32), fld = 2 * fb;
    LQ_TRY(blas_zero(c, z, P32, 1, fld, 2));
    SapArgs a;
    memset(&a, 0, sizeof a);
    a.g = c->g;
    int nblocks = 1;
    a.vol = 1;
    for (int m = 0; m < 4; ++m) {
        a.bs[m] = bs[m];
        a.nb[m] = c->g.L[m] / bs[m];
        nblocks *= a.nb[m];
        a.vol *= bs[m];
    }
    a.nmr = nmr;
    a.gauge = c->gauge[P32];
    a.clov = (c->clover_state && c->csw != 0.0) ? static_cast<const char*>(c->clov[P32]) : nullptr;
    a.clov_pb = c->clov_parity_bytes(P32);
    a.kappa = (float)c->kappa;
    a.rho_out = rho_buf;
    a.dlt = dlt_buf;
    a.z = static_cast<char*>(z);
    a.fb = fb;
    const bool one = a.vol <= SAP_THREADS;
    const int threads = one ? (a.vol + 31) / 32 * 32 : SAP_THREADS;
    const size_t link_bytes = c->cfg.recon == 12 ? SmemLinks<12>::bytes : SmemLinks<18>::bytes;
    const size_t smem = one ? (size_t)a.vol * (6 * sizeof(float4) + 4 * link_bytes)
                            : (size_t)a.vol * 2 * 6 * sizeof(float4);
    const bool r12 = c->cfg.recon == 12;
    const void* fn = one ? (r12 ? (const void*)sap_block_kernel_one<12> : (const void*)sap_block_kernel_one<18>)
                         : (r12 ? (const void*)sap_block_kernel_strided<12> : (const void*)sap_block_kernel_strided<18>);
    LQ_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    for (int cy = 0; cy < ncycle; ++cy)
        for (int colour = 0; colour < 2; ++colour) {
            // the first cycle starts from r on both colours (z = 0 there before
            // the launch); later ones from the block residuals they left
            a.rho_in = cy == 0 ? static_cast<const char*>(r) : rho_buf;
            a.has_prev = !(cy == 0 && colour == 0);
            a.colour = colour;
            if (one && r12) sap_block_kernel_one<12><<<nblocks, threads, smem, c->stream>>>(a);
            else if (one) sap_block_kernel_one<18><<<nblocks, threads, smem, c->stream>>>(a);
            else if (r12) sap_block_kernel_strided<12><<<nblocks, threads, smem, c->stream>>>(a);
            else sap_block_kernel_strided<18><<<nblocks, threads, smem, c->stream>>>(a);
            LQ_CUDA(cudaGetLastError());
            c->launches++;
        }
    return LQCD_OK;
}

}  // namespace lqcd

using namespace lqcd;

extern "C" {

lqcd_status lqcd_set_preconditioner_sap(lqcd_ctx* c, const int block[4], int ncycle, int nmr)
{
    if (!c) return fail(LQCD_ERR_INVALID, "null context");
    if (!block) {
        c->sap_on = 0;
        return LQCD_OK;
    }
    LQ_TRY(sap_check(c, block));
    if (ncycle < 1 || nmr < 1) return fail(LQCD_ERR_INVALID, "SAP: ncycle and nmr must be >= 1");
    for (int m = 0; m < 4; ++m) c->sap_bs[m] = block[m];
    c->sap_ncycle = ncycle;
    c->sap_nmr = nmr;
    c->sap_on = 1;
    c->precond = nullptr;
    return LQCD_OK;
}

lqcd_status lqcd_sap_apply(lqcd_ctx* c, void* z, const void* r, const int block[4], int ncycle, int nmr)
{
    NvtxRange nvtx_range("lqcd_sap_apply");
    if (!c || !z || !r || !block) return fail(LQCD_ERR_INVALID, "lqcd_sap_apply: null argument");
    if (!c->ws) return fail(LQCD_ERR_NOMEM, "no workspace: call lqcd_set_workspace");
    if (!c->gauge_loaded) return fail(LQCD_ERR_STATE, "lqcd_sap_apply: no gauge field loaded");
    if (c->cut()) return fail(LQCD_ERR_STATE, "lqcd_sap_apply: not on a sub-domain of a cut lattice");
    if (ncycle < 1 || nmr < 1) return fail(LQCD_ERR_INVALID, "lqcd_sap_apply: ncycle and nmr must be >= 1");
    DeviceScope dev_scope;
    LQ_TRY(dev_scope.enter(c->device));
    return sap_apply(c, z, r, block, ncycle, nmr, vec64_field(c, 4, 0), vec64_field(c, 5, 0));
}

}  // extern "C"
