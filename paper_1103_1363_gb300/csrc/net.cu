// Gauge-equivariant parallel-transport convolution network (the learned
// preconditioner): forward layers, backward (input and weight gradients),
// loss, Adam, and the conversions between solver fields and activations.
//
// A layer maps C_in channels of spinor fields to C_out channels:
//   out(x)[co][s] = sum_h sum_{ci,r} W_h[co*4+s][ci*4+r] (T_h in)(x)[ci][r]
// with nine hops h (0: identity, 2mu+1: U_mu(x) in(x+mu), 2mu+2:
// U_mu(x-mu)^dag in(x-mu), times the fermion boundary sign in t).  The
// transport acts on colour, W on spin x channel, so the two commute; the
// adjoint layer is therefore the same kernel with W'_h = W_{adj(h)}^dag.
//
// Activations at the C ABI: FP32 complex, [batch][site][channel][spin][colour],
// canonical site order.  Inside the network they are planar: per batch item
// and channel, six float4 planes over the sites, plane q holding complex
// components 2q and 2q+1 of the 12 values k = 3 spin + colour (a warp's
// loads of consecutive sites are then one contiguous stretch).  Per hop,
// the transported inputs of a tile of sites are gathered into shared
// memory, and the real-ified product
//   OUT[row][n2] += X[row][k2] * B_h[k2][n2]
// (row = (site, colour), k2 = 2*(ci*4+r) + {re, im}, n2 = 2*(co*4+s) +
// {re, im}) is accumulated over the nine hops:
// - BF16 path: tcgen05 tensor cores.  A persistent CTA per SM takes tiles
//   of 128 sites; the three colour rows of a site go to three M = 128 MMAs
//   (K = 16 per instruction) whose FP32 accumulators live in tensor memory
//   for all nine hops.  Operands are double-buffered in shared memory, so
//   the gather of hop h+1 runs while the MMAs of hop h execute; one thread
//   issues the MMAs and an mbarrier tracks their completion.
// - FP32 path: FMAs on 64-site tiles, accumulators in registers.
// The weight gradient is the same contraction summed over the rows instead
// (tensor cores for BF16, FMAs for FP32).
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "internal.h"

namespace lqcd {

enum { NET_TS = 64, NET_ROWS = 3 * NET_TS, NET_THREADS = 256, NET_MAXC = 12, NET_PARTIALS = 64 };
// tensor-core path: sites per tile (= MMA M), threads, minimum dynamic shared memory (one CTA per SM)
enum { NTC_TS = 128, NTC_THREADS = 512, NTC_MIN_SMEM = 116 * 1024 };

struct NetLayerArgs {
    int L[4];
    int V;
    int stride;        // of the FP32 gauge copy
    int tanti;
    const void* gauge; // FP32 gauge copy (internal SoA)
    int cin, cout;
    int K2, N2;        // real-ified inner / outer sizes: 8 cin, 8 cout
    int K2p, N2p;      // padded to 16 / 8
    const float* in;   // planar activations, cin channels per batch item
    float* out;        // planar activations, cout channels per batch item
    const float* Bf;   // FP32 real-ified weights [9][K2][N2]
    const uint16_t* Bh;// BF16 real-ified weights [9][N2p][K2p] in 8x8 core-matrix order (see prep)
    int batch;         // tensor-core path: batch items (tiles are strided over batch x sites)
    int tmem_cols;     // tensor-core path: allocated tensor-memory columns (power of 2 >= 3 N2p)
    int* errw;         // device error word (bounded waits that expire set ERRW_TIMEOUT)
    int in_bf16;       // activations in BF16 planes (else FP32): the BF16 network's multi-channel ones
    int out_bf16;
    int gout_bf16;     // weight gradient: the output gradient in BF16 planes
    int nhops;         // tensor-core layer: hops 0 .. nhops - 1 (9; 1 for the stacked contraction)
    unsigned long long wait_ns;  // bound of the tensor-core kernels' mbarrier waits
    int expire_test;   // test of the expiry path: each CTA's last wait is for a phase that never completes
};

__host__ __device__ inline int adj_hop(int h) { return h == 0 ? 0 : (h % 2 == 1 ? h + 1 : h - 1); }

// Planar layout of one batch item: float4 index of plane (channel ci, q) at site 0.
__host__ __device__ inline size_t plane4(int V, int ci, int q) { return ((size_t)ci * 6 + q) * V; }

// Complex value k = 3 spin + colour of channel ci at a site, as a float2 index.
__device__ __forceinline__ size_t planar_c(int V, int ci, int k, int site)
{
    return (plane4(V, ci, k >> 1) + site) * 2 + (k & 1);
}

// Link for hop h at canonical site x: V (3x3 complex, 18 floats) and the
// fermion sign; returns the neighbour site.
template <int RECON>
__device__ __forceinline__ int hop_link(const NetLayerArgs& a, int x, int h, float u[18], float& sign)
{
    const int L0 = a.L[0], L1 = a.L[1], L2 = a.L[2], L3 = a.L[3];
    int s = x;
    const int c0 = s % L0;
    s /= L0;
    const int c1 = s % L1;
    s /= L1;
    const int c2 = s % L2;
    const int c3 = s / L2;
    sign = 1.f;
    if (h == 0) return x;
    const int mu = (h - 1) / 2;
    const bool fwd = ((h - 1) % 2) == 0;
    int cm, Lm, st;  // coordinate, extent and site stride of direction mu
    switch (mu) {
    case 0: cm = c0; Lm = L0; st = 1; break;
    case 1: cm = c1; Lm = L1; st = L0; break;
    case 2: cm = c2; Lm = L2; st = L0 * L1; break;
    default: cm = c3; Lm = L3; st = L0 * L1 * L2; break;
    }
    const int y = fwd ? (cm == Lm - 1 ? x - (Lm - 1) * st : x + st) : (cm == 0 ? x + (Lm - 1) * st : x - st);
    if (a.tanti && mu == 3 && ((fwd && c3 == L3 - 1) || (!fwd && c3 == 0))) sign = -1.f;
    // forward: U_mu(x); backward: U_mu(y)^dag, y of the other parity (all extents are even)
    const int site = fwd ? x : y;
    const int par = (c0 + c1 + c2 + c3 + (fwd ? 0 : 1)) & 1;
    GaugeIO<P32, RECON>::load(a.gauge, a.stride, par, mu, site >> 1, u);
    if (!fwd) {
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = i; j < 3; ++j) {
                const float ar = u[2 * (3 * i + j)], ai = u[2 * (3 * i + j) + 1];
                const float br = u[2 * (3 * j + i)], bi = u[2 * (3 * j + i) + 1];
                u[2 * (3 * i + j)] = br; u[2 * (3 * i + j) + 1] = -bi;
                u[2 * (3 * j + i)] = ar; u[2 * (3 * j + i) + 1] = -ai;
            }
    }
    return y;
}

__device__ __forceinline__ uint16_t f2bf(float f)
{
    __nv_bfloat16 b = __float2bfloat16_rn(f);
    return *reinterpret_cast<uint16_t*>(&b);
}

// Gather the transported inputs of hop h for a 64-site tile into shared
// memory (FP32 path and weight gradient): X[row = site*3 + a][k2]; rows past
// V are zero.  The tile's links and neighbours for the hop are staged once;
// then consecutive threads take consecutive (channel, spin) pieces of the
// same neighbour, whose activations are contiguous, so each warp reads one
// stretch of memory.
template <int RECON>
__device__ __forceinline__ void gather_hop(const NetLayerArgs& a, const float* in_b, int tile0, int h, float* Xs,
                                           int xstride)
{
    __shared__ float us[NET_TS][19];  // link (18 floats) and fermion sign per site of the tile
    __shared__ int ys[NET_TS];        // neighbour site, -1 past the lattice
    const int tid = threadIdx.x;
    if (tid < NET_TS) {
        const int x = tile0 + tid;
        float u[18];
        float sign = 1.f;
        int y = -1;
        if (x < a.V) {
            y = hop_link<RECON>(a, x, h, u, sign);
        } else {
#pragma unroll
            for (int q = 0; q < 18; ++q) u[q] = 0.f;
        }
#pragma unroll
        for (int q = 0; q < 18; ++q) us[tid][q] = u[q];
        us[tid][18] = sign;
        ys[tid] = y;
    }
    __syncthreads();
    const int nk = 4 * a.cin;
    const int kp = a.K2p / 2;
    for (int e = tid; e < NET_TS * kp; e += NET_THREADS) {
        const int sl = e / kp, k = e - sl * kp;
        const int y = ys[sl];
        float o[6] = {0, 0, 0, 0, 0, 0};
        if (y >= 0 && k < nk) {
            const float2* src = reinterpret_cast<const float2*>(in_b);
            const int ci = k >> 2, r = k & 3;  // k = ci * 4 + spin: colours 0..2 are k' = 3 r + a
            const float2 p0 = src[planar_c(a.V, ci, 3 * r, y)], p1 = src[planar_c(a.V, ci, 3 * r + 1, y)],
                         p2 = src[planar_c(a.V, ci, 3 * r + 2, y)];
            if (h == 0) {
                o[0] = p0.x; o[1] = p0.y; o[2] = p1.x; o[3] = p1.y; o[4] = p2.x; o[5] = p2.y;
            } else {
                const float sign = us[sl][18];
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    const float* ur = &us[sl][6 * r];
                    o[2 * r] = sign * (ur[0] * p0.x - ur[1] * p0.y + ur[2] * p1.x - ur[3] * p1.y + ur[4] * p2.x - ur[5] * p2.y);
                    o[2 * r + 1] = sign * (ur[0] * p0.y + ur[1] * p0.x + ur[2] * p1.y + ur[3] * p1.x + ur[4] * p2.y + ur[5] * p2.x);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const int row = sl * 3 + r;
            reinterpret_cast<float2*>(Xs + (size_t)row * xstride)[k] = make_float2(o[2 * r], o[2 * r + 1]);
        }
    }
}

// ---------------------------------------------------------------- tcgen05
// Inline-PTX wrappers for the 5th-generation tensor cores (sm_100 family):
// tensor-memory allocation, single-thread MMA issue with shared-memory
// operand descriptors, completion through an mbarrier, and tensor-memory
// loads for the epilogue.
namespace tc {

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor of a K-major operand without swizzling.
// The operand is tiled into core matrices of 8 rows x 16 bytes (128
// contiguous bytes); lbo = bytes between core matrices adjacent in K, sbo =
// bytes between adjacent 8-row groups.  Bits 46-47: descriptor version 1;
// base offset, LBO mode and layout type (bits 49-52, 61-63) are 0.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16
// A and B (bits 7-9 and 10-12 = 1), both K-major (bits 15, 16 = 0), N / 8 in
// bits 17-22 and M / 16 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int m, int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ uint64_t now_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Wait until the phase of parity `parity` has completed; false once
// `limit_ns` of wall time have passed without that.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns)
{
    const uint64_t t0 = now_ns();
    for (;;) {
        uint32_t done;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done)
                     : "r"(smem_addr(bar)), "r"(parity)
                     : "memory");
        if (done) return true;
        if (now_ns() - t0 > limit_ns) return false;
    }
}

// Warp-wide: allocate `ncols` tensor-memory columns (all 128 lanes); the
// address is written to *slot.  Executed by one whole warp.
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)), "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes -> visible to the tensor cores' reads
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// D[tmem] (+)= A[smem] * B[smem]^T, issued by one thread; accumulate = 0
// overwrites D.
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t accumulate)
{
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
                 "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

// One arrival on *bar that also expects `bytes` of asynchronous copies.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

// Bulk copy global -> shared (16-byte aligned, size a multiple of 16) that
// completes `bytes` transactions on *bar.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// Arrive once on *bar when every MMA this thread issued so far has completed.
__device__ __forceinline__ void commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}

// 16 consecutive 32-bit columns of the warp's 32 lanes (lane quarter of the
// warp within its warpgroup); completes with wait_ld.
__device__ __forceinline__ void ld_x16(uint32_t taddr, uint32_t v[16])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                   "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                 : "r"(taddr));
}
__device__ __forceinline__ void wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

}  // namespace tc

// Two floats rounded to nearest BF16, lo in the low half: one packing
// conversion instead of two conversions, a shift and an or.
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&h);
}

// Neighbour of canonical site x (coordinates c0..c3) under hop h; h = 0 is x.
__device__ __forceinline__ int hop_neighbour(const NetLayerArgs& a, int x, int c0, int c1, int c2, int c3, int h)
{
    if (h == 0) return x;
    const int mu = (h - 1) / 2;
    const bool fwd = ((h - 1) % 2) == 0;
    int cm, Lm, st;
    switch (mu) {
    case 0: cm = c0; Lm = a.L[0]; st = 1; break;
    case 1: cm = c1; Lm = a.L[1]; st = a.L[0]; break;
    case 2: cm = c2; Lm = a.L[2]; st = a.L[0] * a.L[1]; break;
    default: cm = c3; Lm = a.L[3]; st = a.L[0] * a.L[1] * a.L[2]; break;
    }
    return fwd ? (cm == Lm - 1 ? x - (Lm - 1) * st : x + st) : (cm == 0 ? x + (Lm - 1) * st : x - st);
}

// Batch item b of planar activations with ch channels: FP32 (six float4
// planes per channel, 96 bytes per channel and site) or BF16 (three planes of
// eight BF16 values, i.e. four complex, per channel: 48 bytes).
__host__ __device__ inline size_t act_item_bytes(int V, int ch, int bf) { return (size_t)V * ch * (bf ? 48 : 96); }

// The 24 floats of channel ci at site y of BF16 planar activations of one
// item (zeros for y < 0).  BF16 is the upper half of FP32: a shift converts.
__device__ __forceinline__ void load_channel_bf16(const uint4* in_b, int V, int ci, int y, float p[24])
{
    if (y >= 0) {
        const uint4* src = in_b + (size_t)ci * 3 * V + y;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const uint4 v = __ldg(src + (size_t)q * V);
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                p[8 * q + 2 * m] = __uint_as_float(w[m] << 16);
                p[8 * q + 2 * m + 1] = __uint_as_float(w[m] & 0xffff0000u);
            }
        }
    } else {
#pragma unroll
        for (int q = 0; q < 24; ++q) p[q] = 0.f;
    }
}

// The 24 floats of channel ci at site y of planar activations (zeros for y < 0).
__device__ __forceinline__ void load_channel(const float* in_b, int V, int ci, int y, float p[24])
{
    if (y >= 0) {
        const float4* src = reinterpret_cast<const float4*>(in_b) + plane4(V, ci, 0) + y;
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const float4 v = __ldg(src + (size_t)q * V);
            p[4 * q] = v.x; p[4 * q + 1] = v.y; p[4 * q + 2] = v.z; p[4 * q + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int q = 0; q < 24; ++q) p[q] = 0.f;
    }
}

// Channel ci at site y of batch item b of activations `act` (FP32 or BF16 planes).
__device__ __forceinline__ void load_act(const void* act, int bf, int V, int ch, int b, int ci, int y, float p[24])
{
    const char* item = static_cast<const char*>(act) + (size_t)b * act_item_bytes(V, ch, bf);
    if (bf) load_channel_bf16(reinterpret_cast<const uint4*>(item), V, ci, y, p);
    else load_channel(reinterpret_cast<const float*>(item), V, ci, y, p);
}

// Default bound of a wait on the kernels' own MMAs and copies (a hop's MMAs
// take microseconds); an expired wait sets ERRW_TIMEOUT and the CTA stops,
// after waiting (with this bound) for its own operations in flight and
// freeing its tensor memory.
#define NTC_WAIT_NS 2000000000ull

// BF16 forward of one layer on the tensor cores.  Shared memory: two
// operand stages, each X (3 colour blocks of 128 sites x K2p) and B_h
// (N2p x K2p), both BF16 in core-matrix order; two link stages (per site
// the hop's link times the boundary sign in 18 floats, plus one float of
// padding: the odd stride makes the reads conflict-free); then four
// mbarriers (MMAs of stage s done, B_h of stage s landed) and the
// tensor-memory address.  Thread (site sl = tid % 128, group grp = tid /
// 128): group 0 stages hop h+1's links while groups 1-3 gather hop h
// (channels grp - 1 + 3 j; hop 0, the identity, needs no link; giving group
// 0 channels too was measured slower: 180 against 164 us for the 12 -> 12
// layer at 16^4).  B_h
// arrives by one bulk copy per hop.  Tensor memory: the accumulator of
// colour a in columns [a N2p, (a+1) N2p), lane = site of the tile.
template <int RECON>
__global__ void __launch_bounds__(NTC_THREADS, 1) net_layer_tc_kernel(const NetLayerArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    // thread group 0 stages links; groups 1.. gather and transport channels grp - 1 + TG j
    constexpr int TG = NTC_THREADS / NTC_TS - 1, CPT = (NET_MAXC + TG - 1) / TG;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int K2p = a.K2p, N2p = a.N2p;
    const uint32_t blk = (uint32_t)NTC_TS * K2p * 2;  // one colour block of X
    const uint32_t xbytes = 3 * blk, bbytes = (uint32_t)N2p * K2p * 2;
    float* lbuf = reinterpret_cast<float*>(smem + 2 * xbytes + 2 * bbytes);              // [2][NTC_TS][19]
    uint64_t* mma_bar = reinterpret_cast<uint64_t*>(lbuf + 2 * NTC_TS * 19);              // [2]
    uint64_t* b_bar = mma_bar + 2;                                                     // [2]
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mma_bar + 4);
    const uint32_t sbo = (uint32_t)(K2p / 8) * 128;  // 8-row groups; K-adjacent core matrices are 128 B apart
    const uint32_t idesc = tc::idesc_bf16_f32(NTC_TS, N2p);
    const uint32_t ncols = (uint32_t)a.tmem_cols;

    // zero both X stages once: the columns of channels >= cin (K padding) are never written
    for (uint32_t e = tid; e < 2 * xbytes / 16; e += NTC_THREADS)
        reinterpret_cast<uint4*>(smem)[e] = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) {
        for (int i = 0; i < 4; ++i) tc::mbar_init(&mma_bar[i], 1);
    }
    if (warp == 0) tc::tmem_alloc(tslot, ncols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;

    const int ntiles = (a.V + NTC_TS - 1) / NTC_TS;
    const int total = ntiles * a.batch;
    const int sl = tid & (NTC_TS - 1), grp = tid / NTC_TS;
    uint32_t g = 0;       // hops whose MMAs were issued (each commits once to mma_bar[g & 1])
    int copies = 0;       // bulk copies issued (hop g's lands on b_bar[g & 1])
    bool failed = false;
    // Each gathering thread walks the items (tile, hop h, channel cfirst + TG j),
    // j < nj, and loads one item ahead, so that a load is in flight while the
    // previous item is transported (across the hop barrier and into the next tile).
    const int cfirst = grp - 1;
    const int nj = (grp > 0 && cfirst < a.cin) ? (a.cin - cfirst + TG - 1) / TG : 0;
    float nxt[24];
    if ((int)blockIdx.x < total && nj > 0) {
        const int t = blockIdx.x, b = t / ntiles, x0 = (t - b * ntiles) * NTC_TS + sl;
        load_act(a.in, a.in_bf16, a.V, a.cin, b, cfirst, x0 < a.V ? x0 : -1, nxt);
    }
    bool wait_failed = false;
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int b = t / ntiles, tile0 = (t - b * ntiles) * NTC_TS;
        const int x = tile0 + sl;
        const int c0 = x % a.L[0], c1 = (x / a.L[0]) % a.L[1], c2 = (x / (a.L[0] * a.L[1])) % a.L[2],
                  c3 = x / (a.L[0] * a.L[1] * a.L[2]);
        const int tn = t + gridDim.x;  // this CTA's next tile
        for (int h = 0; h < a.nhops; ++h) {
            const int s = g & 1;
            unsigned char* const Xst = smem + s * xbytes;               // stage s: X
            unsigned char* const Bst = smem + 2 * xbytes + s * bbytes;  // stage s: B_h
            // stage s is free once the MMAs of hop g - 2 have completed (each
            // thread waits for itself; a failure is shared at the barrier below)
            if (g >= 2 && !wait_failed) wait_failed = !tc::mbar_wait(&mma_bar[s], ((g - 2) >> 1) & 1u, a.wait_ns);
            if (grp == 0 && h + 1 < a.nhops) {  // links of hop h + 1 (read after this hop's barrier)
                float un[18];
                float sign = 1.f;
                if (x < a.V) {
                    hop_link<RECON>(a, x, h + 1, un, sign);
                } else {
#pragma unroll
                    for (int k = 0; k < 18; ++k) un[k] = 0.f;
                }
                float* ls = lbuf + (((h + 1) & 1) * NTC_TS + sl) * 19;
#pragma unroll
                for (int k = 0; k < 18; ++k) ls[k] = sign * un[k];
            }
            if (tid == 0) {  // B_h, stored in core-matrix order: one contiguous bulk copy
                tc::mbar_arrive_expect_tx(&b_bar[s], bbytes);
                tc::bulk_g2s(Bst, a.Bh + (size_t)h * N2p * K2p, bbytes, &b_bar[s]);
            }
            ++copies;
            float u[18];  // link of the hop times the boundary sign (staged at hop h - 1)
            if (h > 0 && nj > 0) {
                const float* ls = lbuf + ((h & 1) * NTC_TS + sl) * 19;
#pragma unroll
                for (int k = 0; k < 18; ++k) u[k] = ls[k];
            }
            const int yh = x < a.V ? hop_neighbour(a, x, c0, c1, c2, c3, h) : -1;
            unsigned char* xrow = Xst + (sl >> 3) * sbo + (sl & 7) * 16;
#pragma unroll
            for (int j = 0; j < CPT; ++j) {
                if (j >= nj) break;
                const int ci = cfirst + TG * j;
                float cur[24];
#pragma unroll
                for (int q = 0; q < 24; ++q) cur[q] = nxt[q];
                if (j + 1 < nj) {
                    load_act(a.in, a.in_bf16, a.V, a.cin, b, ci + TG, yh, nxt);
                } else if (h + 1 < a.nhops) {
                    load_act(a.in, a.in_bf16, a.V, a.cin, b, cfirst,
                             x < a.V ? hop_neighbour(a, x, c0, c1, c2, c3, h + 1) : -1, nxt);
                } else if (tn < total) {
                    const int bn = tn / ntiles, xn = (tn - bn * ntiles) * NTC_TS + sl;
                    load_act(a.in, a.in_bf16, a.V, a.cin, bn, cfirst, xn < a.V ? xn : -1, nxt);
                }
#pragma unroll
                for (int ca = 0; ca < 3; ++ca) {
                    uint32_t w[4];
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        float re, im;
                        if (h == 0) {
                            re = cur[2 * (3 * r + ca)];
                            im = cur[2 * (3 * r + ca) + 1];
                        } else {
                            re = 0.f;
                            im = 0.f;
#pragma unroll
                            for (int cb = 0; cb < 3; ++cb) {  // one multiply-add per real product
                                const float ur = u[2 * (3 * ca + cb)], ui = u[2 * (3 * ca + cb) + 1];
                                const float pr = cur[2 * (3 * r + cb)], pi = cur[2 * (3 * r + cb) + 1];
                                re += ur * pr;
                                re -= ui * pi;
                                im += ur * pi;
                                im += ui * pr;
                            }
                        }
                        w[r] = pack_bf16x2(re, im);
                    }
                    // k2 = 8 ci .. 8 ci + 7: one 16-byte row of core matrix (site group, ci)
                    *reinterpret_cast<uint4*>(xrow + ca * blk + ci * 128) = make_uint4(w[0], w[1], w[2], w[3]);
                }
            }
            tc::fence_proxy_async();
            if (!wait_failed) wait_failed = !tc::mbar_wait(&b_bar[s], (g >> 1) & 1u, a.wait_ns);
            if (__syncthreads_or(wait_failed)) {
                failed = true;
                break;
            }
            if (tid == 0) {
                tc::fence_after();
                const uint32_t xa = tc::smem_addr(Xst), ba = tc::smem_addr(Bst);
                for (int ca = 0; ca < 3; ++ca)
                    for (int ks = 0; ks < K2p / 16; ++ks)
                        tc::mma_bf16(tmem + ca * N2p, tc::smem_desc(xa + ca * blk + ks * 256, 128, sbo),
                                     tc::smem_desc(ba + ks * 256, 128, sbo), idesc, (h > 0 || ks > 0) ? 1u : 0u);
                tc::commit(&mma_bar[s]);
            }
            ++g;
        }
        if (failed) break;
        {  // the tile's last MMAs (their commit covers every earlier one)
            const uint32_t gl = g - 1;
            bool ok = tc::mbar_wait(&mma_bar[gl & 1], (gl >> 1) & 1u, a.wait_ns);
            // expiry test: then wait for the next phase, which nothing completes
            if (ok && a.expire_test) ok = tc::mbar_wait(&mma_bar[gl & 1], ((gl >> 1) & 1u) ^ 1u, a.wait_ns);
            if (__syncthreads_or(!ok)) {
                failed = true;
                break;
            }
        }
        tc::fence_after();
        // epilogue: warp w reads lanes 32 (w % 4) .. +31 (its sites); column
        // chunks of 16 (8 complex outputs n = co * 4 + spin, i.e. two output
        // channels) go round-robin to the four warpgroups; each channel's six
        // float4 planes are written at the site, coalesced over the warp
        const int q4 = warp & 3, wg = warp >> 2;
        const int site = tile0 + 32 * q4 + lane;
        const uint32_t trow = tmem + ((uint32_t)(32 * q4) << 16);
        char* out_item = static_cast<char*>(static_cast<void*>(a.out)) + (size_t)b * act_item_bytes(a.V, a.cout, a.out_bf16);
        for (int c0 = 16 * wg; c0 < N2p; c0 += 16 * (NTC_THREADS / 128)) {
            uint32_t v[3][16];
#pragma unroll
            for (int ca = 0; ca < 3; ++ca) tc::ld_x16(trow + ca * N2p + c0, v[ca]);
            tc::wait_ld();
            if (site < a.V) {
#pragma unroll
                for (int hc = 0; hc < 2; ++hc) {
                    const int co = c0 / 8 + hc;
                    if (co >= a.cout) break;
                    if (a.out_bf16) {
                        uint4* ob = reinterpret_cast<uint4*>(out_item) + (size_t)co * 3 * a.V + site;
#pragma unroll
                        for (int q = 0; q < 3; ++q) {
                            // complex k = 4q .. 4q+3 of channel co: spin k / 3, colour k % 3
                            uint32_t w[4];
#pragma unroll
                            for (int m = 0; m < 4; ++m) {
                                const int kk = 4 * q + m, j = 4 * hc + kk / 3;
                                w[m] = pack_bf16x2(__uint_as_float(v[kk % 3][2 * j]), __uint_as_float(v[kk % 3][2 * j + 1]));
                            }
                            ob[(size_t)q * a.V] = make_uint4(w[0], w[1], w[2], w[3]);
                        }
                    } else {
                        float4* out_b = reinterpret_cast<float4*>(out_item);
#pragma unroll
                        for (int q = 0; q < 6; ++q) {
                            // complex k = 2q, 2q+1 of channel co: spin k / 3, colour k % 3
                            const int k0 = 2 * q, k1 = 2 * q + 1;
                            const int j0 = 4 * hc + k0 / 3, j1 = 4 * hc + k1 / 3;
                            out_b[plane4(a.V, co, q) + site] = make_float4(
                                __uint_as_float(v[k0 % 3][2 * j0]), __uint_as_float(v[k0 % 3][2 * j0 + 1]),
                                __uint_as_float(v[k1 % 3][2 * j1]), __uint_as_float(v[k1 % 3][2 * j1 + 1]));
                        }
                    }
                }
            }
        }
        tc::fence_before();
        __syncthreads();  // tensor memory read before the next tile's first MMA overwrites it
    }
    if (failed) {  // bounded waits for this CTA's own operations in flight, then free the tensor memory
        if (copies > 0) {
            const uint32_t gc = (uint32_t)copies - 1;
            tc::mbar_wait(&b_bar[gc & 1], (gc >> 1) & 1u, NTC_WAIT_NS);
        }
        if (g > 0) {
            const uint32_t gl = g - 1;
            tc::mbar_wait(&mma_bar[gl & 1], (gl >> 1) & 1u, NTC_WAIT_NS);
        }
        if (tid == 0) atomicOr(a.errw, ERRW_TIMEOUT);
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

// BF16 forward of a layer with one input channel (the network's first layer,
// and the adjoint of its last): the nine hops' transported inputs, 8 reals
// each, are laid side by side along K (K = 9 x 8, padded to NC1_K = 80), so
// that one tile needs one gather, one CTA barrier and 3 x 5 MMAs instead of
// nine hop stages of 16-wide K of which half is padding.  All four thread
// groups gather: thread (site sl, group grp) handles hops grp, grp + 4, grp
// + 8.  The weights of all hops, folded the same way, are built in shared
// memory once per CTA from the per-hop BF16 weights.  Two X stages: the
// gather of the next tile runs while the MMAs of this one execute; the
// accumulator in tensor memory is read out before the next tile's MMAs.
enum { NC1_KG = 10, NC1_K = 8 * NC1_KG };  // K groups of 8 (9 hops + one zero group)

template <int RECON>
__global__ void __launch_bounds__(NTC_THREADS, 1) net_layer_c1_kernel(const NetLayerArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int N2p = a.N2p;
    const uint32_t sbo = (uint32_t)NC1_KG * 128;          // bytes between 8-row groups (X and B)
    const uint32_t blk = (uint32_t)NTC_TS * NC1_K * 2;     // one colour block of X
    const uint32_t xbytes = 3 * blk;
    unsigned char* const Bs = smem + 2 * xbytes;           // folded weights [N2p][NC1_K]
    uint64_t* mma_bar = reinterpret_cast<uint64_t*>(Bs + (size_t)N2p * NC1_K * 2);  // [2]
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mma_bar + 2);
    const uint32_t idesc = tc::idesc_bf16_f32(NTC_TS, N2p);
    const uint32_t ncols = (uint32_t)a.tmem_cols;

    // zero both X stages (the padding group is never written), fold the weights:
    // B[n2][8 h + k] = B_h[n2][k] for the 8 real K of each hop (K2p = 16)
    for (uint32_t e = tid; e < 2 * xbytes / 16; e += NTC_THREADS)
        reinterpret_cast<uint4*>(smem)[e] = make_uint4(0u, 0u, 0u, 0u);
    for (int e = tid; e < NC1_KG * N2p; e += NTC_THREADS) {
        const int h = e / N2p, n2 = e - h * N2p;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (h < 9) v = *reinterpret_cast<const uint4*>(a.Bh + (size_t)h * N2p * 16 + (n2 / 8) * 128 + (n2 % 8) * 8);
        *reinterpret_cast<uint4*>(Bs + ((size_t)(n2 / 8) * NC1_KG * 64 + h * 64 + (n2 % 8) * 8) * 2) = v;
    }
    if (tid == 0) {
        tc::mbar_init(&mma_bar[0], 1);
        tc::mbar_init(&mma_bar[1], 1);
    }
    if (warp == 0) tc::tmem_alloc(tslot, ncols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;

    const int ntiles = (a.V + NTC_TS - 1) / NTC_TS;
    const int total = ntiles * a.batch;
    const int sl = tid & (NTC_TS - 1), grp = tid / NTC_TS;

    // transported input of the thread's hops for tile t into X stage s
    auto gather = [&](int t, int s) {
        const int b = t / ntiles, x = (t - b * ntiles) * NTC_TS + sl;
        unsigned char* xrow = smem + s * xbytes + (sl >> 3) * sbo + (sl & 7) * 16;
        for (int h = grp; h < 9; h += NTC_THREADS / NTC_TS) {
            float u[18], p[24];
            float sign = 1.f;
            int y = -1;
#pragma unroll
            for (int k = 0; k < 18; ++k) u[k] = 0.f;  // padding sites: zero link, zero input
            if (x < a.V) {
                if (h > 0) {
                    y = hop_link<RECON>(a, x, h, u, sign);
#pragma unroll
                    for (int k = 0; k < 18; ++k) u[k] = sign * u[k];
                } else {
                    y = x;
                }
            }
            load_act(a.in, a.in_bf16, a.V, 1, b, 0, y, p);
#pragma unroll
            for (int ca = 0; ca < 3; ++ca) {
                uint32_t w[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    float re, im;
                    if (h == 0) {
                        re = p[2 * (3 * r + ca)];
                        im = p[2 * (3 * r + ca) + 1];
                    } else {
                        re = 0.f;
                        im = 0.f;
#pragma unroll
                        for (int cb = 0; cb < 3; ++cb) {  // one multiply-add per real product
                            const float ur = u[2 * (3 * ca + cb)], ui = u[2 * (3 * ca + cb) + 1];
                            const float pr = p[2 * (3 * r + cb)], pi = p[2 * (3 * r + cb) + 1];
                            re += ur * pr;
                            re -= ui * pi;
                            im += ur * pi;
                            im += ui * pr;
                        }
                    }
                    w[r] = pack_bf16x2(re, im);
                }
                *reinterpret_cast<uint4*>(xrow + ca * blk + h * 128) = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
    };

    bool failed = false;
    uint32_t k = 0;  // tiles of this CTA whose MMAs were issued (tile k commits to mma_bar[k & 1])
    if ((int)blockIdx.x < total) gather(blockIdx.x, 0);
    for (int t = blockIdx.x; t < total; t += gridDim.x, ++k) {
        const int s = k & 1;
        tc::fence_proxy_async();
        tc::fence_before();
        __syncthreads();  // X stage s complete; the previous tile's accumulator has been read
        if (tid == 0) {
            tc::fence_after();
            const uint32_t xa = tc::smem_addr(smem + s * xbytes), ba = tc::smem_addr(Bs);
            for (int ca = 0; ca < 3; ++ca)
                for (int ks = 0; ks < NC1_K / 16; ++ks)
                    tc::mma_bf16(tmem + ca * N2p, tc::smem_desc(xa + ca * blk + ks * 256, 128, sbo),
                                 tc::smem_desc(ba + ks * 256, 128, sbo), idesc, ks > 0 ? 1u : 0u);
            tc::commit(&mma_bar[s]);
        }
        // the next tile's gather overlaps these MMAs (stage 1 - s was last
        // read by the MMAs of tile k - 1, complete before its epilogue)
        const int tn = t + gridDim.x;
        if (tn < total) gather(tn, 1 - s);
        bool ok = tc::mbar_wait(&mma_bar[s], (k >> 1) & 1u, a.wait_ns);
        // expiry test: then wait for the next phase, which nothing completes
        if (ok && a.expire_test) ok = tc::mbar_wait(&mma_bar[s], ((k >> 1) & 1u) ^ 1u, a.wait_ns);
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        tc::fence_after();
        // epilogue: as the layer kernel's (warp w reads lanes 32 (w % 4) ..)
        const int b = t / ntiles, tile0 = (t - b * ntiles) * NTC_TS;
        const int q4 = warp & 3, wg = warp >> 2;
        const int site = tile0 + 32 * q4 + lane;
        const uint32_t trow = tmem + ((uint32_t)(32 * q4) << 16);
        char* out_item = static_cast<char*>(static_cast<void*>(a.out)) + (size_t)b * act_item_bytes(a.V, a.cout, a.out_bf16);
        for (int c0 = 16 * wg; c0 < N2p; c0 += 16 * (NTC_THREADS / 128)) {
            uint32_t v[3][16];
#pragma unroll
            for (int ca = 0; ca < 3; ++ca) tc::ld_x16(trow + ca * N2p + c0, v[ca]);
            tc::wait_ld();
            if (site < a.V) {
#pragma unroll
                for (int hc = 0; hc < 2; ++hc) {
                    const int co = c0 / 8 + hc;
                    if (co >= a.cout) break;
                    if (a.out_bf16) {
                        uint4* ob = reinterpret_cast<uint4*>(out_item) + (size_t)co * 3 * a.V + site;
#pragma unroll
                        for (int q = 0; q < 3; ++q) {
                            uint32_t w[4];
#pragma unroll
                            for (int m = 0; m < 4; ++m) {
                                const int kk = 4 * q + m, j = 4 * hc + kk / 3;
                                w[m] = pack_bf16x2(__uint_as_float(v[kk % 3][2 * j]), __uint_as_float(v[kk % 3][2 * j + 1]));
                            }
                            ob[(size_t)q * a.V] = make_uint4(w[0], w[1], w[2], w[3]);
                        }
                    } else {
                        float4* out_b = reinterpret_cast<float4*>(out_item);
#pragma unroll
                        for (int q = 0; q < 6; ++q) {
                            const int k0 = 2 * q, k1 = 2 * q + 1;
                            const int j0 = 4 * hc + k0 / 3, j1 = 4 * hc + k1 / 3;
                            out_b[plane4(a.V, co, q) + site] = make_float4(
                                __uint_as_float(v[k0 % 3][2 * j0]), __uint_as_float(v[k0 % 3][2 * j0 + 1]),
                                __uint_as_float(v[k1 % 3][2 * j1]), __uint_as_float(v[k1 % 3][2 * j1 + 1]));
                        }
                    }
                }
            }
        }
    }
    if (failed) {  // bounded wait for the MMAs of tile k (issued, not seen complete), then free the tensor memory
        tc::mbar_wait(&mma_bar[k & 1], (k >> 1) & 1u, NTC_WAIT_NS);
        if (tid == 0) atomicOr(a.errw, ERRW_TIMEOUT);
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

// BF16 weight gradient of a layer with one input channel, all nine hops in
// one pass: D[8 h + k][n2] = sum over rows (site, colour) of X_h[row][k]
// G[row][n2], the hops' transported inputs folded along M (72 of the MMA's
// 128 rows), so that the output gradient G of a tile is loaded once instead
// of once per hop.  One CTA per SM over the batch x site tiles, the
// accumulator in tensor memory across all of them; the operands (read by
// the MMAs as MN-major: M = k2, N = n2, K = the 128 sites of a colour block)
// are single-buffered.  All four thread groups gather.  The epilogue forms
// the complex gradient from the real-ified sums:
//   G_h[n][k] += (D[2k][2n] + D[2k+1][2n+1], D[2k][2n+1] - D[2k+1][2n]).
template <int RECON>
__global__ void __launch_bounds__(NTC_THREADS, 1) net_wgrad_c1_kernel(const NetLayerArgs a, const float* gout, float* gW)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int MX = 128, G4 = NTC_THREADS / NTC_TS;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int N2p = a.N2p;
    const int nn = 4 * a.cout;
    const uint32_t sbox = (MX / 8) * 128, sbog = (uint32_t)(N2p / 8) * 128;  // bytes between 8-site groups
    const uint32_t blkx = (uint32_t)NTC_TS * MX * 2, blkg = (uint32_t)NTC_TS * N2p * 2;
    unsigned char* const Xs = smem;
    unsigned char* const Gs = smem + 3 * blkx;
    uint64_t* mma_bar = reinterpret_cast<uint64_t*>(Gs + 3 * blkg);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mma_bar + 1);
    const uint32_t idesc = tc::idesc_bf16_f32(MX, N2p) | (1u << 15) | (1u << 16);  // A and B MN-major
    const uint32_t ncols = (uint32_t)a.tmem_cols;

    for (uint32_t e = tid; e < 3 * (blkx + blkg) / 16; e += NTC_THREADS)  // M and N padding stays zero
        reinterpret_cast<uint4*>(smem)[e] = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) tc::mbar_init(mma_bar, 1);
    if (warp == 0) tc::tmem_alloc(tslot, ncols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;

    const int ntiles = (a.V + NTC_TS - 1) / NTC_TS;
    const int total = ntiles * a.batch;
    const int sl = tid & (NTC_TS - 1), grp = tid / NTC_TS;
    const uint32_t rowoff = (sl & 7) * 16;  // row of the site within its 8-site core matrix
    uint32_t k = 0;  // tiles of this CTA so far (tile k commits once to mma_bar)
    bool wait_failed = false, failed = false;
    for (int t = blockIdx.x; t < total; t += gridDim.x, ++k) {
        const int b = t / ntiles, x = (t - b * ntiles) * NTC_TS + sl;
        // the operand tiles are free once the MMAs of tile k - 1 have completed
        if (k >= 1 && !wait_failed) wait_failed = !tc::mbar_wait(mma_bar, (k - 1) & 1, a.wait_ns);
        // X: the transported input of hops grp, grp + 4, grp + 8 at M rows 8 h .. 8 h + 7
        for (int h = grp; h < 9; h += G4) {
            float u[18], p[24];
            float sign = 1.f;
            int y = -1;
#pragma unroll
            for (int q = 0; q < 18; ++q) u[q] = 0.f;  // padding sites: zero link, zero input
            if (x < a.V) {
                if (h > 0) {
                    y = hop_link<RECON>(a, x, h, u, sign);
#pragma unroll
                    for (int q = 0; q < 18; ++q) u[q] = sign * u[q];
                } else {
                    y = x;
                }
            }
            load_act(a.in, a.in_bf16, a.V, 1, b, 0, y, p);
#pragma unroll
            for (int ca = 0; ca < 3; ++ca) {
                uint32_t w[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    float re, im;
                    if (h == 0) {
                        re = p[2 * (3 * r + ca)];
                        im = p[2 * (3 * r + ca) + 1];
                    } else {
                        re = 0.f;
                        im = 0.f;
#pragma unroll
                        for (int cb = 0; cb < 3; ++cb) {  // one multiply-add per real product
                            const float ur = u[2 * (3 * ca + cb)], ui = u[2 * (3 * ca + cb) + 1];
                            const float pr = p[2 * (3 * r + cb)], pi = p[2 * (3 * r + cb) + 1];
                            re += ur * pr;
                            re -= ui * pi;
                            im += ur * pi;
                            im += ui * pr;
                        }
                    }
                    w[r] = pack_bf16x2(re, im);
                }
                *reinterpret_cast<uint4*>(Xs + ca * blkx + (sl >> 3) * sbox + h * 128 + rowoff) =
                    make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
        // G: output-gradient channels grp, grp + 4, ... at the site
        for (int co = grp; co < a.cout; co += G4) {
            float p[24];
            load_act(gout, a.gout_bf16, a.V, a.cout, b, co, x < a.V ? x : -1, p);
#pragma unroll
            for (int ca = 0; ca < 3; ++ca) {
                uint32_t w[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) w[r] = pack_bf16x2(p[2 * (3 * r + ca)], p[2 * (3 * r + ca) + 1]);
                *reinterpret_cast<uint4*>(Gs + ca * blkg + (sl >> 3) * sbog + co * 128 + rowoff) =
                    make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
        tc::fence_proxy_async();
        if (__syncthreads_or(wait_failed)) {
            failed = true;
            break;
        }
        if (tid == 0) {
            tc::fence_after();
            const uint32_t xa = tc::smem_addr(Xs), ga = tc::smem_addr(Gs);
            for (int ca = 0; ca < 3; ++ca)
                for (int ks = 0; ks < NTC_TS / 16; ++ks)
                    tc::mma_bf16(tmem, tc::smem_desc(xa + ca * blkx + ks * 2 * sbox, sbox, 128),
                                 tc::smem_desc(ga + ca * blkg + ks * 2 * sbog, sbog, 128), idesc,
                                 (k > 0 || ca > 0 || ks > 0) ? 1u : 0u);
            tc::commit(mma_bar);
        }
    }
    if (!failed && k > 0) {
        bool ok = tc::mbar_wait(mma_bar, (k - 1) & 1, a.wait_ns);
        // expiry test: then wait for the next phase, which nothing completes
        if (ok && a.expire_test) ok = tc::mbar_wait(mma_bar, ((k - 1) & 1) ^ 1u, a.wait_ns);
        if (__syncthreads_or(!ok)) failed = true;
    }
    if (!failed && k > 0) {
        tc::fence_after();
        // lane m = 8 h + 2 kk + {re, im} of hop h, input complex kk (4 per hop)
        const int q4 = warp & 3, wg = warp >> 2;
        const int m = 32 * q4 + lane;
        const int h = m >> 3, kk = (m & 7) >> 1;
        const uint32_t trow = tmem + ((uint32_t)(32 * q4) << 16);
        for (int c0 = 16 * wg; c0 < N2p; c0 += 16 * (NTC_THREADS / 128)) {
            uint32_t v[16];
            tc::ld_x16(trow + c0, v);
            tc::wait_ld();
            float pv[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) pv[j] = __shfl_xor_sync(0xffffffffu, __uint_as_float(v[j]), 1);
            if ((m & 1) == 0 && h < 9) {
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int n = c0 / 2 + i;
                    if (n >= nn) break;
                    float* dst = gW + (((size_t)h * nn + n) * 4 + kk) * 2;
                    atomicAdd(dst, __uint_as_float(v[2 * i]) + pv[2 * i + 1]);
                    atomicAdd(dst + 1, __uint_as_float(v[2 * i + 1]) - pv[2 * i]);
                }
            }
        }
    }
    if (failed) {  // bounded wait for this CTA's MMAs in flight, then free the tensor memory
        if (k > 0) tc::mbar_wait(mma_bar, (k - 1) & 1, NTC_WAIT_NS);
        if (tid == 0) atomicOr(a.errw, ERRW_TIMEOUT);
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

// BF16 weight gradient of a layer with one output channel (the last layer),
// all nine hops in one pass.  With X_h(x) = U_h(x) in(x + h) the gradient
// sum over (x, colour) of conj(X_h) G equals the sum over (y, colour) of
// conj(in(y)) (T_adj(h) G)(y): the transport moves to the one-channel
// output gradient (the adjoint hop, which brings G from x = y - h to y), and
// the input is read once per tile for every hop.  The hops' transported G
// are folded along N (72 of 80): D[k2][8 h + n'] over the rows (y, colour).
// One CTA per SM; operands single-buffered; all four thread groups gather.
template <int RECON>
__global__ void __launch_bounds__(NTC_THREADS, 1) net_wgrad_o1_kernel(const NetLayerArgs a, const float* gout, float* gW)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int MX = 128, G4 = NTC_THREADS / NTC_TS;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nk = 4 * a.cin;
    const uint32_t sbox = (MX / 8) * 128, sbog = (uint32_t)NC1_KG * 128;  // bytes between 8-site groups
    const uint32_t blkx = (uint32_t)NTC_TS * MX * 2, blkg = (uint32_t)NTC_TS * NC1_K * 2;
    unsigned char* const Xs = smem;
    unsigned char* const Gs = smem + 3 * blkx;
    uint64_t* mma_bar = reinterpret_cast<uint64_t*>(Gs + 3 * blkg);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mma_bar + 1);
    const uint32_t idesc = tc::idesc_bf16_f32(MX, NC1_K) | (1u << 15) | (1u << 16);  // A and B MN-major
    const uint32_t ncols = (uint32_t)a.tmem_cols;

    for (uint32_t e = tid; e < 3 * (blkx + blkg) / 16; e += NTC_THREADS)  // M and N padding stays zero
        reinterpret_cast<uint4*>(smem)[e] = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) tc::mbar_init(mma_bar, 1);
    if (warp == 0) tc::tmem_alloc(tslot, ncols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;

    const int ntiles = (a.V + NTC_TS - 1) / NTC_TS;
    const int total = ntiles * a.batch;
    const int sl = tid & (NTC_TS - 1), grp = tid / NTC_TS;
    const uint32_t rowoff = (sl & 7) * 16;
    uint32_t k = 0;
    bool wait_failed = false, failed = false;
    for (int t = blockIdx.x; t < total; t += gridDim.x, ++k) {
        const int b = t / ntiles, y = (t - b * ntiles) * NTC_TS + sl;
        if (k >= 1 && !wait_failed) wait_failed = !tc::mbar_wait(mma_bar, (k - 1) & 1, a.wait_ns);
        // A: the input channels grp, grp + 4, ... at the site, untransported
        for (int ci = grp; ci < a.cin; ci += G4) {
            float p[24];
            load_act(a.in, a.in_bf16, a.V, a.cin, b, ci, y < a.V ? y : -1, p);
#pragma unroll
            for (int ca = 0; ca < 3; ++ca) {
                uint32_t w[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) w[r] = pack_bf16x2(p[2 * (3 * r + ca)], p[2 * (3 * r + ca) + 1]);
                *reinterpret_cast<uint4*>(Xs + ca * blkx + (sl >> 3) * sbox + ci * 128 + rowoff) =
                    make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
        // B: the output gradient brought to the site by the adjoint of hops grp, grp + 4, grp + 8
        for (int h = grp; h < 9; h += G4) {
            float u[18], p[24];
            float sign = 1.f;
            int src = -1;
#pragma unroll
            for (int q = 0; q < 18; ++q) u[q] = 0.f;  // padding sites: zero link, zero input
            if (y < a.V) {
                if (h > 0) {
                    src = hop_link<RECON>(a, y, adj_hop(h), u, sign);
#pragma unroll
                    for (int q = 0; q < 18; ++q) u[q] = sign * u[q];
                } else {
                    src = y;
                }
            }
            load_act(gout, a.gout_bf16, a.V, 1, b, 0, src, p);
#pragma unroll
            for (int ca = 0; ca < 3; ++ca) {
                uint32_t w[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    float re, im;
                    if (h == 0) {
                        re = p[2 * (3 * r + ca)];
                        im = p[2 * (3 * r + ca) + 1];
                    } else {
                        re = 0.f;
                        im = 0.f;
#pragma unroll
                        for (int cb = 0; cb < 3; ++cb) {  // one multiply-add per real product
                            const float ur = u[2 * (3 * ca + cb)], ui = u[2 * (3 * ca + cb) + 1];
                            const float pr = p[2 * (3 * r + cb)], pi = p[2 * (3 * r + cb) + 1];
                            re += ur * pr;
                            re -= ui * pi;
                            im += ur * pi;
                            im += ui * pr;
                        }
                    }
                    w[r] = pack_bf16x2(re, im);
                }
                *reinterpret_cast<uint4*>(Gs + ca * blkg + (sl >> 3) * sbog + h * 128 + rowoff) =
                    make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
        tc::fence_proxy_async();
        if (__syncthreads_or(wait_failed)) {
            failed = true;
            break;
        }
        if (tid == 0) {
            tc::fence_after();
            const uint32_t xa = tc::smem_addr(Xs), ga = tc::smem_addr(Gs);
            for (int ca = 0; ca < 3; ++ca)
                for (int ks = 0; ks < NTC_TS / 16; ++ks)
                    tc::mma_bf16(tmem, tc::smem_desc(xa + ca * blkx + ks * 2 * sbox, sbox, 128),
                                 tc::smem_desc(ga + ca * blkg + ks * 2 * sbog, sbog, 128), idesc,
                                 (k > 0 || ca > 0 || ks > 0) ? 1u : 0u);
            tc::commit(mma_bar);
        }
    }
    if (!failed && k > 0) {
        bool ok = tc::mbar_wait(mma_bar, (k - 1) & 1, a.wait_ns);
        // expiry test: then wait for the next phase, which nothing completes
        if (ok && a.expire_test) ok = tc::mbar_wait(mma_bar, ((k - 1) & 1) ^ 1u, a.wait_ns);
        if (__syncthreads_or(!ok)) failed = true;
    }
    if (!failed && k > 0) {
        tc::fence_after();
        // lane k2 = 2 kk + {re, im} (input complex kk); column 8 h + 2 n + {re, im}
        const int q4 = warp & 3, wg = warp >> 2;
        const int k2 = 32 * q4 + lane;
        const int kk = k2 >> 1;
        const uint32_t trow = tmem + ((uint32_t)(32 * q4) << 16);
        for (int c0 = 16 * wg; c0 < NC1_K; c0 += 16 * (NTC_THREADS / 128)) {
            uint32_t v[16];
            tc::ld_x16(trow + c0, v);
            tc::wait_ld();
            float pv[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) pv[j] = __shfl_xor_sync(0xffffffffu, __uint_as_float(v[j]), 1);
            if ((k2 & 1) == 0 && kk < nk) {
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int col = c0 + 2 * i, h = col >> 3, n = (col & 7) >> 1;
                    if (h >= 9) break;
                    float* dst = gW + (((size_t)h * 4 + n) * nk + kk) * 2;
                    atomicAdd(dst, __uint_as_float(v[2 * i]) + pv[2 * i + 1]);
                    atomicAdd(dst + 1, __uint_as_float(v[2 * i + 1]) - pv[2 * i]);
                }
            }
        }
    }
    if (failed) {  // bounded wait for this CTA's MMAs in flight, then free the tensor memory
        if (k > 0) tc::mbar_wait(mma_bar, (k - 1) & 1, NTC_WAIT_NS);
        if (tid == 0) atomicOr(a.errw, ERRW_TIMEOUT);
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

// BF16 weight gradient of a multi-channel layer, pipelined like the forward:
// D_h^T[n2][k2] = sum over rows (site, colour) of G[row][n2] X_h[row][k2],
// so the output gradient G (M = n2, padded to 128) is the A operand and the
// transported input X_h (N = k2) the B operand.  A CTA takes one group of
// hops (blockIdx.y: hops 0-4 or 5-8, their accumulators side by side in
// tensor memory) over a stride of the batch x site tiles of 64 sites.  Each
// (tile, hop) is a stage: X_h double-buffered, G loaded once per tile (two
// buffers, by tile parity), the links of the next stage staged by thread
// group 0 while groups 1-7 gather this stage's channels one item ahead.
enum { WG_TS = 64, WG_HOPS = 5, WG_MN = 128 };

__device__ __forceinline__ int site_neighbour(const NetLayerArgs& a, int x, int h)
{
    const int c0 = x % a.L[0], c1 = (x / a.L[0]) % a.L[1], c2 = (x / (a.L[0] * a.L[1])) % a.L[2],
              c3 = x / (a.L[0] * a.L[1] * a.L[2]);
    return hop_neighbour(a, x, c0, c1, c2, c3, h);
}

template <int RECON>
__global__ void __launch_bounds__(NTC_THREADS, 1) net_wgrad_hg_kernel(const NetLayerArgs a, const float* gout, float* gW)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int NG = NTC_THREADS / WG_TS;  // 8 thread groups of 64
    constexpr int TG = NG - 1;               // gathering groups 1..7
    constexpr int CPT = (NET_MAXC + TG - 1) / TG;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int K2p = a.K2p, nk = 4 * a.cin, nn = 4 * a.cout;
    const int h0 = blockIdx.y * WG_HOPS, nh = (9 - h0) < WG_HOPS ? (9 - h0) : WG_HOPS;
    const uint32_t sbox = (uint32_t)(K2p / 8) * 128, sbog = (WG_MN / 8) * 128;  // bytes between 8-site groups
    const uint32_t blkx = (uint32_t)WG_TS * K2p * 2, blkg = (uint32_t)WG_TS * WG_MN * 2;
    unsigned char* const Xs = smem;                  // [2][3][blkx]
    unsigned char* const Gs = smem + 6 * blkx;       // [2][3][blkg]
    float* lbuf = reinterpret_cast<float*>(Gs + 6 * blkg);                        // [2][WG_TS][19]
    uint64_t* mma_bar = reinterpret_cast<uint64_t*>(lbuf + 2 * WG_TS * 19);       // [2]
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mma_bar + 2);
    const uint32_t idesc = tc::idesc_bf16_f32(WG_MN, K2p) | (1u << 15) | (1u << 16);  // A and B MN-major
    const uint32_t ncols = (uint32_t)a.tmem_cols;

    for (uint32_t e = tid; e < 6 * (blkx + blkg) / 16; e += NTC_THREADS)  // channel and n2 padding stays zero
        reinterpret_cast<uint4*>(smem)[e] = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) {
        tc::mbar_init(&mma_bar[0], 1);
        tc::mbar_init(&mma_bar[1], 1);
    }
    if (warp == 0) tc::tmem_alloc(tslot, ncols);

    const int ntiles = (a.V + WG_TS - 1) / WG_TS;
    const int total = ntiles * a.batch;
    const int sl = tid & (WG_TS - 1), grp = tid / WG_TS;
    const uint32_t rowoff = (sl & 7) * 16;
    const int cfirst = grp - 1;
    const int nj = (grp > 0 && cfirst < a.cin) ? (a.cin - cfirst + TG - 1) / TG : 0;
    // links of hop h at site x into slot `slot` (group 0): times the boundary sign, zero past V or for h = 0
    auto stage_links = [&](int x, int h, int slot) {
        float un[18];
        float sign = 1.f;
        if (x < a.V && h > 0) {
            hop_link<RECON>(a, x, h, un, sign);
        } else {
#pragma unroll
            for (int q = 0; q < 18; ++q) un[q] = 0.f;
        }
        float* ls = lbuf + (slot * WG_TS + sl) * 19;
#pragma unroll
        for (int q = 0; q < 18; ++q) ls[q] = sign * un[q];
    };
    float nxt[24];
    if ((int)blockIdx.x < total) {
        const int t = blockIdx.x, b = t / ntiles, x = (t - b * ntiles) * WG_TS + sl;
        if (grp == 0) stage_links(x, h0, 0);
        if (nj > 0) load_act(a.in, a.in_bf16, a.V, a.cin, b, cfirst, x < a.V ? site_neighbour(a, x, h0) : -1, nxt);
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;

    uint32_t g = 0;  // stages whose MMAs were issued (stage g commits to mma_bar[g & 1])
    int q = 0;       // tiles of this CTA so far
    bool wait_failed = false, failed = false;
    for (int t = blockIdx.x; t < total && !failed; t += gridDim.x, ++q) {
        const int b = t / ntiles, x = (t - b * ntiles) * WG_TS + sl;
        const int tn = t + gridDim.x;
        const int bn = tn / ntiles, xn = (tn - bn * ntiles) * WG_TS + sl;
        for (int hl = 0; hl < nh; ++hl) {
            const int h = h0 + hl, s = g & 1;
            // X stage s (and the G buffer of this tile's parity) is free once stage g - 2's MMAs completed
            if (g >= 2 && !wait_failed) wait_failed = !tc::mbar_wait(&mma_bar[s], ((g - 2) >> 1) & 1u, a.wait_ns);
            // the next stage: hop h + 1 of this tile, else the first hop of the next tile
            const bool last = hl + 1 == nh;
            const int xs = last ? xn : x, hs = last ? h0 : h + 1;
            const bool more = !last || tn < total;
            if (grp == 0 && more) stage_links(xs, hs, (g + 1) & 1);
            unsigned char* const Gb = Gs + (q & 1) * 3 * blkg;
            if (hl == 0) {  // the output gradient at the tile's sites, once per tile
                for (int co = grp; co < a.cout; co += NG) {
                    float p[24];
                    load_act(gout, a.gout_bf16, a.V, a.cout, b, co, x < a.V ? x : -1, p);
#pragma unroll
                    for (int ca = 0; ca < 3; ++ca) {
                        uint32_t w[4];
#pragma unroll
                        for (int r = 0; r < 4; ++r) w[r] = pack_bf16x2(p[2 * (3 * r + ca)], p[2 * (3 * r + ca) + 1]);
                        *reinterpret_cast<uint4*>(Gb + ca * blkg + (sl >> 3) * sbog + co * 128 + rowoff) =
                            make_uint4(w[0], w[1], w[2], w[3]);
                    }
                }
            }
            float u[18];
            if (nj > 0) {
                const float* ls = lbuf + (s * WG_TS + sl) * 19;
#pragma unroll
                for (int k = 0; k < 18; ++k) u[k] = ls[k];
            }
            const int yh = x < a.V ? site_neighbour(a, x, h) : -1;
            unsigned char* const Xb = Xs + s * 3 * blkx;
#pragma unroll
            for (int j = 0; j < CPT; ++j) {
                if (j >= nj) break;
                const int ci = cfirst + TG * j;
                float cur[24];
#pragma unroll
                for (int k = 0; k < 24; ++k) cur[k] = nxt[k];
                if (j + 1 < nj) {
                    load_act(a.in, a.in_bf16, a.V, a.cin, b, ci + TG, yh, nxt);
                } else if (more) {
                    load_act(a.in, a.in_bf16, a.V, a.cin, last ? bn : b, cfirst,
                             xs < a.V ? site_neighbour(a, xs, hs) : -1, nxt);
                }
#pragma unroll
                for (int ca = 0; ca < 3; ++ca) {
                    uint32_t w[4];
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        float re, im;
                        if (h == 0) {
                            re = cur[2 * (3 * r + ca)];
                            im = cur[2 * (3 * r + ca) + 1];
                        } else {
                            re = 0.f;
                            im = 0.f;
#pragma unroll
                            for (int cb = 0; cb < 3; ++cb) {  // one multiply-add per real product
                                const float ur = u[2 * (3 * ca + cb)], ui = u[2 * (3 * ca + cb) + 1];
                                const float pr = cur[2 * (3 * r + cb)], pi = cur[2 * (3 * r + cb) + 1];
                                re += ur * pr;
                                re -= ui * pi;
                                im += ur * pi;
                                im += ui * pr;
                            }
                        }
                        w[r] = pack_bf16x2(re, im);
                    }
                    *reinterpret_cast<uint4*>(Xb + ca * blkx + (sl >> 3) * sbox + ci * 128 + rowoff) =
                        make_uint4(w[0], w[1], w[2], w[3]);
                }
            }
            tc::fence_proxy_async();
            if (__syncthreads_or(wait_failed)) {
                failed = true;
                break;
            }
            if (tid == 0) {
                tc::fence_after();
                const uint32_t ga = tc::smem_addr(Gb), xa = tc::smem_addr(Xb);
                for (int ca = 0; ca < 3; ++ca)
                    for (int ks = 0; ks < WG_TS / 16; ++ks)
                        tc::mma_bf16(tmem + hl * K2p, tc::smem_desc(ga + ca * blkg + ks * 2 * sbog, sbog, 128),
                                     tc::smem_desc(xa + ca * blkx + ks * 2 * sbox, sbox, 128), idesc,
                                     (q > 0 || ca > 0 || ks > 0) ? 1u : 0u);
                tc::commit(&mma_bar[s]);
            }
            ++g;
        }
    }
    if (!failed && g > 0) {
        const uint32_t gl = g - 1;
        bool ok = tc::mbar_wait(&mma_bar[gl & 1], (gl >> 1) & 1u, a.wait_ns);
        // expiry test: then wait for the next phase, which nothing completes
        if (ok && a.expire_test) ok = tc::mbar_wait(&mma_bar[gl & 1], ((gl >> 1) & 1u) ^ 1u, a.wait_ns);
        if (__syncthreads_or(!ok)) failed = true;
    }
    if (!failed && g > 0) {
        tc::fence_after();
        // lane n2 = 2 n + {re, im} (output complex n); column hl K2p + 2 kk + {re, im}
        const int q4 = warp & 3, wg = warp >> 2;
        const int n2 = 32 * q4 + lane, n = n2 >> 1;
        const uint32_t trow = tmem + ((uint32_t)(32 * q4) << 16);
        for (int hl = 0; hl < nh; ++hl)
            for (int c0 = 16 * wg; c0 < K2p; c0 += 16 * (NTC_THREADS / 128)) {
                uint32_t v[16];
                tc::ld_x16(trow + hl * K2p + c0, v);
                tc::wait_ld();
                float pv[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) pv[j] = __shfl_xor_sync(0xffffffffu, __uint_as_float(v[j]), 1);
                if ((n2 & 1) == 0 && n < nn) {
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int kk = (c0 >> 1) + i;
                        if (kk >= nk) break;
                        float* dst = gW + (((size_t)(h0 + hl) * nn + n) * nk + kk) * 2;
                        atomicAdd(dst, __uint_as_float(v[2 * i]) + pv[2 * i + 1]);
                        atomicAdd(dst + 1, pv[2 * i] - __uint_as_float(v[2 * i + 1]));
                    }
                }
            }
    }
    if (failed) {  // bounded wait for this CTA's MMAs in flight, then free the tensor memory
        if (g > 0) {
            const uint32_t gl = g - 1;
            tc::mbar_wait(&mma_bar[gl & 1], (gl >> 1) & 1u, NTC_WAIT_NS);
        }
        if (tid == 0) atomicOr(a.errw, ERRW_TIMEOUT);
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

// FP32 forward of one layer (64-site tiles, one CTA each, batch in blockIdx.y).
template <int RECON>
__global__ void __launch_bounds__(NET_THREADS) net_layer_kernel(const NetLayerArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int tile0 = blockIdx.x * NET_TS;
    const int b = blockIdx.y;
    const float* in_b = a.in + (size_t)b * a.V * a.cin * 24;
    float* out_b = a.out + (size_t)b * a.V * a.cout * 24;
    const int tid = threadIdx.x;
    // shared: X [192][K2 + 4] f32, B [K2][N2 + 4] f32; thread tile 6 rows x 12 cols
    const int xs = a.K2p + 4, bs = a.N2p + 4;
    float* Xs = reinterpret_cast<float*>(smem);
    float* Bs = Xs + NET_ROWS * xs;
    const int rb = tid / 8, cb = tid % 8;  // 32 row blocks x 8 column blocks
    float acc[6][12];
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = 0; j < 12; ++j) acc[i][j] = 0.f;
    for (int h = 0; h < 9; ++h) {
        gather_hop<RECON>(a, in_b, tile0, h, Xs, xs);
        const float* Bg = a.Bf + (size_t)h * a.K2 * a.N2;
        for (int e = tid; e < a.K2 * a.N2; e += NET_THREADS) Bs[(e / a.N2) * bs + e % a.N2] = Bg[e];
        __syncthreads();
        for (int k = 0; k < a.K2; ++k) {
            float xv[6], bv[12];
#pragma unroll
            for (int i = 0; i < 6; ++i) xv[i] = Xs[(rb * 6 + i) * xs + k];
#pragma unroll
            for (int j = 0; j < 12; ++j) bv[j] = (cb * 12 + j < a.N2) ? Bs[k * bs + cb * 12 + j] : 0.f;
#pragma unroll
            for (int i = 0; i < 6; ++i)
#pragma unroll
                for (int j = 0; j < 12; ++j) acc[i][j] = fmaf(xv[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const int row = rb * 6 + i;
        const int site = tile0 + row / 3, col = row % 3;
        if (site >= a.V) continue;
#pragma unroll
        for (int j = 0; j < 12; j += 2) {
            const int n2 = cb * 12 + j;
            if (n2 < a.N2) {
                const int n = n2 / 2;  // n = co * 4 + spin
                reinterpret_cast<float2*>(out_b)[planar_c(a.V, n >> 2, 3 * (n & 3) + col, site)] =
                    make_float2(acc[i][j], acc[i][j + 1]);
            }
        }
    }
}

// Weight gradient of one layer: G_h[n][k] += sum_{x, a} Gout(x)[n][a] conj((T_h in)(x)[k][a])
// (complex, = dL/dRe W + i dL/dIm W).  One CTA per (tile range, hop); FP32
// partial sums, added to gW with atomics.
template <int RECON>
__global__ void __launch_bounds__(NET_THREADS) net_wgrad_kernel(const NetLayerArgs a, const float* gout, int batch,
                                                                float* gW)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int h = blockIdx.y;
    const int nk = 4 * a.cin, nn = 4 * a.cout;
    const int xs = a.K2p + 4;
    float* Xs = reinterpret_cast<float*>(smem);              // [192][K2p + 4]
    float* Gs = Xs + NET_ROWS * xs;                           // [192][2 nn]
    const int ntiles = (a.V + NET_TS - 1) / NET_TS;
    const int total = ntiles * batch;
    const int npair = nn * nk;
    float accr[9], acci[9];  // up to 9 (n, k) pairs per thread (48 x 48 / 256)
#pragma unroll
    for (int q = 0; q < 9; ++q) accr[q] = acci[q] = 0.f;
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int b = t / ntiles, tile0 = (t % ntiles) * NET_TS;
        gather_hop<RECON>(a, a.in + (size_t)b * a.V * a.cin * 24, tile0, h, Xs, xs);
        const float* gb = gout + (size_t)b * a.V * a.cout * 24;
        for (int e = threadIdx.x; e < NET_ROWS * nn; e += NET_THREADS) {
            const int row = e / nn, n = e % nn;
            const int site = tile0 + row / 3, col = row % 3;
            float2 v = make_float2(0.f, 0.f);
            if (site < a.V) v = reinterpret_cast<const float2*>(gb)[planar_c(a.V, n >> 2, 3 * (n & 3) + col, site)];
            Gs[row * 2 * nn + 2 * n] = v.x;
            Gs[row * 2 * nn + 2 * n + 1] = v.y;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const int pidx = threadIdx.x + q * NET_THREADS;
            if (pidx >= npair) break;
            const int n = pidx / nk, k = pidx % nk;
            float sr = 0.f, si = 0.f;
            for (int row = 0; row < NET_ROWS; ++row) {
                const float gr = Gs[row * 2 * nn + 2 * n], gi = Gs[row * 2 * nn + 2 * n + 1];
                const float xr = Xs[row * xs + 2 * k], xi = Xs[row * xs + 2 * k + 1];
                sr += gr * xr + gi * xi;  // g conj(x)
                si += gi * xr - gr * xi;
            }
            accr[q] += sr;
            acci[q] += si;
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        const int pidx = threadIdx.x + q * NET_THREADS;
        if (pidx >= npair) break;
        const int n = pidx / nk, k = pidx % nk;
        float* dst = gW + (((size_t)h * nn + n) * nk + k) * 2;
        atomicAdd(dst, accr[q]);
        atomicAdd(dst + 1, acci[q]);
    }
}

// Real-ified weights from complex W[h][n][k]: FP32 B[h][k2][n2] and BF16
// Bh[h] (N2p x K2p, zero padded), the latter in the tensor cores' K-major
// core-matrix order: element (n2, k2) at (n2/8) (K2p/8) 64 + (k2/8) 64 +
// (n2%8) 8 + k2%8.  With W' = adjoint-hop conjugate transpose when
// `adjoint` (the layer's input gradient).
__global__ void net_prep_weights_kernel(const float* W, int cin, int cout, int adjoint, float* Bf, uint16_t* Bh,
                                        int K2p, int N2p)
{
    // effective layer: inputs ki (4 * cin_eff), outputs no (4 * cout_eff)
    const int cin_e = adjoint ? cout : cin, cout_e = adjoint ? cin : cout;
    const int nk = 4 * cin_e, nn = 4 * cout_e;
    const int K2 = 2 * nk, N2 = 2 * nn;
    const int total = 9 * N2p * K2p;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int h = e / (N2p * K2p);
        const int n2 = (e / K2p) % N2p, k2 = e % K2p;
        float v = 0.f;
        if (n2 < N2 && k2 < K2) {
            const int n = n2 / 2, k = k2 / 2;
            float wr, wi;
            if (adjoint) {  // W'_h[n][k] = conj(W_{adj h}[k][n]), W stored [h][4 cout][4 cin]
                const float* w = W + (((size_t)adj_hop(h) * (4 * cout) + k) * (4 * cin) + n) * 2;
                wr = w[0];
                wi = -w[1];
            } else {
                const float* w = W + (((size_t)h * nn + n) * nk + k) * 2;
                wr = w[0];
                wi = w[1];
            }
            // out_re += wr x_re - wi x_im ; out_im += wi x_re + wr x_im
            if ((n2 & 1) == 0) v = (k2 & 1) == 0 ? wr : -wi;
            else v = (k2 & 1) == 0 ? wi : wr;
            Bf[((size_t)h * K2 + k2) * N2 + n2] = v;
        }
        Bh[(size_t)h * N2p * K2p + (n2 / 8) * (K2p / 8) * 64 + (k2 / 8) * 64 + (n2 % 8) * 8 + k2 % 8] = f2bf(v);
    }
}

// Stacked weights of a layer with one output channel, for the contraction
// before the transport: one "hop" whose outputs n2' = 8 h + n2 are the nine
// hops' real-ified outputs (Z_h = W_h in, spin and re / im), BF16 in the same
// core-matrix order as net_prep_weights_kernel.
__global__ void net_prep_stacked_kernel(const float* W, int cin, uint16_t* Bh, int K2p, int N2p)
{
    const int nk = 4 * cin, K2 = 2 * nk;
    const int total = N2p * K2p;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int n2s = e / K2p, k2 = e % K2p;
        float v = 0.f;
        if (n2s < 72 && k2 < K2) {
            const int h = n2s / 8, n2 = n2s % 8, n = n2 / 2, k = k2 / 2;
            const float* w = W + (((size_t)h * 4 + n) * nk + k) * 2;
            const float wr = w[0], wi = w[1];
            if ((n2 & 1) == 0) v = (k2 & 1) == 0 ? wr : -wi;
            else v = (k2 & 1) == 0 ? wi : wr;
        }
        Bh[(n2s / 8) * (K2p / 8) * 64 + (k2 / 8) * 64 + (n2s % 8) * 8 + k2 % 8] = f2bf(v);
    }
}

// Transport after the contraction for a layer with one output channel:
// out(x) = Z_0(x) + sum_{h >= 1} U_h(x) Z_h(x + h) (fermion sign included),
// Z_h = W_h in the stacked contraction's nine BF16 channels.  W_h acts on
// spin and channel, U_h on colour, so the two commute: four colour vectors
// are transported per hop instead of 4 C_in.  Output: one FP32 channel.
template <int RECON>
__global__ void __launch_bounds__(128) net_gather_transport_kernel(const NetLayerArgs a, const void* z, float* out)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    if (x >= a.V) return;
    float acc[24];
    load_act(z, 1, a.V, 9, b, 0, x, acc);
    for (int h = 1; h < 9; ++h) {
        float u[18], sign;
        const int y = hop_link<RECON>(a, x, h, u, sign);
        float p[24];
        load_act(z, 1, a.V, 9, b, h, y, p);
#pragma unroll
        for (int sp = 0; sp < 4; ++sp)
#pragma unroll
            for (int ca = 0; ca < 3; ++ca) {
                float re = 0.f, im = 0.f;
#pragma unroll
                for (int cb = 0; cb < 3; ++cb) {  // one multiply-add per real product
                    const float ur = u[2 * (3 * ca + cb)], ui = u[2 * (3 * ca + cb) + 1];
                    const float pr = p[2 * (3 * sp + cb)], pi = p[2 * (3 * sp + cb) + 1];
                    re += ur * pr;
                    re -= ui * pi;
                    im += ur * pi;
                    im += ui * pr;
                }
                acc[2 * (3 * sp + ca)] += sign * re;
                acc[2 * (3 * sp + ca) + 1] += sign * im;
            }
    }
    float4* o = reinterpret_cast<float4*>(out) + (size_t)b * a.V * 6;
#pragma unroll
    for (int q = 0; q < 6; ++q) o[plane4(a.V, 0, q) + x] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
}

// Canonical complex spinor (Cin = 1 activation) <-> internal FP32 full field.
__global__ void net_from_internal_kernel(Geom g, const char* in, size_t in_rb, float* act, int L0, int nb)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int par = blockIdx.y % 2, b = blockIdx.y / 2;
    if (i >= g.Vh || b >= nb) return;
    int c[4];
    cb_coords(g, i, par, c);
    const size_t V = (size_t)2 * g.Vh;
    float v[24];
    SpinorIO<P32>::load(in + b * in_rb + par * spinor_field_bytes(P32, g.stride), g.stride, i, v);
    float4* dst = reinterpret_cast<float4*>(act) + (size_t)b * V * 6 + full_index(g, c);
#pragma unroll
    for (int k = 0; k < 6; ++k) dst[(size_t)k * V] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
}

__global__ void net_to_internal_kernel(Geom g, char* out, size_t out_rb, const float* act, int nb)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int par = blockIdx.y % 2, b = blockIdx.y / 2;
    if (i >= g.Vh || b >= nb) return;
    int c[4];
    cb_coords(g, i, par, c);
    const size_t V = (size_t)2 * g.Vh;
    const float4* src = reinterpret_cast<const float4*>(act) + (size_t)b * V * 6 + full_index(g, c);
    float v[24];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        float4 q = src[(size_t)k * V];
        v[4 * k] = q.x; v[4 * k + 1] = q.y; v[4 * k + 2] = q.z; v[4 * k + 3] = q.w;
    }
    SpinorIO<P32>::store(out + b * out_rb + par * spinor_field_bytes(P32, g.stride), g.stride, i, v);
}

// Canonical [b][site][ch][4][3] complex <-> planar activations of nb batch
// items (to_planar = 1: canonical -> planar).  Thread e walks the planar
// order, so the planar side is coalesced.
__global__ void net_layout_kernel(const float4* src, float4* dst, int V, int ch, int nb, int to_planar)
{
    const size_t per = (size_t)V * ch * 6, total = per * nb;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const size_t b = e / per, r = e - b * per;
        const size_t site = r % V, cq = r / V;
        const size_t can = b * per + (site * ch + cq / 6) * 6 + cq % 6;
        if (to_planar) dst[e] = src[can];
        else dst[can] = src[e];
    }
}

// Canonical FP32 <-> BF16 planar: plane q of channel c holds complex 4q .. 4q+3
// (two canonical float4) of every site, as eight BF16 values.
__global__ void net_layout_bf16_kernel(const void* src, void* dst, int V, int ch, int nb, int to_planar)
{
    const size_t per = (size_t)V * ch * 3, total = per * nb;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const size_t b = e / per, r = e - b * per;
        const size_t site = r % V, cq = r / V;
        const size_t can = (b * (size_t)V * ch + site * ch + cq / 3) * 6 + 2 * (cq % 3);  // float4 index
        if (to_planar) {
            const float4* s4 = static_cast<const float4*>(src);
            const float4 x = s4[can], y = s4[can + 1];
            static_cast<uint4*>(dst)[e] = make_uint4(pack_bf16x2(x.x, x.y), pack_bf16x2(x.z, x.w), pack_bf16x2(y.x, y.y),
                                                     pack_bf16x2(y.z, y.w));
        } else {
            const uint4 v = static_cast<const uint4*>(src)[e];
            float4* d4 = static_cast<float4*>(dst);
            d4[can] = make_float4(__uint_as_float(v.x << 16), __uint_as_float(v.x & 0xffff0000u),
                                  __uint_as_float(v.y << 16), __uint_as_float(v.y & 0xffff0000u));
            d4[can + 1] = make_float4(__uint_as_float(v.z << 16), __uint_as_float(v.z & 0xffff0000u),
                                      __uint_as_float(v.w << 16), __uint_as_float(v.w & 0xffff0000u));
        }
    }
}

// Loss L = (1/B) sum_b |y_b - e_b|^2 / |e_b|^2; gout_b = 2 (y_b - e_b) / (B |e_b|^2).
// Pass 1 reduces |y - e|^2 and |e|^2 per batch item (deterministic two-stage).
__global__ void net_loss_reduce_kernel(const float* y, const float* e, size_t n_per, double* partials, size_t part_rs,
                                       unsigned* tickets, double* red)
{
    const int b = blockIdx.y;
    double d2 = 0.0, e2 = 0.0;
    const float* yb = y + (size_t)b * n_per;
    const float* eb = e + (size_t)b * n_per;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_per; i += (size_t)gridDim.x * blockDim.x) {
        const float d = yb[i] - eb[i];
        d2 += (double)d * d;
        e2 += (double)eb[i] * eb[i];
    }
    double v[2] = {d2, e2};
    block_reduce_finalize<2>(v, partials + b * part_rs, tickets + b, red + b * 2);
}

__global__ void net_loss_grad_kernel(const float* y, const float* e, size_t n_per, const double* red, int nb, float* g)
{
    const int b = blockIdx.y;
    const float s = (float)(2.0 / (nb * red[2 * b + 1]));
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_per; i += (size_t)gridDim.x * blockDim.x)
        g[(size_t)b * n_per + i] = s * (y[(size_t)b * n_per + i] - e[(size_t)b * n_per + i]);
}

// Adam on real parameters (re and im of W separately).
__global__ void net_adam_kernel(float* w, float* m, float* v, const float* g, int n, float lr, float b1, float b2,
                                float eps, float c1, float c2)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

}  // namespace lqcd

// ------------------------------------------------------------------ host side

using namespace lqcd;

// CUDA-event timing of the layer and weight-gradient launches (while enabled).
struct NetProfiler {
    struct Rec { int idx; cudaEvent_t a, b; double bytes, flops; };
    bool on = false;
    std::vector<cudaEvent_t> pool;
    std::vector<Rec> pending;
    cudaEvent_t get()
    {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        return e;
    }
    ~NetProfiler()
    {
        for (auto e : pool) cudaEventDestroy(e);
        for (auto& r : pending) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    }
};

struct lqcd_net {
    NetProfiler* prof;     // null unless lqcd_net_profile_enable was called
    lqcd_ctx* ctx;
    int nlayers;
    int ch[8];             // channels, ch[0] = ch[nlayers] = 1
    int bf16;              // 1: tensor-core BF16 operands
    int max_batch;
    char* ws;
    size_t ws_bytes, need;
    // carve-up
    float* W;              // FP32 master weights, layer l at woff[l] (complex)
    float* gW;             // gradients
    float* m1;             // Adam moments
    float* m2;
    float* Bf[8];          // real-ified FP32 weights per layer (forward)
    uint16_t* Bh[8];
    float* BfA[8];         // adjoint (input-gradient) weights
    uint16_t* BhA[8];
    uint16_t* BhS[8];      // stacked BF16 weights of layers with one output channel (stacked[l])
    int stacked[8];        // layer l contracts before it transports (BF16, C_out = 1 < C_in)
    float* zbuf;           // the stacked contraction's nine BF16 channels, max_batch items (any stacked)
    float* act[9];         // planar activations per layer boundary, max_batch items
    float* gact[2];        // gradient ping-pong buffers (max channels)
    double* red;           // loss reductions [max_batch][2]
    double* partials;      // loss reduction partials [max_batch][NET_PARTIALS][2]
    unsigned* tickets;     // [max_batch]
    size_t woff[9];        // float offsets of layer weights in W (layer nlayers = total)
    size_t boff[8], bhoff[8];
    long adam_t;
    int max_ctas;          // cap on the CTAs of the persistent tensor-core launches (0: one per SM)
    unsigned long long wait_ns = NTC_WAIT_NS;  // bound of the tensor-core kernels' mbarrier waits
    int expire_test = 0;   // lqcd_net_set_wait's test of the expiry path
    size_t nW() const { return woff[nlayers]; }
};

namespace {

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }
int pad16(int x) { return (x + 15) / 16 * 16; }

NetLayerArgs layer_args(const lqcd_net* n, int l, bool adjoint, const float* in, float* out)
{
    const lqcd_ctx* c = n->ctx;
    NetLayerArgs a;
    memset(&a, 0, sizeof a);
    for (int m = 0; m < 4; ++m) a.L[m] = c->g.L[m];
    a.V = 2 * c->g.Vh;
    a.stride = c->g.stride;
    a.tanti = c->g.tanti;
    a.gauge = c->gauge[P32];
    a.cin = adjoint ? n->ch[l + 1] : n->ch[l];
    a.cout = adjoint ? n->ch[l] : n->ch[l + 1];
    a.K2 = 8 * a.cin;
    a.N2 = 8 * a.cout;
    a.K2p = pad16(a.K2);
    a.N2p = pad16(a.N2);  // the M = 128 MMA takes N in multiples of 16
    a.in = in;
    a.out = out;
    a.Bf = adjoint ? n->BfA[l] : n->Bf[l];
    a.Bh = adjoint ? n->BhA[l] : n->Bh[l];
    a.batch = 1;
    int cols = 32;
    while (cols < 3 * a.N2p) cols *= 2;
    a.tmem_cols = cols;
    a.errw = c->errw;
    a.wait_ns = n->wait_ns;
    a.expire_test = n->expire_test;
    a.in_bf16 = n->bf16 && a.cin > 1;   // multi-channel activations of the BF16 network: BF16 planes
    a.out_bf16 = n->bf16 && a.cout > 1;
    a.nhops = 9;
    return a;
}

// Dynamic shared memory of the tensor-core kernel: two stages of X, B_h and
// links, four mbarriers and the tensor-memory address; at least NTC_MIN_SMEM, so
// that one CTA runs per SM and its tensor-memory allocation never waits.
size_t layer_smem_tc(const NetLayerArgs& a)
{
    const size_t need = 2 * ((size_t)3 * NTC_TS * a.K2p * 2 + (size_t)a.N2p * a.K2p * 2) + 2 * NTC_TS * 19 * 4 + 4 * 8 + 16;
    return need > (size_t)NTC_MIN_SMEM ? need : (size_t)NTC_MIN_SMEM;
}

size_t layer_smem_f32(const NetLayerArgs& a)
{
    return (size_t)NET_ROWS * (a.K2p + 4) * 4 + (size_t)a.K2 * (a.N2p + 4) * 4;
}

int sm_count()
{
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            sms = 0;
    }
    return sms;
}

// Algorithmic work of one layer launch over `batch` items: the channel
// contraction (8 real flops per complex multiply-add, 4 C_out x 4 C_in x 3
// colours x 9 hops per site) and the compulsory bytes (input activations,
// output activations or gradient, 96 bytes per channel and site in FP32 or
// 48 in BF16, each FP32 link once).
void layer_work(const NetLayerArgs& a, int batch, double& bytes, double& flops)
{
    const double V = (double)a.V * batch;
    flops = 8.0 * (4.0 * a.cout) * (4.0 * a.cin) * 3.0 * 9.0 * V;
    bytes = ((a.in_bf16 ? 48.0 : 96.0) * a.cin + (a.out_bf16 ? 48.0 : 96.0) * a.cout) * V +
            4.0 * gauge_link_bytes(P32, 12) * a.V;
}

// Event pair around one launch when profiling (not while capturing a graph).
struct NetTimed {
    lqcd_net* n;
    NetProfiler::Rec rec{};
    bool timed = false;
    lqcd_status begin(lqcd_net* net, int idx, double bytes, double flops);
    lqcd_status end();
};

lqcd_status run_layer(lqcd_net* n, const NetLayerArgs& a0, int batch, int prof_idx)
{
    lqcd_ctx* c = n->ctx;
    NetLayerArgs a = a0;
    a.batch = batch;
    double wb = 0.0, wf = 0.0;
    layer_work(a, batch, wb, wf);
    NetTimed tm;
    LQ_TRY(tm.begin(n, prof_idx, wb, wf));
    const int layer = prof_idx / 3, kind = prof_idx % 3;
    const bool stack = n->bf16 && kind == 0 && n->stacked[layer];
    NetLayerArgs z = a;  // the stacked contraction: one hop, nine "channels" Z_h = W_h in
    if (stack) {
        z.nhops = 1;
        z.cout = 9;
        z.N2 = 72;
        z.N2p = 80;
        z.Bh = n->BhS[layer];
        z.out = n->zbuf;
        z.out_bf16 = 1;
        int cols = 32;
        while (cols < 3 * z.N2p) cols *= 2;
        z.tmem_cols = cols;
    }
    if (n->bf16) {
        // persistent: one CTA per SM strides over the batch x site tiles
        const NetLayerArgs& t = stack ? z : a;
        const int sms = sm_count();
        if (sms <= 0) return fail(LQCD_ERR_CUDA, "net layer: no SM count");
        const int total = (t.V + NTC_TS - 1) / NTC_TS * batch;
        const size_t sm = layer_smem_tc(t);
        int grid = total < sms ? total : sms;
        if (n->max_ctas > 0 && grid > n->max_ctas) grid = n->max_ctas;
        if (t.cin == 1 && t.nhops == 9 && t.K2p == 16) {  // the hops folded into K
            const size_t sm1 = (size_t)2 * 3 * NTC_TS * NC1_K * 2 + (size_t)t.N2p * NC1_K * 2 + 2 * 8 + 16;
            if (c->cfg.recon == 12) {
                LQ_CUDA(cudaFuncSetAttribute(net_layer_c1_kernel<12>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1));
                net_layer_c1_kernel<12><<<grid, NTC_THREADS, sm1, c->stream>>>(t);
            } else {
                LQ_CUDA(cudaFuncSetAttribute(net_layer_c1_kernel<18>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1));
                net_layer_c1_kernel<18><<<grid, NTC_THREADS, sm1, c->stream>>>(t);
            }
        } else if (c->cfg.recon == 12) {
            LQ_CUDA(cudaFuncSetAttribute(net_layer_tc_kernel<12>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
            net_layer_tc_kernel<12><<<grid, NTC_THREADS, sm, c->stream>>>(t);
        } else {
            LQ_CUDA(cudaFuncSetAttribute(net_layer_tc_kernel<18>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
            net_layer_tc_kernel<18><<<grid, NTC_THREADS, sm, c->stream>>>(t);
        }
        if (stack) {  // then the transport of the four colour vectors per hop
            LQ_CUDA(cudaGetLastError());
            c->launches++;
            dim3 g2((a.V + 127) / 128, batch);
            if (c->cfg.recon == 12) net_gather_transport_kernel<12><<<g2, 128, 0, c->stream>>>(a, n->zbuf, a.out);
            else net_gather_transport_kernel<18><<<g2, 128, 0, c->stream>>>(a, n->zbuf, a.out);
        }
    } else {
        const size_t sm = layer_smem_f32(a);
        dim3 grid((a.V + NET_TS - 1) / NET_TS, batch);
        if (c->cfg.recon == 12) {
            LQ_CUDA(cudaFuncSetAttribute(net_layer_kernel<12>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
            net_layer_kernel<12><<<grid, NET_THREADS, sm, c->stream>>>(a);
        } else {
            LQ_CUDA(cudaFuncSetAttribute(net_layer_kernel<18>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
            net_layer_kernel<18><<<grid, NET_THREADS, sm, c->stream>>>(a);
        }
    }
    LQ_CUDA(cudaGetLastError());
    c->launches++;
    return tm.end();
}

lqcd_status prep_weights(lqcd_net* n)
{
    lqcd_ctx* c = n->ctx;
    for (int l = 0; l < n->nlayers; ++l)
        for (int adj = 0; adj < 2; ++adj) {
            NetLayerArgs a = layer_args(n, l, adj != 0, nullptr, nullptr);
            net_prep_weights_kernel<<<64, 256, 0, c->stream>>>(n->W + n->woff[l], n->ch[l], n->ch[l + 1], adj,
                                                               adj ? n->BfA[l] : n->Bf[l], adj ? n->BhA[l] : n->Bh[l],
                                                               a.K2p, a.N2p);
            LQ_CUDA(cudaGetLastError());
            c->launches++;
        }
    for (int l = 0; l < n->nlayers; ++l) {
        if (!n->stacked[l]) continue;
        net_prep_stacked_kernel<<<32, 256, 0, c->stream>>>(n->W + n->woff[l], n->ch[l], n->BhS[l], pad16(8 * n->ch[l]), 80);
        LQ_CUDA(cudaGetLastError());
        c->launches++;
    }
    return LQCD_OK;
}

size_t act_floats(const lqcd_net* n, int chn) { return (size_t)2 * n->ctx->g.Vh * chn * 24; }

// Canonical <-> planar copy of `batch` activations with `ch` channels.
lqcd_status convert_layout(lqcd_net* n, const float* src, float* dst, int ch, int batch, bool to_planar)
{
    lqcd_ctx* c = n->ctx;
    const int V = 2 * c->g.Vh;
    const size_t total = (size_t)V * ch * 6 * batch;
    const int grid = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
    if (n->bf16 && ch > 1)
        net_layout_bf16_kernel<<<grid, 256, 0, c->stream>>>(src, dst, V, ch, batch, to_planar ? 1 : 0);
    else
        net_layout_kernel<<<grid, 256, 0, c->stream>>>(reinterpret_cast<const float4*>(src), reinterpret_cast<float4*>(dst),
                                                       V, ch, batch, to_planar ? 1 : 0);
    LQ_CUDA(cudaGetLastError());
    c->launches++;
    return LQCD_OK;
}

// Weight gradient of one layer on planar activations (zeroing it first when `zero`).
lqcd_status run_wgrad(lqcd_net* n, int layer, const float* in, const float* gout, int batch, int zero)
{
    lqcd_ctx* c = n->ctx;
    float* gl = n->gW + n->woff[layer];
    const size_t nw = n->woff[layer + 1] - n->woff[layer];
    if (zero) LQ_CUDA(cudaMemsetAsync(gl, 0, nw * 4, c->stream));
    NetLayerArgs a = layer_args(n, layer, false, in, nullptr);
    a.gout_bf16 = a.out_bf16;  // the output gradient is stored like the layer's output
    double wb = 0.0, wf = 0.0;
    layer_work(a, batch, wb, wf);
    NetTimed tm;
    LQ_TRY(tm.begin(n, 3 * layer + 2, wb, wf));
    if (n->bf16) {
        // tensor cores: one CTA per SM, each over a stride of the batch x site tiles
        // (one input or one output channel: all nine hops per CTA; otherwise
        // half the SMs per group of five or four hops)
        const int sms = sm_count();
        if (sms <= 0) return fail(LQCD_ERR_CUDA, "net wgrad: no SM count");
        a.batch = batch;
        int cols = 32;
        while (cols < a.N2p) cols *= 2;
        a.tmem_cols = cols;
        const int total = (a.V + NTC_TS - 1) / NTC_TS * batch;
        if (a.cout == 1) {  // all hops in one pass, the transport on the output gradient
            int g1 = total < sms ? total : sms;
            if (n->max_ctas > 0 && g1 > n->max_ctas) g1 = n->max_ctas;
            NetLayerArgs o = a;
            o.tmem_cols = 128;  // NC1_K = 80 columns
            const size_t sm1 = (size_t)3 * NTC_TS * (128 + NC1_K) * 2 + 8 + 16;
            if (c->cfg.recon == 12) {
                LQ_CUDA(cudaFuncSetAttribute(net_wgrad_o1_kernel<12>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1));
                net_wgrad_o1_kernel<12><<<g1, NTC_THREADS, sm1, c->stream>>>(o, gout, gl);
            } else {
                LQ_CUDA(cudaFuncSetAttribute(net_wgrad_o1_kernel<18>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1));
                net_wgrad_o1_kernel<18><<<g1, NTC_THREADS, sm1, c->stream>>>(o, gout, gl);
            }
        } else if (a.cin > 1) {  // hop groups, pipelined (K2p <= 96: five hops fit 512 columns)
            const int per = (sms / 2 > 0 ? sms / 2 : 1);
            const int tiles = (a.V + WG_TS - 1) / WG_TS * batch;
            int gx = tiles < per ? tiles : per;
            if (n->max_ctas > 0 && gx > n->max_ctas) gx = n->max_ctas;
            NetLayerArgs w = a;
            w.tmem_cols = 512;
            const size_t smw = (size_t)6 * WG_TS * (a.K2p + WG_MN) * 2 + (size_t)2 * WG_TS * 19 * 4 + 2 * 8 + 16;
            dim3 gw(gx, 2);
            if (c->cfg.recon == 12) {
                LQ_CUDA(cudaFuncSetAttribute(net_wgrad_hg_kernel<12>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smw));
                net_wgrad_hg_kernel<12><<<gw, NTC_THREADS, smw, c->stream>>>(w, gout, gl);
            } else {
                LQ_CUDA(cudaFuncSetAttribute(net_wgrad_hg_kernel<18>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smw));
                net_wgrad_hg_kernel<18><<<gw, NTC_THREADS, smw, c->stream>>>(w, gout, gl);
            }
        } else {  // one input channel: all hops in one pass (M = 9 x 8 of 128)
            int g1 = total < sms ? total : sms;
            if (n->max_ctas > 0 && g1 > n->max_ctas) g1 = n->max_ctas;
            const size_t sm1 = (size_t)3 * NTC_TS * (128 + a.N2p) * 2 + 8 + 16;
            if (c->cfg.recon == 12) {
                LQ_CUDA(cudaFuncSetAttribute(net_wgrad_c1_kernel<12>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1));
                net_wgrad_c1_kernel<12><<<g1, NTC_THREADS, sm1, c->stream>>>(a, gout, gl);
            } else {
                LQ_CUDA(cudaFuncSetAttribute(net_wgrad_c1_kernel<18>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1));
                net_wgrad_c1_kernel<18><<<g1, NTC_THREADS, sm1, c->stream>>>(a, gout, gl);
            }
        }
        LQ_CUDA(cudaGetLastError());
        c->launches++;
        return tm.end();
    }
    const size_t sm = (size_t)NET_ROWS * (a.K2p + 4) * 4 + (size_t)NET_ROWS * 8 * a.cout * 4;
    const int ntiles = (a.V + NET_TS - 1) / NET_TS * batch;
    int gx = ntiles < 2 * 152 ? ntiles : 2 * 152;
    if (n->max_ctas > 0 && gx > n->max_ctas) gx = n->max_ctas;
    dim3 grid(gx, 9);
    if (c->cfg.recon == 12) {
        LQ_CUDA(cudaFuncSetAttribute(net_wgrad_kernel<12>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        net_wgrad_kernel<12><<<grid, NET_THREADS, sm, c->stream>>>(a, gout, batch, gl);
    } else {
        LQ_CUDA(cudaFuncSetAttribute(net_wgrad_kernel<18>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        net_wgrad_kernel<18><<<grid, NET_THREADS, sm, c->stream>>>(a, gout, batch, gl);
    }
    LQ_CUDA(cudaGetLastError());
    c->launches++;
    return tm.end();
}

lqcd_status NetTimed::begin(lqcd_net* net, int idx, double bytes, double flops)
{
    n = net;
    NetProfiler* pr = n->prof;
    if (!pr || !pr->on) return LQCD_OK;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    LQ_CUDA(cudaStreamIsCapturing(n->ctx->stream, &cap));
    if (cap != cudaStreamCaptureStatusNone) return LQCD_OK;
    rec.idx = idx;
    rec.bytes = bytes;
    rec.flops = flops;
    rec.a = pr->get();
    rec.b = pr->get();
    if (!rec.a || !rec.b) return fail(LQCD_ERR_CUDA, "net profiler: cudaEventCreate failed");
    LQ_CUDA(cudaEventRecord(rec.a, n->ctx->stream));
    timed = true;
    return LQCD_OK;
}

lqcd_status NetTimed::end()
{
    if (!timed) return LQCD_OK;
    LQ_CUDA(cudaEventRecord(rec.b, n->ctx->stream));
    n->prof->pending.push_back(rec);
    timed = false;
    return LQCD_OK;
}

}  // namespace

namespace lqcd {

// Forward of the whole net for `batch` Cin = 1 activations (act[0] filled).
lqcd_status net_forward_all(lqcd_net* n, int batch)
{
    for (int l = 0; l < n->nlayers; ++l)
        LQ_TRY(run_layer(n, layer_args(n, l, false, n->act[l], n->act[l + 1]), batch, 3 * l));
    return LQCD_OK;
}

// z = N(r) on internal FP32 full fields (FGCR preconditioner).
lqcd_status net_apply_internal(lqcd_net* n, void* z, const void* r, size_t rb)
{
    lqcd_ctx* c = n->ctx;
    dim3 grid((c->g.Vh + 127) / 128, 2);
    net_from_internal_kernel<<<grid, 128, 0, c->stream>>>(c->g, static_cast<const char*>(r), rb, n->act[0], 0, 1);
    LQ_CUDA(cudaGetLastError());
    LQ_TRY(net_forward_all(n, 1));
    net_to_internal_kernel<<<grid, 128, 0, c->stream>>>(c->g, static_cast<char*>(z), rb, n->act[n->nlayers], 1);
    LQ_CUDA(cudaGetLastError());
    c->launches += 2;
    return LQCD_OK;
}

}  // namespace lqcd

extern "C" {

lqcd_status lqcd_net_create(lqcd_ctx* c, int nlayers, const int* channels, int bf16, int max_batch, lqcd_net** out)
{
    try {
        if (!c || !channels || !out) return fail(LQCD_ERR_INVALID, "lqcd_net_create: null argument");
        if (nlayers < 1 || nlayers > 8) return fail(LQCD_ERR_INVALID, "lqcd_net_create: 1..8 layers");
        if (channels[0] != 1 || channels[nlayers] != 1)
            return fail(LQCD_ERR_INVALID, "lqcd_net_create: the first and last widths must be 1 (spinor in, spinor out)");
        for (int l = 0; l <= nlayers; ++l)
            if (channels[l] < 1 || channels[l] > NET_MAXC) return fail(LQCD_ERR_INVALID, "lqcd_net_create: widths in [1, 12]");
        if (max_batch < 1) return fail(LQCD_ERR_INVALID, "lqcd_net_create: max_batch >= 1");
        if (!c->holds(P32)) return fail(LQCD_ERR_STATE, "lqcd_net_create: the context must hold F32 links");
        if (c->cut()) return fail(LQCD_ERR_STATE, "lqcd_net_create: not on a sub-domain of a cut lattice");
        lqcd_net* n = new lqcd_net();
        memset(n, 0, sizeof(*n));
        n->ctx = c;
        n->nlayers = nlayers;
        for (int l = 0; l <= nlayers; ++l) n->ch[l] = channels[l];
        n->bf16 = bf16 ? 1 : 0;
        n->max_batch = max_batch;
        size_t w = 0;
        for (int l = 0; l < nlayers; ++l) {
            n->woff[l] = w;
            w += (size_t)9 * 4 * channels[l + 1] * 4 * channels[l] * 2;
        }
        n->woff[nlayers] = w;
        size_t off = 0;
        auto take = [&](size_t bytes) { size_t o = off; off += a256(bytes); return o; };
        size_t oW = take(w * 4), ogW = take(w * 4), om1 = take(w * 4), om2 = take(w * 4);
        size_t oB[8], oBh[8], oBA[8], oBhA[8];
        for (int l = 0; l < nlayers; ++l) {
            const int K2p = pad16(8 * channels[l]), N2p = pad16(8 * channels[l + 1]);
            const int K2pa = pad16(8 * channels[l + 1]), N2pa = pad16(8 * channels[l]);
            oB[l] = take((size_t)9 * K2p * N2p * 4);
            oBh[l] = take((size_t)9 * K2p * N2p * 2);
            oBA[l] = take((size_t)9 * K2pa * N2pa * 4);
            oBhA[l] = take((size_t)9 * K2pa * N2pa * 2);
        }
        size_t oS[8] = {0, 0, 0, 0, 0, 0, 0, 0}, oZ = 0;
        bool any_stack = false;
        for (int l = 0; l < nlayers; ++l) {
            n->stacked[l] = n->bf16 && channels[l + 1] == 1 && channels[l] > 1;
            if (n->stacked[l]) {
                oS[l] = take((size_t)80 * pad16(8 * channels[l]) * 2);
                any_stack = true;
            }
        }
        if (any_stack) oZ = take((size_t)max_batch * 2 * c->g.Vh * 9 * 48);
        size_t oA[9];
        int cmax = 1;
        for (int l = 0; l <= nlayers; ++l) {
            oA[l] = take((size_t)max_batch * act_floats(n, channels[l]) * 4);
            cmax = channels[l] > cmax ? channels[l] : cmax;
        }
        size_t oG0 = take((size_t)max_batch * act_floats(n, cmax) * 4);
        size_t oG1 = take((size_t)max_batch * act_floats(n, cmax) * 4);
        size_t oR = take((size_t)max_batch * 2 * sizeof(double));
        size_t oP = take((size_t)max_batch * 2 * NET_PARTIALS * sizeof(double));  // 2 sums per block
        size_t oT = take((size_t)max_batch * sizeof(unsigned));
        n->need = off;
        // stash offsets in the pointer fields until the workspace arrives
        n->W = reinterpret_cast<float*>(oW);
        n->gW = reinterpret_cast<float*>(ogW);
        n->m1 = reinterpret_cast<float*>(om1);
        n->m2 = reinterpret_cast<float*>(om2);
        for (int l = 0; l < nlayers; ++l) {
            n->Bf[l] = reinterpret_cast<float*>(oB[l]);
            n->Bh[l] = reinterpret_cast<uint16_t*>(oBh[l]);
            n->BfA[l] = reinterpret_cast<float*>(oBA[l]);
            n->BhA[l] = reinterpret_cast<uint16_t*>(oBhA[l]);
        }
        for (int l = 0; l <= nlayers; ++l) n->act[l] = reinterpret_cast<float*>(oA[l]);
        for (int l = 0; l < nlayers; ++l) n->BhS[l] = reinterpret_cast<uint16_t*>(oS[l]);
        n->zbuf = reinterpret_cast<float*>(oZ);
        n->gact[0] = reinterpret_cast<float*>(oG0);
        n->gact[1] = reinterpret_cast<float*>(oG1);
        n->red = reinterpret_cast<double*>(oR);
        n->partials = reinterpret_cast<double*>(oP);
        n->tickets = reinterpret_cast<unsigned*>(oT);
        *out = n;
        return LQCD_OK;
    } catch (...) {
        return fail(LQCD_ERR_NOMEM, "lqcd_net_create: host allocation failed");
    }
}

lqcd_status lqcd_net_destroy(lqcd_net* n)
{
    if (n) delete n->prof;
    delete n;
    return LQCD_OK;
}

lqcd_status lqcd_net_profile_enable(lqcd_net* n, int enable)
{
    try {
        if (!n) return fail(LQCD_ERR_INVALID, "lqcd_net_profile_enable: null network");
        if (!n->prof) n->prof = new NetProfiler();
        n->prof->on = enable != 0;
        return LQCD_OK;
    } catch (...) {
        return fail(LQCD_ERR_NOMEM, "lqcd_net_profile_enable: host allocation failed");
    }
}

lqcd_status lqcd_net_profile_read(lqcd_net* n, lqcd_profile_entry* out, int nentries)
{
    if (!n || !out) return fail(LQCD_ERR_INVALID, "lqcd_net_profile_read: null argument");
    if (nentries < 3 * n->nlayers) return fail(LQCD_ERR_INVALID, "lqcd_net_profile_read: needs 3 x nlayers entries");
    for (int i = 0; i < nentries; ++i) out[i] = lqcd_profile_entry{0, 0.0, 0.0, 0.0};
    if (!n->prof) return LQCD_OK;
    DeviceScope dev_scope;
    LQ_TRY(dev_scope.enter(n->ctx->device));
    LQ_CUDA(cudaStreamSynchronize(n->ctx->stream));
    for (auto& r : n->prof->pending) {
        float ms = 0.f;
        LQ_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
        out[r.idx].launches += 1;
        out[r.idx].ms += ms;
        out[r.idx].bytes += r.bytes;
        out[r.idx].flops += r.flops;
        n->prof->pool.push_back(r.a);
        n->prof->pool.push_back(r.b);
    }
    n->prof->pending.clear();
    return LQCD_OK;
}

lqcd_status lqcd_net_workspace_size(const lqcd_net* n, size_t* bytes)
{
    if (!n || !bytes) return fail(LQCD_ERR_INVALID, "lqcd_net_workspace_size: null argument");
    *bytes = n->need;
    return LQCD_OK;
}

lqcd_status lqcd_net_set_workspace(lqcd_net* n, void* ptr, size_t bytes)
{
    if (!n || !ptr) return fail(LQCD_ERR_INVALID, "lqcd_net_set_workspace: null argument");
    if (n->ws) return fail(LQCD_ERR_STATE, "lqcd_net_set_workspace: workspace already set");
    if (bytes < n->need) return fail(LQCD_ERR_NOMEM, "lqcd_net_set_workspace: too small");
    if (reinterpret_cast<uintptr_t>(ptr) & 255) return fail(LQCD_ERR_INVALID, "lqcd_net_set_workspace: 256-byte alignment");
    DeviceScope dev_scope;
    LQ_TRY(dev_scope.enter(n->ctx->device));
    char* base = static_cast<char*>(ptr);
    auto fix = [&](auto*& p) { p = reinterpret_cast<std::remove_reference_t<decltype(p)>>(base + reinterpret_cast<uintptr_t>(p)); };
    fix(n->W); fix(n->gW); fix(n->m1); fix(n->m2);
    for (int l = 0; l < n->nlayers; ++l) { fix(n->Bf[l]); fix(n->Bh[l]); fix(n->BfA[l]); fix(n->BhA[l]); }
    for (int l = 0; l <= n->nlayers; ++l) fix(n->act[l]);
    bool any_stack = false;
    for (int l = 0; l < n->nlayers; ++l)
        if (n->stacked[l]) {
            fix(n->BhS[l]);
            any_stack = true;
        }
    if (any_stack) fix(n->zbuf);
    fix(n->gact[0]); fix(n->gact[1]); fix(n->red); fix(n->partials); fix(n->tickets);
    n->ws = base;
    n->ws_bytes = bytes;
    lqcd_ctx* c = n->ctx;
    LQ_CUDA(cudaMemsetAsync(n->W, 0, n->nW() * 4, c->stream));
    LQ_CUDA(cudaMemsetAsync(n->tickets, 0, (size_t)n->max_batch * sizeof(unsigned), c->stream));
    LQ_CUDA(cudaMemsetAsync(n->m1, 0, n->nW() * 4, c->stream));
    LQ_CUDA(cudaMemsetAsync(n->m2, 0, n->nW() * 4, c->stream));
    n->adam_t = 0;
    return prep_weights(n);
}

// Transport with another context's links from now on (same lattice).
lqcd_status lqcd_net_bind(lqcd_net* n, lqcd_ctx* c)
{
    if (!n || !c) return fail(LQCD_ERR_INVALID, "lqcd_net_bind: null argument");
    const lqcd_ctx* o = n->ctx;
    for (int m = 0; m < 4; ++m)
        if (c->g.L[m] != o->g.L[m]) return fail(LQCD_ERR_INVALID, "lqcd_net_bind: lattice extents differ");
    if (c->g.tanti != o->g.tanti || c->cfg.recon != o->cfg.recon)
        return fail(LQCD_ERR_INVALID, "lqcd_net_bind: boundary condition or link storage differs");
    if (c->device != o->device) return fail(LQCD_ERR_INVALID, "lqcd_net_bind: contexts on different GPUs");
    if (!c->ws || !c->holds(P32) || !c->gauge_loaded)
        return fail(LQCD_ERR_STATE, "lqcd_net_bind: the context needs a workspace and loaded F32 links");
    n->ctx = c;
    return LQCD_OK;
}

// At most max_ctas CTAs per launch of the persistent layer kernel and per hop
// of the weight-gradient kernels (0: the default, one per SM).
lqcd_status lqcd_net_set_max_ctas(lqcd_net* n, int max_ctas)
{
    if (!n) return fail(LQCD_ERR_INVALID, "lqcd_net_set_max_ctas: null network");
    if (max_ctas < 0) return fail(LQCD_ERR_INVALID, "lqcd_net_set_max_ctas: max_ctas must be >= 0");
    n->max_ctas = max_ctas;
    return LQCD_OK;
}

lqcd_status lqcd_net_set_wait(lqcd_net* n, unsigned long long limit_ns, int expire_test)
{
    if (!n) return fail(LQCD_ERR_INVALID, "lqcd_net_set_wait: null network");
    n->wait_ns = limit_ns > 0 ? limit_ns : NTC_WAIT_NS;
    n->expire_test = expire_test ? 1 : 0;
    return LQCD_OK;
}

// Weights: complex FP32, layer after layer, each [9][4 cout][4 cin] (re, im).
lqcd_status lqcd_net_num_weights(const lqcd_net* n, size_t* count)
{
    if (!n || !count) return fail(LQCD_ERR_INVALID, "null argument");
    *count = n->nW() / 2;
    return LQCD_OK;
}

lqcd_status lqcd_net_set_weights(lqcd_net* n, const float* w)
{
    if (!n || !w || !n->ws) return fail(LQCD_ERR_INVALID, "lqcd_net_set_weights: null argument or no workspace");
    DeviceScope dev_scope;
    LQ_TRY(dev_scope.enter(n->ctx->device));
    LQ_CUDA(cudaMemcpyAsync(n->W, w, n->nW() * 4, cudaMemcpyDefault, n->ctx->stream));
    LQ_CUDA(cudaMemsetAsync(n->m1, 0, n->nW() * 4, n->ctx->stream));
    LQ_CUDA(cudaMemsetAsync(n->m2, 0, n->nW() * 4, n->ctx->stream));
    n->adam_t = 0;
    return prep_weights(n);
}

lqcd_status lqcd_net_get_weights(const lqcd_net* n, float* w, float* grad)
{
    if (!n || !n->ws) return fail(LQCD_ERR_INVALID, "lqcd_net_get_weights: no workspace");
    DeviceScope dev_scope;
    LQ_TRY(dev_scope.enter(n->ctx->device));
    if (w) LQ_CUDA(cudaMemcpyAsync(w, n->W, n->nW() * 4, cudaMemcpyDefault, n->ctx->stream));
    if (grad) LQ_CUDA(cudaMemcpyAsync(grad, n->gW, n->nW() * 4, cudaMemcpyDefault, n->ctx->stream));
    LQ_CUDA(cudaStreamSynchronize(n->ctx->stream));
    return LQCD_OK;
}

// One layer forward (adjoint = 0) or its adjoint (adjoint = 1: input
// gradient) on caller-provided device activations of `batch` items.
lqcd_status lqcd_net_layer_apply(lqcd_net* n, int layer, int adjoint, float* out, const float* in, int batch)
{
    if (!n || !n->ws || !out || !in) return fail(LQCD_ERR_INVALID, "lqcd_net_layer_apply: bad argument");
    if (layer < 0 || layer >= n->nlayers || batch < 1 || batch > n->max_batch)
        return fail(LQCD_ERR_INVALID, "lqcd_net_layer_apply: bad layer/batch");
    DeviceScope dev_scope;
    LQ_TRY(dev_scope.enter(n->ctx->device));
    const NetLayerArgs a = layer_args(n, layer, adjoint != 0, n->gact[0], n->gact[1]);
    LQ_TRY(convert_layout(n, in, n->gact[0], a.cin, batch, true));
    LQ_TRY(run_layer(n, a, batch, 3 * layer + (adjoint ? 1 : 0)));
    return convert_layout(n, n->gact[1], out, a.cout, batch, false);
}

// Weight gradient of one layer (accumulated into the net's gradient buffer
// after zeroing it when `zero`): G_W += sum over batch and sites.
lqcd_status lqcd_net_layer_wgrad(lqcd_net* n, int layer, const float* in, const float* gout, int batch, int zero)
{
    if (!n || !n->ws || !in || !gout) return fail(LQCD_ERR_INVALID, "lqcd_net_layer_wgrad: bad argument");
    if (layer < 0 || layer >= n->nlayers || batch < 1 || batch > n->max_batch)
        return fail(LQCD_ERR_INVALID, "lqcd_net_layer_wgrad: bad layer/batch");
    DeviceScope dev_scope;
    LQ_TRY(dev_scope.enter(n->ctx->device));
    LQ_TRY(convert_layout(n, in, n->gact[0], n->ch[layer], batch, true));
    LQ_TRY(convert_layout(n, gout, n->gact[1], n->ch[layer + 1], batch, true));
    return run_wgrad(n, layer, n->gact[0], n->gact[1], batch, zero);
}

// Whole-net forward on canonical FP32 complex spinors (batch items):
// out, in: [batch][site][spin][colour] complex (device).
lqcd_status lqcd_net_forward(lqcd_net* n, float* out, const float* in, int batch)
{
    NvtxRange nvtx_range("lqcd_net_forward");
    if (!n || !n->ws || !out || !in) return fail(LQCD_ERR_INVALID, "lqcd_net_forward: bad argument");
    if (batch < 1 || batch > n->max_batch) return fail(LQCD_ERR_INVALID, "lqcd_net_forward: batch out of range");
    DeviceScope dev_scope;
    LQ_TRY(dev_scope.enter(n->ctx->device));
    LQ_TRY(convert_layout(n, in, n->act[0], 1, batch, true));
    LQ_TRY(net_forward_all(n, batch));
    return convert_layout(n, n->act[n->nlayers], out, 1, batch, false);
}

// One training step on `batch` pairs (r, e) of canonical FP32 complex
// spinors: forward, loss L = mean |N(r) - e|^2 / |e|^2, backward through
// every layer, Adam (lr, beta1, beta2, eps).  *loss receives L (FP64) and
// the call synchronises the stream to read it.
lqcd_status lqcd_net_train_step(lqcd_net* n, const float* r, const float* e, int batch, double lr, double beta1,
                                double beta2, double eps, double* loss)
{
    NvtxRange nvtx_range("lqcd_net_train_step");
    if (!n || !n->ws || !r || !e) return fail(LQCD_ERR_INVALID, "lqcd_net_train_step: bad argument");
    if (batch < 1 || batch > n->max_batch) return fail(LQCD_ERR_INVALID, "lqcd_net_train_step: batch out of range");
    DeviceScope dev_scope;
    LQ_TRY(dev_scope.enter(n->ctx->device));
    lqcd_ctx* c = n->ctx;
    const size_t n_per = act_floats(n, 1);
    LQ_TRY(convert_layout(n, r, n->act[0], 1, batch, true));
    LQ_TRY(convert_layout(n, e, n->gact[1], 1, batch, true));  // planar target; gact[1] is free until the backward
    LQ_TRY(net_forward_all(n, batch));
    const float* ep = n->gact[1];
    // loss and its gradient
    const int nb = 256;
    dim3 g1(NET_PARTIALS, batch);
    net_loss_reduce_kernel<<<g1, nb, 0, c->stream>>>(n->act[n->nlayers], ep, n_per, n->partials, 2 * NET_PARTIALS,
                                                     n->tickets, n->red);
    LQ_CUDA(cudaGetLastError());
    net_loss_grad_kernel<<<g1, nb, 0, c->stream>>>(n->act[n->nlayers], ep, n_per, n->red, batch, n->gact[0]);
    LQ_CUDA(cudaGetLastError());
    c->launches += 2;
    // backward
    int cur = 0;
    for (int l = n->nlayers - 1; l >= 0; --l) {
        LQ_TRY(run_wgrad(n, l, n->act[l], n->gact[cur], batch, 1));
        if (l > 0) {
            LQ_TRY(run_layer(n, layer_args(n, l, true, n->gact[cur], n->gact[1 - cur]), batch, 3 * l + 1));
            cur = 1 - cur;
        }
    }
    // Adam
    n->adam_t++;
    const float c1 = (float)(1.0 - pow(beta1, (double)n->adam_t));
    const float c2 = (float)(1.0 - pow(beta2, (double)n->adam_t));
    net_adam_kernel<<<256, 256, 0, c->stream>>>(n->W, n->m1, n->m2, n->gW, (int)n->nW(), (float)lr, (float)beta1,
                                                (float)beta2, (float)eps, c1, c2);
    LQ_CUDA(cudaGetLastError());
    c->launches++;
    LQ_TRY(prep_weights(n));
    if (loss) {
        std::vector<double> h(2 * batch);
        LQ_CUDA(cudaMemcpyAsync(h.data(), n->red, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        LQ_CUDA(cudaStreamSynchronize(c->stream));
        double L = 0.0;
        for (int b = 0; b < batch; ++b) L += h[2 * b] / h[2 * b + 1];
        *loss = L / batch;
    }
    return LQCD_OK;
}

}  // extern "C"
