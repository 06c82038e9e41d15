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
// Activations: FP32 complex, [batch][site][channel][spin][colour], canonical
// site order.  One CTA handles a tile of 64 consecutive sites: for each hop
// it gathers the transported inputs of its 192 (site, colour) rows into
// shared memory, then accumulates the real-ified product
//   OUT[row][n2] += X[row][k2] * B_h[k2][n2]
// (k2 = 2*(ci*4+r) + {re, im}, n2 = 2*(co*4+s) + {re, im}) on the tensor
// cores (BF16 operands, FP32 accumulation, mma.sync m16n8k16) or, for the
// FP32 path, with FMAs.
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "internal.h"

namespace lqcd {

enum { NET_TS = 64, NET_ROWS = 3 * NET_TS, NET_THREADS = 256, NET_MAXC = 12, NET_PARTIALS = 64 };

struct NetLayerArgs {
    int L[4];
    int V;
    int stride;        // of the FP32 gauge copy
    int tanti;
    const void* gauge; // FP32 gauge copy (internal SoA)
    int cin, cout;
    int K2, N2;        // real-ified inner / outer sizes: 8 cin, 8 cout
    int K2p, N2p;      // padded to 16 / 8
    const float* in;   // [batch][V][cin][4][3] complex
    float* out;        // [batch][V][cout][4][3] complex
    const float* Bf;   // FP32 real-ified weights [9][K2][N2]
    const uint16_t* Bh;// BF16 real-ified weights [9][N2p][K2p] (n-major)
};

__host__ __device__ inline int adj_hop(int h) { return h == 0 ? 0 : (h % 2 == 1 ? h + 1 : h - 1); }

// Link for hop h at canonical site x: V (3x3 complex, 18 floats) and the
// fermion sign; returns the neighbour site.
template <int RECON>
__device__ __forceinline__ int hop_link(const NetLayerArgs& a, int x, int h, float u[18], float& sign)
{
    int c[4];
    int s = x;
    c[0] = s % a.L[0]; s /= a.L[0];
    c[1] = s % a.L[1]; s /= a.L[1];
    c[2] = s % a.L[2];
    c[3] = s / a.L[2];
    sign = 1.f;
    if (h == 0) return x;
    const int mu = (h - 1) / 2;
    const bool fwd = ((h - 1) % 2) == 0;
    int n[4] = {c[0], c[1], c[2], c[3]};
    n[mu] = fwd ? (c[mu] + 1 == a.L[mu] ? 0 : c[mu] + 1) : (c[mu] == 0 ? a.L[mu] - 1 : c[mu] - 1);
    const int y = ((n[3] * a.L[2] + n[2]) * a.L[1] + n[1]) * a.L[0] + n[0];
    if (a.tanti && mu == 3 && ((fwd && c[3] == a.L[3] - 1) || (!fwd && c[3] == 0))) sign = -1.f;
    // forward: U_mu(x); backward: U_mu(y)^dag
    const int site = fwd ? x : y;
    const int* cc = fwd ? c : n;
    const int par = (cc[0] + cc[1] + cc[2] + cc[3]) & 1;
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

// Gather the transported inputs of hop h for the tile into shared memory:
// X[row = site*3 + a][k2]; rows past V are zero.  The tile's links and
// neighbours for the hop are staged once; then consecutive threads take
// consecutive (channel, spin) pieces of the same neighbour, whose
// activations are contiguous, so each warp reads one stretch of memory.
template <int RECON, bool TC>
__device__ __forceinline__ void gather_hop(const NetLayerArgs& a, const float* in_b, int tile0, int h, void* Xs,
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
            const float2* src = reinterpret_cast<const float2*>(in_b) + ((size_t)y * nk + k) * 3;
            const float2 p0 = src[0], p1 = src[1], p2 = src[2];
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
            if (TC) {
                uint32_t v = (uint32_t)f2bf(o[2 * r]) | ((uint32_t)f2bf(o[2 * r + 1]) << 16);
                reinterpret_cast<uint32_t*>(static_cast<uint16_t*>(Xs) + (size_t)row * xstride)[k] = v;
            } else {
                reinterpret_cast<float2*>(static_cast<float*>(Xs) + (size_t)row * xstride)[k] = make_float2(o[2 * r], o[2 * r + 1]);
            }
        }
    }
}

__device__ __forceinline__ void mma_bf16_16816(float d[4], const uint32_t a[4], const uint32_t b[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Forward of one layer for every batch item (blockIdx.y) and tile (blockIdx.x).
template <int RECON, bool TC>
__global__ void __launch_bounds__(NET_THREADS) net_layer_kernel(const NetLayerArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int tile0 = blockIdx.x * NET_TS;
    const int b = blockIdx.y;
    const float* in_b = a.in + (size_t)b * a.V * a.cin * 24;
    float* out_b = a.out + (size_t)b * a.V * a.cout * 24;
    const int tid = threadIdx.x;
    if (TC) {
        // shared: X [192][K2p + 8] bf16, B [N2p][K2p + 8] bf16
        const int xs = a.K2p + 8;
        uint16_t* Xs = reinterpret_cast<uint16_t*>(smem);
        uint16_t* Bs = Xs + NET_ROWS * xs;
        const int warp = tid >> 5, lane = tid & 31, gid = lane >> 2, tig = lane & 3;
        const int NT = a.N2p / 8;                 // n tiles
        const int mt0 = (warp % 4) * 3;           // 3 of the 12 m tiles
        const int ntw = (NT + 1) / 2;             // n tiles per warp half
        const int nt0 = (warp / 4) * ntw;
        float acc[3][6][4];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 6; ++j)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
        for (int h = 0; h < 9; ++h) {
            gather_hop<RECON, true>(a, in_b, tile0, h, Xs, xs);
            const uint16_t* Bg = a.Bh + (size_t)h * a.N2p * a.K2p;
            for (int e = tid; e < a.N2p * a.K2p / 2; e += NET_THREADS) {
                const int n = e / (a.K2p / 2), kk = e % (a.K2p / 2);
                reinterpret_cast<uint32_t*>(Bs + (size_t)n * xs)[kk] = reinterpret_cast<const uint32_t*>(Bg)[e];
            }
            __syncthreads();
            for (int k0 = 0; k0 < a.K2p; k0 += 16) {
                uint32_t af[3][4];
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const int r0 = (mt0 + i) * 16 + gid;
                    af[i][0] = *reinterpret_cast<const uint32_t*>(Xs + (size_t)r0 * xs + k0 + tig * 2);
                    af[i][1] = *reinterpret_cast<const uint32_t*>(Xs + (size_t)(r0 + 8) * xs + k0 + tig * 2);
                    af[i][2] = *reinterpret_cast<const uint32_t*>(Xs + (size_t)r0 * xs + k0 + 8 + tig * 2);
                    af[i][3] = *reinterpret_cast<const uint32_t*>(Xs + (size_t)(r0 + 8) * xs + k0 + 8 + tig * 2);
                }
#pragma unroll
                for (int j = 0; j < 6; ++j) {
                    const int nt = nt0 + j;
                    if (nt >= NT || j >= ntw) break;
                    uint32_t bf[2];
                    const int n = nt * 8 + gid;
                    bf[0] = *reinterpret_cast<const uint32_t*>(Bs + (size_t)n * xs + k0 + tig * 2);
                    bf[1] = *reinterpret_cast<const uint32_t*>(Bs + (size_t)n * xs + k0 + 8 + tig * 2);
#pragma unroll
                    for (int i = 0; i < 3; ++i) mma_bf16_16816(acc[i][j], af[i], bf);
                }
            }
            __syncthreads();
        }
        // epilogue: acc -> out[site][co][s][a] (complex)
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 6; ++j) {
                const int nt = nt0 + j;
                if (nt >= NT || j >= ntw) break;
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    const int row = (mt0 + i) * 16 + gid + 8 * hh;
                    const int n2 = nt * 8 + tig * 2;  // even: (re, im) of output n2/2
                    const int site = tile0 + row / 3, col = row % 3, n = n2 / 2;
                    if (site < a.V && n2 < a.N2)
                        reinterpret_cast<float2*>(out_b)[((size_t)site * 4 * a.cout + n) * 3 + col] =
                            make_float2(acc[i][j][2 * hh], acc[i][j][2 * hh + 1]);
                }
            }
    } else {
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
            gather_hop<RECON, false>(a, in_b, tile0, h, Xs, xs);
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
                if (n2 < a.N2)
                    reinterpret_cast<float2*>(out_b)[((size_t)site * 4 * a.cout + n2 / 2) * 3 + col] =
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
        gather_hop<RECON, false>(a, a.in + (size_t)b * a.V * a.cin * 24, tile0, h, Xs, xs);
        const float* gb = gout + (size_t)b * a.V * a.cout * 24;
        for (int e = threadIdx.x; e < NET_ROWS * nn; e += NET_THREADS) {
            const int row = e / nn, n = e % nn;
            const int site = tile0 + row / 3, col = row % 3;
            float2 v = make_float2(0.f, 0.f);
            if (site < a.V) v = reinterpret_cast<const float2*>(gb)[((size_t)site * nn + n) * 3 + col];
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
// Bh[h][n2][k2] (zero padded).  With W' = adjoint-hop conjugate transpose
// when `adjoint` (the layer's input gradient).
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
        Bh[e] = f2bf(v);
    }
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
    float4* dst = reinterpret_cast<float4*>(act + ((size_t)b * V + full_index(g, c)) * 24);
#pragma unroll
    for (int k = 0; k < 6; ++k) dst[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
}

__global__ void net_to_internal_kernel(Geom g, char* out, size_t out_rb, const float* act, int nb)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int par = blockIdx.y % 2, b = blockIdx.y / 2;
    if (i >= g.Vh || b >= nb) return;
    int c[4];
    cb_coords(g, i, par, c);
    const size_t V = (size_t)2 * g.Vh;
    const float4* src = reinterpret_cast<const float4*>(act + ((size_t)b * V + full_index(g, c)) * 24);
    float v[24];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        float4 q = src[k];
        v[4 * k] = q.x; v[4 * k + 1] = q.y; v[4 * k + 2] = q.z; v[4 * k + 3] = q.w;
    }
    SpinorIO<P32>::store(out + b * out_rb + par * spinor_field_bytes(P32, g.stride), g.stride, i, v);
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

struct lqcd_net {
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
    float* act[9];         // activations per layer boundary: [max_batch][V][ch][4][3] complex
    float* gact[2];        // gradient ping-pong buffers (max channels)
    double* red;           // loss reductions [max_batch][2]
    double* partials;      // loss reduction partials [max_batch][NET_PARTIALS][2]
    unsigned* tickets;     // [max_batch]
    size_t woff[9];        // float offsets of layer weights in W (layer nlayers = total)
    size_t boff[8], bhoff[8];
    long adam_t;
    size_t nW() const { return woff[nlayers]; }
};

namespace {

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }
int pad16(int x) { return (x + 15) / 16 * 16; }
int pad8(int x) { return (x + 7) / 8 * 8; }

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
    a.N2p = pad8(a.N2);
    a.in = in;
    a.out = out;
    a.Bf = adjoint ? n->BfA[l] : n->Bf[l];
    a.Bh = adjoint ? n->BhA[l] : n->Bh[l];
    return a;
}

size_t layer_smem(const NetLayerArgs& a, bool tc)
{
    if (tc) return (size_t)(NET_ROWS + a.N2p) * (a.K2p + 8) * 2;
    return (size_t)NET_ROWS * (a.K2p + 4) * 4 + (size_t)a.K2 * (a.N2p + 4) * 4;
}

lqcd_status run_layer(lqcd_net* n, const NetLayerArgs& a, int batch)
{
    lqcd_ctx* c = n->ctx;
    const bool tc = n->bf16 != 0;
    const size_t sm = layer_smem(a, tc);
    dim3 grid((a.V + NET_TS - 1) / NET_TS, batch);
#define LQ_NL(RC, TCV)                                                                                   \
    do {                                                                                                 \
        LQ_CUDA(cudaFuncSetAttribute(net_layer_kernel<RC, TCV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)); \
        net_layer_kernel<RC, TCV><<<grid, NET_THREADS, sm, c->stream>>>(a);                            \
    } while (0)
    if (c->cfg.recon == 12) { if (tc) LQ_NL(12, true); else LQ_NL(12, false); }
    else { if (tc) LQ_NL(18, true); else LQ_NL(18, false); }
#undef LQ_NL
    LQ_CUDA(cudaGetLastError());
    c->launches++;
    return LQCD_OK;
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
    return LQCD_OK;
}

size_t act_floats(const lqcd_net* n, int chn) { return (size_t)2 * n->ctx->g.Vh * chn * 24; }

}  // namespace

namespace lqcd {

// Forward of the whole net for `batch` Cin = 1 activations (act[0] filled).
lqcd_status net_forward_all(lqcd_net* n, int batch)
{
    for (int l = 0; l < n->nlayers; ++l)
        LQ_TRY(run_layer(n, layer_args(n, l, false, n->act[l], n->act[l + 1]), batch));
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
            const int K2p = pad16(8 * channels[l]), N2p = pad8(8 * channels[l + 1]);
            const int K2pa = pad16(8 * channels[l + 1]), N2pa = pad8(8 * channels[l]);
            oB[l] = take((size_t)9 * K2p * N2p * 4);
            oBh[l] = take((size_t)9 * K2p * N2p * 2);
            oBA[l] = take((size_t)9 * K2pa * N2pa * 4);
            oBhA[l] = take((size_t)9 * K2pa * N2pa * 2);
        }
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
    delete n;
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
    char* base = static_cast<char*>(ptr);
    auto fix = [&](auto*& p) { p = reinterpret_cast<std::remove_reference_t<decltype(p)>>(base + reinterpret_cast<uintptr_t>(p)); };
    fix(n->W); fix(n->gW); fix(n->m1); fix(n->m2);
    for (int l = 0; l < n->nlayers; ++l) { fix(n->Bf[l]); fix(n->Bh[l]); fix(n->BfA[l]); fix(n->BhA[l]); }
    for (int l = 0; l <= n->nlayers; ++l) fix(n->act[l]);
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
    LQ_CUDA(cudaMemcpyAsync(n->W, w, n->nW() * 4, cudaMemcpyDefault, n->ctx->stream));
    LQ_CUDA(cudaMemsetAsync(n->m1, 0, n->nW() * 4, n->ctx->stream));
    LQ_CUDA(cudaMemsetAsync(n->m2, 0, n->nW() * 4, n->ctx->stream));
    n->adam_t = 0;
    return prep_weights(n);
}

lqcd_status lqcd_net_get_weights(const lqcd_net* n, float* w, float* grad)
{
    if (!n || !n->ws) return fail(LQCD_ERR_INVALID, "lqcd_net_get_weights: no workspace");
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
    if (layer < 0 || layer >= n->nlayers || batch < 1) return fail(LQCD_ERR_INVALID, "lqcd_net_layer_apply: bad layer/batch");
    return run_layer(n, layer_args(n, layer, adjoint != 0, in, out), batch);
}

// Weight gradient of one layer (accumulated into the net's gradient buffer
// after zeroing it when `zero`): G_W += sum over batch and sites.
lqcd_status lqcd_net_layer_wgrad(lqcd_net* n, int layer, const float* in, const float* gout, int batch, int zero)
{
    if (!n || !n->ws || !in || !gout) return fail(LQCD_ERR_INVALID, "lqcd_net_layer_wgrad: bad argument");
    if (layer < 0 || layer >= n->nlayers || batch < 1) return fail(LQCD_ERR_INVALID, "lqcd_net_layer_wgrad: bad layer");
    lqcd_ctx* c = n->ctx;
    float* gl = n->gW + n->woff[layer];
    const size_t nw = n->woff[layer + 1] - n->woff[layer];
    if (zero) LQ_CUDA(cudaMemsetAsync(gl, 0, nw * 4, c->stream));
    NetLayerArgs a = layer_args(n, layer, false, in, nullptr);
    const size_t sm = (size_t)NET_ROWS * (a.K2p + 4) * 4 + (size_t)NET_ROWS * 8 * a.cout * 4;
    const int ntiles = (a.V + NET_TS - 1) / NET_TS * batch;
    dim3 grid(ntiles < 2 * 152 ? ntiles : 2 * 152, 9);
    if (c->cfg.recon == 12) {
        LQ_CUDA(cudaFuncSetAttribute(net_wgrad_kernel<12>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        net_wgrad_kernel<12><<<grid, NET_THREADS, sm, c->stream>>>(a, gout, batch, gl);
    } else {
        LQ_CUDA(cudaFuncSetAttribute(net_wgrad_kernel<18>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        net_wgrad_kernel<18><<<grid, NET_THREADS, sm, c->stream>>>(a, gout, batch, gl);
    }
    LQ_CUDA(cudaGetLastError());
    c->launches++;
    return LQCD_OK;
}

// Whole-net forward on canonical FP32 complex spinors (batch items):
// out, in: [batch][site][spin][colour] complex (device).
lqcd_status lqcd_net_forward(lqcd_net* n, float* out, const float* in, int batch)
{
    if (!n || !n->ws || !out || !in) return fail(LQCD_ERR_INVALID, "lqcd_net_forward: bad argument");
    if (batch < 1 || batch > n->max_batch) return fail(LQCD_ERR_INVALID, "lqcd_net_forward: batch out of range");
    lqcd_ctx* c = n->ctx;
    const size_t bytes = (size_t)batch * act_floats(n, 1) * 4;
    LQ_CUDA(cudaMemcpyAsync(n->act[0], in, bytes, cudaMemcpyDeviceToDevice, c->stream));
    LQ_TRY(net_forward_all(n, batch));
    LQ_CUDA(cudaMemcpyAsync(out, n->act[n->nlayers], bytes, cudaMemcpyDeviceToDevice, c->stream));
    return LQCD_OK;
}

// One training step on `batch` pairs (r, e) of canonical FP32 complex
// spinors: forward, loss L = mean |N(r) - e|^2 / |e|^2, backward through
// every layer, Adam (lr, beta1, beta2, eps).  *loss receives L (FP64) and
// the call synchronises the stream to read it.
lqcd_status lqcd_net_train_step(lqcd_net* n, const float* r, const float* e, int batch, double lr, double beta1,
                                double beta2, double eps, double* loss)
{
    if (!n || !n->ws || !r || !e) return fail(LQCD_ERR_INVALID, "lqcd_net_train_step: bad argument");
    if (batch < 1 || batch > n->max_batch) return fail(LQCD_ERR_INVALID, "lqcd_net_train_step: batch out of range");
    lqcd_ctx* c = n->ctx;
    const size_t n_per = act_floats(n, 1);
    LQ_CUDA(cudaMemcpyAsync(n->act[0], r, (size_t)batch * n_per * 4, cudaMemcpyDeviceToDevice, c->stream));
    LQ_TRY(net_forward_all(n, batch));
    // loss and its gradient
    const int nb = 256;
    dim3 g1(NET_PARTIALS, batch);
    net_loss_reduce_kernel<<<g1, nb, 0, c->stream>>>(n->act[n->nlayers], e, n_per, n->partials, 2 * NET_PARTIALS,
                                                     n->tickets, n->red);
    LQ_CUDA(cudaGetLastError());
    net_loss_grad_kernel<<<g1, nb, 0, c->stream>>>(n->act[n->nlayers], e, n_per, n->red, batch, n->gact[0]);
    LQ_CUDA(cudaGetLastError());
    c->launches += 2;
    // backward
    int cur = 0;
    for (int l = n->nlayers - 1; l >= 0; --l) {
        LQ_TRY(lqcd_net_layer_wgrad(n, l, n->act[l], n->gact[cur], batch, 1));
        if (l > 0) {
            LQ_TRY(run_layer(n, layer_args(n, l, true, n->gact[cur], n->gact[1 - cur]), batch));
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
