// Wilson hopping term ("dslash") on one parity, with fused epilogues.
//
//   out_p(x) = epi( sum_mu (1 - g_mu) U_mu(x) in(x+mu) + (1 + g_mu) U_mu(x-mu)^dag in(x-mu) )
//
// (the matrix-vector product the paper identifies as the dominant cost of
// every Krylov solver, Sec. 3 and Sec. 5; even-odd splitting makes each
// application touch one parity of output and the other of input, Sec. 5).
//
// One thread per output site (launches that reduce stride over the sites
// with one wave of blocks).  Every neighbour spinor is spin-projected to
// a half spinor (two colour vectors) before the SU(3) multiply and
// reconstructed afterwards, which is the 1320-flop form of the operator.
// The adjoint (DAG) swaps the projectors, since H^dag = g5 H g5.  The t
// boundary sign multiplies the half spinor of hops that cross t = Lt-1 <-> 0.
//
// Epilogues, in the compute precision:
//   EPI_NONE     out = a * D
//   EPI_CLOVINV  out = a * Cl D                  (Cl = A^{-1} of the output parity)
//   EPI_XPAY     out = Cl y + a * D               (Cl = A, or 1 without clover)
//   EPI_CG       s = Cl y + a * D; x += alpha p; r -= alpha s  (s never stored)
// and optionally (RED) the grid sum of |out|^2 (|r|^2 for EPI_CG) in FP64.
#pragma once
#include "core.cuh"

namespace lqcd {

enum Epi { EPI_NONE = 0, EPI_CLOVINV = 1, EPI_XPAY = 2, EPI_CG = 3 };

struct DslashArgs {
    Geom g;
    int par;                 // output parity
    void* out;               // output fields (EPI_CG: unused)
    size_t out_rb;           // bytes between right-hand sides
    const void* in;          // input fields, parity 1 - par
    size_t in_rb;
    const void* gauge;       // gauge copy of this precision / recon
    const void* clov;        // clover field of the output parity, or nullptr (= 1)
    const void* y;           // EPI_XPAY / EPI_CG: field of the output parity
    size_t y_rb;
    double a;                // coefficient of the hopping term
    // reductions (RED): per rhs r, partials + r * part_rs, tickets[r], red + r * red_rs
    double* partials;
    size_t part_rs;
    unsigned* tickets;
    double* red;
    size_t red_rs;
    // EPI_CG: x, r in the accumulation precision; p in P; scalars per rhs
    void* x;
    void* r;
    size_t acc_rb;
    const void* p;
    size_t p_rb;
    const double* scal;      // per rhs: scal + r * scal_rs
    size_t scal_rs;
    int s_num, s_num2;       // alpha = (scal[s_num] + scal[s_num2]) / (scal[s_den] + scal[s_den2])
    int s_den, s_den2;
    const int* skip;         // per rhs: nonzero = converged, do nothing (may be nullptr)
    int sites_per_thread;    // reducing launches: grid of Vh / (block * this); 0 = one wave of blocks
    int nrhs;                // right-hand sides of the launch (set by the launcher)
};

// ---- spin projection (1 + S g_mu), S = -1 or +1, onto two colour vectors
template <int MU, int S, class R>
__device__ __forceinline__ void project(const R v[24], R h[12])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const R p0r = v[2 * c], p0i = v[2 * c + 1];
        const R p1r = v[2 * (3 + c)], p1i = v[2 * (3 + c) + 1];
        const R p2r = v[2 * (6 + c)], p2i = v[2 * (6 + c) + 1];
        const R p3r = v[2 * (9 + c)], p3i = v[2 * (9 + c) + 1];
        R h0r, h0i, h1r, h1i;
        if (MU == 0) {        // h0 = p0 + S i p3, h1 = p1 + S i p2
            h0r = p0r - S * p3i; h0i = p0i + S * p3r;
            h1r = p1r - S * p2i; h1i = p1i + S * p2r;
        } else if (MU == 1) { // h0 = p0 - S p3, h1 = p1 + S p2
            h0r = p0r - S * p3r; h0i = p0i - S * p3i;
            h1r = p1r + S * p2r; h1i = p1i + S * p2i;
        } else if (MU == 2) { // h0 = p0 + S i p2, h1 = p1 - S i p3
            h0r = p0r - S * p2i; h0i = p0i + S * p2r;
            h1r = p1r + S * p3i; h1i = p1i - S * p3r;
        } else {              // h0 = p0 + S p2, h1 = p1 + S p3
            h0r = p0r + S * p2r; h0i = p0i + S * p2i;
            h1r = p1r + S * p3r; h1i = p1i + S * p3i;
        }
        h[2 * c] = h0r; h[2 * c + 1] = h0i;
        h[2 * (3 + c)] = h1r; h[2 * (3 + c) + 1] = h1i;
    }
}

// ---- reconstruct the lower spins from the two rotated colour vectors
template <int MU, int S, class R>
__device__ __forceinline__ void accumulate(R acc[24], const R w[12])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const R w0r = w[2 * c], w0i = w[2 * c + 1];
        const R w1r = w[2 * (3 + c)], w1i = w[2 * (3 + c) + 1];
        acc[2 * c] += w0r; acc[2 * c + 1] += w0i;
        acc[2 * (3 + c)] += w1r; acc[2 * (3 + c) + 1] += w1i;
        R r2r, r2i, r3r, r3i;
        if (MU == 0) {        // r2 = -S i w1, r3 = -S i w0
            r2r = S * w1i; r2i = -S * w1r;
            r3r = S * w0i; r3i = -S * w0r;
        } else if (MU == 1) { // r2 = S w1, r3 = -S w0
            r2r = S * w1r; r2i = S * w1i;
            r3r = -S * w0r; r3i = -S * w0i;
        } else if (MU == 2) { // r2 = -S i w0, r3 = S i w1
            r2r = S * w0i; r2i = -S * w0r;
            r3r = -S * w1i; r3i = S * w1r;
        } else {              // r2 = S w0, r3 = S w1
            r2r = S * w0r; r2i = S * w0i;
            r3r = S * w1r; r3i = S * w1i;
        }
        acc[2 * (6 + c)] += r2r; acc[2 * (6 + c) + 1] += r2i;
        acc[2 * (9 + c)] += r3r; acc[2 * (9 + c) + 1] += r3i;
    }
}

// w = U h (ADJ = false) or U^dag h (ADJ = true) for both colour vectors of h.
// Each real product is its own multiply-add into the running sum (one
// fused instruction each; a - b*c contracts with the sign folded in).
// PACK (FP32 only): the same products as packed two-lane instructions.
template <bool ADJ, bool PACK = false, class R>
__device__ __forceinline__ void su3_mul_half(const R u[18], const R h[12], R w[12])
{
    if constexpr (PACK && sizeof(R) == 4) {
        // FP32: the two colour vectors share every link entry, so lane s of
        // a packed pair carries colour vector s through the same sequence of
        // products (per lane the same roundings as the scalar form below)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float2 re, im;
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const int k = ADJ ? 2 * (3 * b + a) : 2 * (3 * a + b);
                const float2 ur = make_float2(u[k], u[k]);
                const float2 ui = make_float2(u[k + 1], u[k + 1]);
                const float2 nui = make_float2(-u[k + 1], -u[k + 1]);
                const float2 hr = make_float2(h[2 * b], h[2 * (3 + b)]);
                const float2 hi = make_float2(h[2 * b + 1], h[2 * (3 + b) + 1]);
                if (b == 0) {
                    re = __fmul2_rn(ur, hr);
                    im = __fmul2_rn(ur, hi);
                } else {
                    re = __ffma2_rn(ur, hr, re);
                    im = __ffma2_rn(ur, hi, im);
                }
                if (ADJ) {
                    re = __ffma2_rn(ui, hi, re);
                    im = __ffma2_rn(nui, hr, im);
                } else {
                    re = __ffma2_rn(nui, hi, re);
                    im = __ffma2_rn(ui, hr, im);
                }
            }
            w[2 * a] = re.x;
            w[2 * a + 1] = im.x;
            w[2 * (3 + a)] = re.y;
            w[2 * (3 + a) + 1] = im.y;
        }
        return;
    }
#pragma unroll
    for (int s = 0; s < 2; ++s) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            R re, im;
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const int k = ADJ ? 2 * (3 * b + a) : 2 * (3 * a + b);
                const R ur = u[k], ui = u[k + 1];
                const R hr = h[2 * (3 * s + b)], hi = h[2 * (3 * s + b) + 1];
                if (b == 0) {
                    re = ur * hr;
                    im = ur * hi;
                } else {
                    re += ur * hr;
                    im += ur * hi;
                }
                if (ADJ) {  // conj(u): (ur - i ui)(hr + i hi)
                    re += ui * hi;
                    im -= ui * hr;
                } else {
                    re -= ui * hi;
                    im += ui * hr;
                }
            }
            w[2 * (3 * s + a)] = re;
            w[2 * (3 * s + a) + 1] = im;
        }
    }
}

// One hop of the sum for the neighbour spinor v: forward (BWD false)
// (1 - g_mu) U_mu(x) v, backward (1 + g_mu) U_mu(x - mu)^dag v (projectors
// swapped by DAG); the link is U_mu at checkerboard index lidx of parity
// lpar; flip: the hop crosses the antiperiodic t boundary.
template <int PG, int RECON, int MU, bool DAG, bool BWD, bool PACK, class R>
__device__ __forceinline__ void hop_term(const DslashArgs& A, const R v[24], bool flip, int lpar, int lidx, R acc[24])
{
    constexpr int S = (BWD != DAG) ? +1 : -1;
    R h[12], u[18], w[12];
    project<MU, S>(v, h);
    if (flip) {
#pragma unroll
        for (int k = 0; k < 12; ++k) h[k] = -h[k];
    }
    GaugeIO<PG, RECON>::load(A.gauge, A.g.stride, lpar, MU, lidx, u);
    su3_mul_half<BWD, PACK>(u, h, w);
    accumulate<MU, S>(acc, w);
}

// PG: storage of links and clover; PS: storage of spinor fields; the
// arithmetic is in RealT<PS> (FP64 only when everything is FP64).
// HALO (sub-domain interior pass): a hop across the local boundary of a
// cut direction is left out; it arrives later as a face.
template <int PG, int PS, int RECON, int MU, bool DAG, bool HALO = false, bool PACK = false>
__device__ __forceinline__ void hop_dir(const DslashArgs& A, const char* in, int i, int full, const int c[4],
                                        int stepmu, typename RealT<PS>::type acc[24])
{
    typedef typename RealT<PS>::type R;
    const int L = A.g.L[MU];
    const int fwd = (c[MU] == L - 1) ? full - (L - 1) * stepmu : full + stepmu;
    const int bwd = (c[MU] == 0) ? full + (L - 1) * stepmu : full - stepmu;
    const bool tb = (MU == 3) && A.g.tanti;
    const bool cut = HALO && ((A.g.part >> MU) & 1);
    R v[24];
    if (!(cut && c[MU] == L - 1)) {
        SpinorIO<PS>::load(in, A.g.stride, fwd >> 1, v);
        hop_term<PG, RECON, MU, DAG, false, PACK>(A, v, tb && c[3] == L - 1, A.par, i, acc);
    }
    if (!(cut && c[MU] == 0)) {
        SpinorIO<PS>::load(in, A.g.stride, bwd >> 1, v);
        hop_term<PG, RECON, MU, DAG, true, PACK>(A, v, tb && c[3] == 0, 1 - A.par, bwd >> 1, acc);
    }
}

// ---- software-pipelined gather for half-precision spinors + recon-12 links
// The packed 16-bit data of hop d+1 (3 x uint4 + norm, 3 x uint2) is loaded
// before hop d is decoded and computed, so that two hops' loads are in
// flight per thread: half-precision loads move few bytes each, and one hop
// at a time does not cover DRAM latency.
template <int RECON>
struct HalfHopRaw {
    uint4 s[3];
    float n;
    uint32_t u[RECON == 12 ? 6 : 9];  // packed half2: two (recon-12) or three rows
};

struct HopPlan {
    int nb[8];      // neighbour checkerboard index per hop (2 mu: forward, 2 mu + 1: backward)
    int lidx[8];    // link index (the site itself forward, the neighbour backward)
    unsigned flip;  // bit h: the hop crosses the antiperiodic t boundary
};

template <int RECON>
__device__ __forceinline__ void load_half_hop(const char* in, const void* gauge, int stride, int par,
                                              const HopPlan& hp, int h, HalfHopRaw<RECON>& r)
{
    const uint4* sp = reinterpret_cast<const uint4*>(in);
    const int j = hp.nb[h];
    r.n = __ldg(reinterpret_cast<const float*>(sp + (size_t)3 * stride) + j);
#pragma unroll
    for (int k = 0; k < 3; ++k) r.s[k] = __ldg(sp + (size_t)k * stride + j);
    const int mu = h >> 1, lpar = (h & 1) ? 1 - par : par;
    if constexpr (RECON == 12) {
        const uint2* lp = static_cast<const uint2*>(gauge) + (size_t)((lpar * 4 + mu) * 3) * stride + hp.lidx[h];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const uint2 q = __ldg(lp + (size_t)k * stride);
            r.u[2 * k] = q.x;
            r.u[2 * k + 1] = q.y;
        }
    } else {
        const uint32_t* lp = static_cast<const uint32_t*>(gauge) + (size_t)((lpar * 4 + mu) * 9) * stride + hp.lidx[h];
#pragma unroll
        for (int k = 0; k < 9; ++k) r.u[k] = __ldg(lp + (size_t)k * stride);
    }
}

template <int ISBF, int RECON, int MU, bool BWD, bool DAG, bool PACK>
__device__ __forceinline__ void compute_half_hop(const HalfHopRaw<RECON>& r, bool flip, float acc[24])
{
    float v[24], h[12], u[18], w[12];
    // decode without the norm: the projection is linear, so the norm (and the
    // boundary sign) scale the 12 projected values instead of the 24 inputs
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const uint4 c = r.s[k];
        const float2 a = h2f(c.x, ISBF), b = h2f(c.y, ISBF), d = h2f(c.z, ISBF), e = h2f(c.w, ISBF);
        v[8 * k + 0] = a.x; v[8 * k + 1] = a.y; v[8 * k + 2] = b.x; v[8 * k + 3] = b.y;
        v[8 * k + 4] = d.x; v[8 * k + 5] = d.y; v[8 * k + 6] = e.x; v[8 * k + 7] = e.y;
    }
#pragma unroll
    for (int k = 0; k < (RECON == 12 ? 6 : 9); ++k) {
        const float2 a = h2f(r.u[k], ISBF);
        u[2 * k] = a.x;
        u[2 * k + 1] = a.y;
    }
    if constexpr (RECON == 12) reconstruct_row2(u);
    constexpr int S = (BWD != DAG) ? +1 : -1;  // forward (1 - g), backward (1 + g); swapped by DAG
    project<MU, S>(v, h);
    const float scale = flip ? -r.n : r.n;
#pragma unroll
    for (int k = 0; k < 12; ++k) h[k] *= scale;
    su3_mul_half<BWD, PACK>(u, h, w);
    accumulate<MU, S>(acc, w);
}

template <int ISBF, int RECON, bool DAG, bool PACK, int H>
__device__ __forceinline__ void half_pipeline_step(const char* in, const void* gauge, int stride, int par,
                                                   const HopPlan& hp, HalfHopRaw<RECON> (&buf)[2], float acc[24])
{
    if constexpr (H < 7) load_half_hop<RECON>(in, gauge, stride, par, hp, H + 1, buf[(H + 1) & 1]);
    compute_half_hop<ISBF, RECON, H / 2, (H & 1) != 0, DAG, PACK>(buf[H & 1], (hp.flip >> H) & 1u, acc);
    if constexpr (H < 7) half_pipeline_step<ISBF, RECON, DAG, PACK, H + 1>(in, gauge, stride, par, hp, buf, acc);
}

template <int ISBF, int RECON, bool DAG, bool PACK>
__device__ __forceinline__ void hop_all_half(const DslashArgs& A, const char* in, int i, int full, const int c[4],
                                             float acc[24])
{
    HopPlan hp;
    hp.flip = 0u;
    int step = 1;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        const int L = A.g.L[mu];
        const int fwd = (c[mu] == L - 1) ? full - (L - 1) * step : full + step;
        const int bwd = (c[mu] == 0) ? full + (L - 1) * step : full - step;
        hp.nb[2 * mu] = fwd >> 1;
        hp.nb[2 * mu + 1] = bwd >> 1;
        hp.lidx[2 * mu] = i;
        hp.lidx[2 * mu + 1] = bwd >> 1;
        step *= L;
    }
    if (A.g.tanti) {
        if (c[3] == A.g.L[3] - 1) hp.flip |= 1u << 6;
        if (c[3] == 0) hp.flip |= 1u << 7;
    }
    HalfHopRaw<RECON> buf[2];
    load_half_hop<RECON>(in, A.gauge, A.g.stride, A.par, hp, 0, buf[0]);
    half_pipeline_step<ISBF, RECON, DAG, PACK, 0>(in, A.gauge, A.g.stride, A.par, hp, buf, acc);
}

// Threads per block are at most DSLASH_MAX_BLOCK; DSLASH_MIN_BLOCKS resident
// blocks per SM caps the registers so that enough warps are in flight to
// cover the latency of the neighbour gathers.
#ifndef LQCD_DSLASH_MINB
#define LQCD_DSLASH_MINB 4  // <= 128 registers; 4, 5, 6 measured within 5% on 32^3x64
#endif
#define DSLASH_MAX_BLOCK 128
#define DSLASH_STAGED 1  // a "block size" that selects the shared-memory staged kernel (LQCD_BLOCK_STAGED)
// Epilogue at output site i of right-hand side rhs for the hopping term
// acc; nrm accumulates |out|^2 (|r|^2 for EPI_CG).
template <int PG, int PS, bool DAG, int EPI, bool RED>
__device__ __forceinline__ void dslash_epilogue(const DslashArgs& A, int rhs, int i, typename RealT<PS>::type acc[24],
                                                double& nrm)
{
    typedef typename RealT<PS>::type R;
    const R a = (R)A.a;
    if (EPI == EPI_NONE) {
#pragma unroll
        for (int k = 0; k < 24; ++k) acc[k] *= a;
    } else if (EPI == EPI_CLOVINV) {
        if (A.clov) {
            R t[24];
            clover_apply_site<PG>(A.clov, A.g.stride, i, acc, t);
#pragma unroll
            for (int k = 0; k < 24; ++k) acc[k] = a * t[k];
        } else {
#pragma unroll
            for (int k = 0; k < 24; ++k) acc[k] *= a;
        }
    } else {  // EPI_XPAY, EPI_CG
        R yv[24], t[24];
        SpinorIO<PS>::load(static_cast<const char*>(A.y) + rhs * A.y_rb, A.g.stride, i, yv);
        if (A.clov) {
            clover_apply_site<PG>(A.clov, A.g.stride, i, yv, t);
        } else {
#pragma unroll
            for (int k = 0; k < 24; ++k) t[k] = yv[k];
        }
#pragma unroll
        for (int k = 0; k < 24; ++k) acc[k] = t[k] + a * acc[k];
    }
    if constexpr (EPI == EPI_CG) {
        typedef typename RealT<AccumP<PS>::value>::type RA;
        const double* sc = A.scal + rhs * A.scal_rs;
        // alpha = |r|^2 / |Mp|^2; once r is exactly zero (an exact solution
        // inside a check interval) both vanish: no step instead of 0/0
        const double den = sc[A.s_den] + sc[A.s_den2];
        const RA alpha = den > 0.0 ? (RA)((sc[A.s_num] + sc[A.s_num2]) / den) : (RA)0;
        R pv[24];
        RA xv[24], rv[24];
        SpinorIO<PS>::load(static_cast<const char*>(A.p) + rhs * A.p_rb, A.g.stride, i, pv);
        char* xb = static_cast<char*>(A.x) + rhs * A.acc_rb;
        char* rb = static_cast<char*>(A.r) + rhs * A.acc_rb;
        SpinorIO<AccumP<PS>::value>::load(xb, A.g.stride, i, xv);
        SpinorIO<AccumP<PS>::value>::load(rb, A.g.stride, i, rv);
        RA n = 0;
#pragma unroll
        for (int k = 0; k < 24; ++k) {
            xv[k] += alpha * (RA)pv[k];
            rv[k] -= alpha * (RA)acc[k];
            n += rv[k] * rv[k];
        }
        nrm += (double)n;
        SpinorIO<AccumP<PS>::value>::store(xb, A.g.stride, i, xv);
        SpinorIO<AccumP<PS>::value>::store(rb, A.g.stride, i, rv);
    } else {
        SpinorIO<PS>::store(static_cast<char*>(A.out) + rhs * A.out_rb, A.g.stride, i, acc);
        if (RED) {
            R n = 0;
#pragma unroll
            for (int k = 0; k < 24; ++k) n += acc[k] * acc[k];
            nrm += (double)n;
        }
    }
}

// True if site c of a sub-domain has a neighbour across a cut boundary.
__device__ __forceinline__ bool on_cut_face(const Geom& g, const int c[4])
{
    bool f = false;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu)
        if (((g.part >> mu) & 1) && (c[mu] == 0 || c[mu] == g.L[mu] - 1)) f = true;
    return f;
}

// The hopping term and epilogue at output site i of right-hand side rhs;
// nrm accumulates |out|^2 (|r|^2 for EPI_CG).  HALO: the interior pass of a
// sub-domain; a site with a neighbour across a cut boundary stores its
// partial sum unfinished (no epilogue) for the face pass to complete.
template <int PG, int PS, int RECON, bool DAG, int EPI, bool RED, bool HALO = false>
__device__ __forceinline__ void dslash_site(const DslashArgs& A, int rhs, int i, double& nrm)
{
    typedef typename RealT<PS>::type R;
    int c[4];
    cb_coords(A.g, i, A.par, c);
    const int full = full_index(A.g, c);
    const char* in = static_cast<const char*>(A.in) + rhs * A.in_rb;
    R acc[24];
#pragma unroll
    for (int k = 0; k < 24; ++k) acc[k] = 0;
    // packed link products in the launches that neither reduce nor update
    // (measured faster there; slower in the reducing launches of the solver)
    constexpr bool PACK = !(RED || EPI == EPI_CG);
    if constexpr ((PS == P16 || PS == PB16) && PG == PS) {
        static_assert(!HALO, "sub-domain hops use the generic gather");
        hop_all_half<PS == PB16 ? 1 : 0, RECON, DAG, PACK>(A, in, i, full, c, acc);
    } else {
        hop_dir<PG, PS, RECON, 0, DAG, HALO, PACK>(A, in, i, full, c, 1, acc);
        hop_dir<PG, PS, RECON, 1, DAG, HALO, PACK>(A, in, i, full, c, A.g.L[0], acc);
        hop_dir<PG, PS, RECON, 2, DAG, HALO, PACK>(A, in, i, full, c, A.g.L[0] * A.g.L[1], acc);
        hop_dir<PG, PS, RECON, 3, DAG, HALO, PACK>(A, in, i, full, c, A.g.L[0] * A.g.L[1] * A.g.L[2], acc);
    }
    if (HALO && on_cut_face(A.g, c)) {
        SpinorIO<PS>::store(static_cast<char*>(A.out) + rhs * A.out_rb, A.g.stride, i, acc);
        return;
    }
    dslash_epilogue<PG, PS, DAG, EPI, RED>(A, rhs, i, acc, nrm);
}

// One-dimensional grid: block b serves right-hand side b % nrhs and site
// block b / nrhs, so that the blocks of all right-hand sides for the same
// sites run together and share each link (and clover) read through L2.
// (Applying each loaded link to several right-hand sides in one thread was
// measured slower: the extra accumulators cost occupancy in a kernel whose
// neighbour gathers are latency-bound.)
template <int PG, int PS, int RECON, bool DAG, int EPI, bool RED>
__global__ void __launch_bounds__(DSLASH_MAX_BLOCK, (PG == P64 ? 1 : LQCD_DSLASH_MINB))
    dslash_kernel(const DslashArgs A)
{
    const int rhs = (int)(blockIdx.x % (unsigned)A.nrhs);
    const int sb = (int)(blockIdx.x / (unsigned)A.nrhs), nsb = (int)(gridDim.x / (unsigned)A.nrhs);
    if (A.skip && A.skip[rhs]) return;  // uniform over the rhs: no block of it reduces
    double nrm = 0.0;
    if constexpr (RED || EPI == EPI_CG) {
        // grid-stride: the launcher runs one wave of blocks, so that each
        // block's partial sum covers many sites
        for (int i = sb * blockDim.x + threadIdx.x; i < A.g.Vh; i += nsb * blockDim.x)
            dslash_site<PG, PS, RECON, DAG, EPI, RED>(A, rhs, i, nrm);
        double v[1] = {nrm};
        block_reduce_finalize<1>(v, A.partials + rhs * A.part_rs, A.tickets + rhs, A.red + rhs * A.red_rs, sb, nsb);
    } else {
        const int i = sb * blockDim.x + threadIdx.x;
        if (i < A.g.Vh) dslash_site<PG, PS, RECON, DAG, EPI, RED>(A, rhs, i, nrm);
    }
}

// Launch helper: ceil(Vh / block) x nrhs blocks, one site per thread; for
// launches that reduce (fused norms, fused CG update) at most one wave of
// resident blocks, so that each block's partial sum covers more sites and the
// deterministic two-stage reduction handles 608 instead of 8192 partials at
// 32^3x64 (measured: solve 4 % faster; plain launches are faster with the
// full grid).
template <int PG, int PS, int RECON, bool DAG, int EPI, bool RED>
cudaError_t launch_dslash_t(const DslashArgs& A, int nrhs, int block, cudaStream_t s)
{
    static int wave[DSLASH_MAX_BLOCK / 32 + 1];  // per block size, 0 = not yet queried
    const int bi = block / 32;
    if ((RED || EPI == EPI_CG) && wave[bi] == 0) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dslash_kernel<PG, PS, RECON, DAG, EPI, RED>,
                                                              block, 0);
        if (e != cudaSuccess) return e;
        wave[bi] = per_sm > 0 && sms > 0 ? per_sm * sms : 1 << 30;
    }
    int gx = (A.g.Vh + block - 1) / block;
    if (RED || EPI == EPI_CG) {
        if (A.sites_per_thread > 0) {
            const long per_block = (long)block * A.sites_per_thread;
            gx = (int)((A.g.Vh + per_block - 1) / per_block);
        } else if (gx > wave[bi]) {
            gx = wave[bi];
        }
    }
    if ((long)gx * nrhs > 0x7fffffffL) return cudaErrorInvalidConfiguration;
    DslashArgs Ar = A;
    Ar.nrhs = nrhs;
    dslash_kernel<PG, PS, RECON, DAG, EPI, RED><<<gx * nrhs, block, 0, s>>>(Ar);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Shared-memory staged hop (plain launches, FP32 links): a block takes a
// tile of STG_TY x STG_TZ x STG_TT rows (y, z, t) of all Lx/2 checkerboard
// sites, one site per thread, and first copies the input spinors of the
// tile and of its six faces (the rows one step outside in y, z and t) into
// shared memory with asynchronous 16-byte copies, which hold no registers
// while in flight; every neighbour is then read from shared memory (x
// neighbours lie in the site's own row).  Faces are copied from the
// periodically wrapped rows.  Rows of the staging buffer: the tile's
// interior r = (tl TZ + zl) TY + yl, then y-, y+ (index tl TZ + zl), z-, z+
// (tl TY + yl), t-, t+ (zl TY + yl).
enum {
    STG_TY = 4, STG_TZ = 2, STG_TT = 2, STG_NIN = STG_TY * STG_TZ * STG_TT,
    STG_FY = STG_TZ * STG_TT, STG_FZ = STG_TY * STG_TT, STG_FT = STG_TY * STG_TZ,
    STG_NROW = STG_NIN + 2 * (STG_FY + STG_FZ + STG_FT), STG_MAXLXH = 16
};

__host__ __device__ inline bool staged_supported(const Geom& g)
{
    return g.part == 0 && g.Lxh <= STG_MAXLXH && g.L[1] % STG_TY == 0 && g.L[2] % STG_TZ == 0 &&
           g.L[3] % STG_TT == 0;
}

// Bytes of the staging buffer for spinor storage PS and Lx/2 = lxh.
__host__ __device__ inline size_t staged_smem_bytes(int PS, int lxh)
{
    const size_t ns = (size_t)STG_NROW * lxh;
    return PS == P32 ? ns * 96 : ns * 52;
}

// Checkerboard row index ((t Lz + z) Ly + y) of staging row r of the tile
// with origin (y0, z0, t0).
__device__ __forceinline__ int stg_row_global(const Geom& g, int r, int y0, int z0, int t0)
{
    int yl, zl, tl;
    if (r < STG_NIN) {
        yl = r % STG_TY;
        zl = (r / STG_TY) % STG_TZ;
        tl = r / (STG_TY * STG_TZ);
    } else if (r < STG_NIN + 2 * STG_FY) {
        const int q = r - STG_NIN, f = q % STG_FY;
        yl = q < STG_FY ? -1 : STG_TY;
        zl = f % STG_TZ;
        tl = f / STG_TZ;
    } else if (r < STG_NIN + 2 * (STG_FY + STG_FZ)) {
        const int q = r - STG_NIN - 2 * STG_FY, f = q % STG_FZ;
        zl = q < STG_FZ ? -1 : STG_TZ;
        yl = f % STG_TY;
        tl = f / STG_TY;
    } else {
        const int q = r - STG_NIN - 2 * (STG_FY + STG_FZ), f = q % STG_FT;
        tl = q < STG_FT ? -1 : STG_TT;
        yl = f % STG_TY;
        zl = f / STG_TY;
    }
    int y = y0 + yl, z = z0 + zl, t = t0 + tl;
    y = y < 0 ? y + g.L[1] : (y >= g.L[1] ? y - g.L[1] : y);
    z = z < 0 ? z + g.L[2] : (z >= g.L[2] ? z - g.L[2] : z);
    t = t < 0 ? t + g.L[3] : (t >= g.L[3] ? t - g.L[3] : t);
    return (t * g.L[2] + z) * g.L[1] + y;
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}

// A staged spinor (row-major staging rows, the field's chunk order).
template <int PS> struct SpinorSmem;
template <> struct SpinorSmem<P32> {
    __device__ __forceinline__ static void load(const unsigned char* sm, int ns, int j, float v[24])
    {
        const float4* p = reinterpret_cast<const float4*>(sm);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float4 c = p[k * ns + j];
            v[4 * k] = c.x;
            v[4 * k + 1] = c.y;
            v[4 * k + 2] = c.z;
            v[4 * k + 3] = c.w;
        }
    }
};
template <int ISBF> struct SpinorSmemHalf {
    __device__ __forceinline__ static void load(const unsigned char* sm, int ns, int j, float v[24])
    {
        const uint4* p = reinterpret_cast<const uint4*>(sm);
        const float n = reinterpret_cast<const float*>(p + 3 * ns)[j];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const uint4 c = p[k * ns + j];
            const float2 a = h2f(c.x, ISBF), b = h2f(c.y, ISBF), d = h2f(c.z, ISBF), e = h2f(c.w, ISBF);
            v[8 * k + 0] = a.x * n; v[8 * k + 1] = a.y * n;
            v[8 * k + 2] = b.x * n; v[8 * k + 3] = b.y * n;
            v[8 * k + 4] = d.x * n; v[8 * k + 5] = d.y * n;
            v[8 * k + 6] = e.x * n; v[8 * k + 7] = e.y * n;
        }
    }
};
template <> struct SpinorSmem<P16> : SpinorSmemHalf<0> {};
template <> struct SpinorSmem<PB16> : SpinorSmemHalf<1> {};

// One hop direction of the staged kernel: the neighbours' staging indices
// jf, jb, the backward link's checkerboard index bwd_cb.
template <int PG, int PS, int RECON, int MU, bool DAG>
__device__ __forceinline__ void hop_dir_staged(const DslashArgs& A, const unsigned char* sm, int ns, int i, int jf,
                                               int jb, int bwd_cb, bool flipf, bool flipb, float acc[24])
{
    float v[24];
    SpinorSmem<PS>::load(sm, ns, jf, v);
    hop_term<PG, RECON, MU, DAG, false, true>(A, v, flipf, A.par, i, acc);
    SpinorSmem<PS>::load(sm, ns, jb, v);
    hop_term<PG, RECON, MU, DAG, true, true>(A, v, flipb, 1 - A.par, bwd_cb, acc);
}

// Block b: right-hand side b % nrhs, tile b / nrhs (y fastest, then z, t);
// blockDim = STG_NIN * Lx/2.  Same arithmetic, in the same order, as the
// gathering kernel's plain launches.
template <int PG, int PS, int RECON, bool DAG, int EPI>
__global__ void __launch_bounds__(STG_NIN * STG_MAXLXH, 2) dslash_staged_kernel(const DslashArgs A)
{
    extern __shared__ __align__(16) unsigned char stg_smem[];
    const Geom& g = A.g;
    const int rhs = (int)(blockIdx.x % (unsigned)A.nrhs);
    if (A.skip && A.skip[rhs]) return;  // uniform over the block
    const int tile = (int)(blockIdx.x / (unsigned)A.nrhs);
    const int nty = g.L[1] / STG_TY, ntz = g.L[2] / STG_TZ;
    const int y0 = (tile % nty) * STG_TY, z0 = ((tile / nty) % ntz) * STG_TZ, t0 = (tile / (nty * ntz)) * STG_TT;
    const int lxh = g.Lxh, ns = STG_NROW * lxh;
    const int xh = threadIdx.x % lxh, rl = threadIdx.x / lxh;  // this thread's site in the tile
    const char* in = static_cast<const char*>(A.in) + rhs * A.in_rb;

    // stage: thread (rl, xh) copies column xh of rows rl, rl + NIN, ... of every chunk
    constexpr int NCH = PS == P32 ? 6 : 3;
    for (int q = rl; q < NCH * STG_NROW; q += STG_NIN) {
        const int k = q / STG_NROW, r = q - k * STG_NROW;
        const int gi = stg_row_global(g, r, y0, z0, t0) * lxh + xh;
        cp_async16(stg_smem + ((size_t)k * ns + r * lxh + xh) * 16, in + ((size_t)k * g.stride + gi) * 16);
    }
    if constexpr (PS != P32) {  // the per-site norms
        for (int r = rl; r < STG_NROW; r += STG_NIN) {
            const int gi = stg_row_global(g, r, y0, z0, t0) * lxh + xh;
            cp_async4(stg_smem + (size_t)3 * ns * 16 + (size_t)(r * lxh + xh) * 4,
                      in + (size_t)3 * g.stride * 16 + (size_t)gi * 4);
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();

    const int yl = rl % STG_TY, zl = (rl / STG_TY) % STG_TZ, tl = rl / (STG_TY * STG_TZ);
    int c[4];
    c[1] = y0 + yl;
    c[2] = z0 + zl;
    c[3] = t0 + tl;
    c[0] = 2 * xh + ((c[1] + c[2] + c[3] + A.par) & 1);
    const int i = ((c[3] * g.L[2] + c[2]) * g.L[1] + c[1]) * lxh + xh;
    const int full = full_index(g, c);
    const int row = rl * lxh;
    float acc[24];
#pragma unroll
    for (int k = 0; k < 24; ++k) acc[k] = 0.f;
    // staging indices of the eight neighbours and checkerboard indices of the backward links
    {
        const int xf = c[0] == g.L[0] - 1 ? 0 : c[0] + 1, xb = c[0] == 0 ? g.L[0] - 1 : c[0] - 1;
        const int bwd = c[0] == 0 ? full + (g.L[0] - 1) : full - 1;
        hop_dir_staged<PG, PS, RECON, 0, DAG>(A, stg_smem, ns, i, row + (xf >> 1), row + (xb >> 1), bwd >> 1, false,
                                              false, acc);
    }
    {
        const int s1 = g.L[0];
        const int jf = (yl + 1 < STG_TY ? rl + 1 : STG_NIN + STG_FY + tl * STG_TZ + zl) * lxh + xh;
        const int jb = (yl > 0 ? rl - 1 : STG_NIN + tl * STG_TZ + zl) * lxh + xh;
        const int bwd = c[1] == 0 ? full + (g.L[1] - 1) * s1 : full - s1;
        hop_dir_staged<PG, PS, RECON, 1, DAG>(A, stg_smem, ns, i, jf, jb, bwd >> 1, false, false, acc);
    }
    {
        const int s2 = g.L[0] * g.L[1];
        constexpr int bz = STG_NIN + 2 * STG_FY;
        const int jf = (zl + 1 < STG_TZ ? rl + STG_TY : bz + STG_FZ + tl * STG_TY + yl) * lxh + xh;
        const int jb = (zl > 0 ? rl - STG_TY : bz + tl * STG_TY + yl) * lxh + xh;
        const int bwd = c[2] == 0 ? full + (g.L[2] - 1) * s2 : full - s2;
        hop_dir_staged<PG, PS, RECON, 2, DAG>(A, stg_smem, ns, i, jf, jb, bwd >> 1, false, false, acc);
    }
    {
        const int s3 = g.L[0] * g.L[1] * g.L[2];
        constexpr int bt = STG_NIN + 2 * (STG_FY + STG_FZ);
        const int jf = (tl + 1 < STG_TT ? rl + STG_TY * STG_TZ : bt + STG_FT + zl * STG_TY + yl) * lxh + xh;
        const int jb = (tl > 0 ? rl - STG_TY * STG_TZ : bt + zl * STG_TY + yl) * lxh + xh;
        const int bwd = c[3] == 0 ? full + (g.L[3] - 1) * s3 : full - s3;
        const bool tb = g.tanti != 0;
        hop_dir_staged<PG, PS, RECON, 3, DAG>(A, stg_smem, ns, i, jf, jb, bwd >> 1, tb && c[3] == g.L[3] - 1,
                                              tb && c[3] == 0, acc);
    }
    double nrm = 0.0;
    dslash_epilogue<PG, PS, DAG, EPI, false>(A, rhs, i, acc, nrm);
}

template <int PG, int PS, int RECON, bool DAG, int EPI>
cudaError_t launch_staged_t(const DslashArgs& A, int nrhs, cudaStream_t s)
{
    // the largest buffer (Lx/2 = 16) is allowed once per instantiation and device
    static bool attr[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !attr[dev]) {
        e = cudaFuncSetAttribute(dslash_staged_kernel<PG, PS, RECON, DAG, EPI>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)staged_smem_bytes(PS, STG_MAXLXH));
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr[dev] = true;
    }
    const long tiles = (long)(A.g.L[1] / STG_TY) * (A.g.L[2] / STG_TZ) * (A.g.L[3] / STG_TT);
    if (tiles * nrhs > 0x7fffffffL) return cudaErrorInvalidConfiguration;
    DslashArgs Ar = A;
    Ar.nrhs = nrhs;
    dslash_staged_kernel<PG, PS, RECON, DAG, EPI>
        <<<(unsigned)(tiles * nrhs), STG_NIN * A.g.Lxh, staged_smem_bytes(PS, A.g.Lxh), s>>>(Ar);
    return cudaGetLastError();
}

// Runtime dispatch over (recon, dag, epi, red) for fixed storage precisions.
// block == DSLASH_STAGED: the staged kernel where it applies (plain launches
// with FP32 links on an uncut lattice whose extents fit its tiles), else the
// gathering kernel with its default block.
template <int PG, int PS>
cudaError_t dispatch_dslash_p(const DslashArgs& A, int recon, bool dag, int epi, bool red, int nrhs, int block,
                              cudaStream_t s)
{
    if (block == DSLASH_STAGED) {
        if constexpr (PG == P32 && PS != P64) {
            if (!red && epi != EPI_CG && recon == 12 && staged_supported(A.g)) {
#define LQ_SCASE(DG, EP) \
    if (dag == DG && epi == EP) return launch_staged_t<PG, PS, 12, DG, EP>(A, nrhs, s);
                LQ_SCASE(false, EPI_NONE)
                LQ_SCASE(false, EPI_CLOVINV)
                LQ_SCASE(false, EPI_XPAY)
                LQ_SCASE(true, EPI_NONE)
                LQ_SCASE(true, EPI_CLOVINV)
                LQ_SCASE(true, EPI_XPAY)
#undef LQ_SCASE
            }
        }
        block = DSLASH_MAX_BLOCK;
    }
#define LQ_CASE(RC, DG, EP, RD)                                                              \
    if (recon == RC && dag == DG && epi == EP && red == RD)                                 \
        return launch_dslash_t<PG, PS, RC, DG, EP, RD>(A, nrhs, block, s);
#define LQ_EPIS(RC, DG)                  \
    LQ_CASE(RC, DG, EPI_NONE, false)     \
    LQ_CASE(RC, DG, EPI_CLOVINV, false)  \
    LQ_CASE(RC, DG, EPI_XPAY, false)     \
    LQ_CASE(RC, DG, EPI_XPAY, true)      \
    LQ_CASE(RC, DG, EPI_CG, true)
    if constexpr (PG == P64) {
        LQ_EPIS(18, false)
        LQ_EPIS(18, true)
    } else {
        LQ_EPIS(12, false)
        LQ_EPIS(12, true)
        LQ_EPIS(18, false)
        LQ_EPIS(18, true)
    }
#undef LQ_EPIS
#undef LQ_CASE
    return cudaErrorInvalidValue;
}

}  // namespace lqcd
