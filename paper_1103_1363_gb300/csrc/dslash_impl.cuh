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
    R v[24], h[12], u[18], w[12];
    // forward: (1 - g) U_mu(x) in(x + mu)   [dagger: (1 + g)]
    if (!(cut && c[MU] == L - 1)) {
        SpinorIO<PS>::load(in, A.g.stride, fwd >> 1, v);
        project<MU, DAG ? +1 : -1>(v, h);
        if (tb && c[3] == L - 1) {
#pragma unroll
            for (int k = 0; k < 12; ++k) h[k] = -h[k];
        }
        GaugeIO<PG, RECON>::load(A.gauge, A.g.stride, A.par, MU, i, u);
        su3_mul_half<false, PACK>(u, h, w);
        accumulate<MU, DAG ? +1 : -1>(acc, w);
    }
    // backward: (1 + g) U_mu(x - mu)^dag in(x - mu)   [dagger: (1 - g)]
    if (!(cut && c[MU] == 0)) {
        SpinorIO<PS>::load(in, A.g.stride, bwd >> 1, v);
        project<MU, DAG ? -1 : +1>(v, h);
        if (tb && c[3] == 0) {
#pragma unroll
            for (int k = 0; k < 12; ++k) h[k] = -h[k];
        }
        GaugeIO<PG, RECON>::load(A.gauge, A.g.stride, 1 - A.par, MU, bwd >> 1, u);
        su3_mul_half<true, PACK>(u, h, w);
        accumulate<MU, DAG ? -1 : +1>(acc, w);
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

// Runtime dispatch over (recon, dag, epi, red) for fixed storage precisions.
template <int PG, int PS>
cudaError_t dispatch_dslash_p(const DslashArgs& A, int recon, bool dag, int epi, bool red, int nrhs, int block,
                              cudaStream_t s)
{
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
