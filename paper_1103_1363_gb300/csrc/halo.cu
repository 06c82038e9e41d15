// Halo exchange of a sub-domain: the hopping term of one piece of a lattice
// cut into sub-domains (one per GPU), with the spin-projected faces of the
// cut boundaries exchanged between them.
//
// The paper's multi-node codes split the lattice over nodes and communicate
// boundaries between sweeps; the Schur operator's two sweeps each need the
// other parity's border (Sec. 5, two-sweep paragraph), and SAP overlaps the
// border traffic with the block solves of the other colour (Sec. 5, SAP).
// Here a sweep is
//   pack:      each sub-domain projects the input spinors on its first and
//              last slices of every cut direction to half spinors (12 reals;
//              the ones sent forward are also multiplied by the sub-domain's
//              own link U_mu^dag, so that no neighbour needs another's links);
//   exchange:  the faces travel to the neighbours (send/recv or copies, by
//              the caller; receive side 0 comes from the forward neighbour);
//   interior:  the hopping kernel with every hop across a cut boundary left
//              out; output sites next to such a boundary keep their partial
//              sum unfinished;
//   faces:     one thread per output site next to a cut boundary adds the
//              received faces (U_mu(x) h for forward hops, the received
//              U^dag h for backward ones; the fermion sign of hops across the
//              global t boundary) and applies the epilogue.
// The interior pass needs no faces, so the exchange can run beside it.
#include <cstring>
#include <vector>

#include "internal.h"

namespace lqcd {

namespace {

// Directions other than mu, increasing: the face coordinates.
__device__ __forceinline__ void face_dirs(int mu, int d[3])
{
    int k = 0;
#pragma unroll
    for (int m = 0; m < 4; ++m)
        if (m != mu) d[k++] = m;
}

// Face index of site c on a face normal to mu (one parity of the face).
__device__ __forceinline__ int face_index(const Geom& g, int mu, const int c[4])
{
    int d[3];
    face_dirs(mu, d);
    const int lex = (c[d[2]] * g.L[d[1]] + c[d[1]]) * g.L[d[0]] + c[d[0]];
    return lex >> 1;
}

// Site of parity q on slice s of the face normal to mu with face index fi.
__device__ __forceinline__ void face_site(const Geom& g, int mu, int s, int q, int fi, int c[4])
{
    int d[3];
    face_dirs(mu, d);
    int lex = 2 * fi;
    c[d[0]] = lex % g.L[d[0]];
    lex /= g.L[d[0]];
    c[d[1]] = lex % g.L[d[1]];
    c[d[2]] = lex / g.L[d[1]];
    c[mu] = s;
    if (((c[0] + c[1] + c[2] + c[3]) & 1) != q) c[d[0]] += 1;  // L[d[0]] is even: stays inside
}

// 12 reals of a face site: FP64 as 6 double2 chunks, FP32 as 3 float4 chunks,
// [chunk][face site].
template <class R> struct FaceIO;
template <> struct FaceIO<double> {
    __device__ __forceinline__ static void load(const char* seg, int nf, int f, double h[12])
    {
        const double2* p = reinterpret_cast<const double2*>(seg);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const double2 v = p[(size_t)k * nf + f];
            h[2 * k] = v.x;
            h[2 * k + 1] = v.y;
        }
    }
    __device__ __forceinline__ static void store(char* seg, int nf, int f, const double h[12])
    {
        double2* p = reinterpret_cast<double2*>(seg);
#pragma unroll
        for (int k = 0; k < 6; ++k) p[(size_t)k * nf + f] = make_double2(h[2 * k], h[2 * k + 1]);
    }
};
template <> struct FaceIO<float> {
    __device__ __forceinline__ static void load(const char* seg, int nf, int f, float h[12])
    {
        const float4* p = reinterpret_cast<const float4*>(seg);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float4 v = p[(size_t)k * nf + f];
            h[4 * k] = v.x;
            h[4 * k + 1] = v.y;
            h[4 * k + 2] = v.z;
            h[4 * k + 3] = v.w;
        }
    }
    __device__ __forceinline__ static void store(char* seg, int nf, int f, const float h[12])
    {
        float4* p = reinterpret_cast<float4*>(seg);
#pragma unroll
        for (int k = 0; k < 3; ++k) p[(size_t)k * nf + f] = make_float4(h[4 * k], h[4 * k + 1], h[4 * k + 2], h[4 * k + 3]);
    }
};

struct HaloSeg {
    size_t off[8];   // segment 2 mu + side, bytes from the start of a buffer set
    int nf[4];       // face sites of one parity per direction
    size_t set_bytes;
};

// Send faces of direction MU for input parity q: side 0 (first slice) the
// forward hop's projection, side 1 (last slice) U_mu^dag times the backward
// hop's projection.
template <int P, int RECON, int MU, bool DAG>
__global__ void halo_pack_kernel(Geom g, const void* gauge, const char* in, size_t in_rb, char* send, HaloSeg hs,
                                 int q)
{
    typedef typename RealT<P>::type R;
    const int nf = hs.nf[MU];
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    const int side = blockIdx.y, rhs = blockIdx.z;
    if (f >= nf) return;
    int c[4];
    face_site(g, MU, side == 0 ? 0 : g.L[MU] - 1, q, f, c);
    const int i = full_index(g, c) >> 1;
    R v[24], h[12];
    SpinorIO<P>::load(in + rhs * in_rb, g.stride, i, v);
    char* seg = send + rhs * hs.set_bytes + hs.off[2 * MU + side];
    if (side == 0) {
        project<MU, DAG ? +1 : -1>(v, h);
        FaceIO<R>::store(seg, nf, f, h);
    } else {
        R u[18], w[12];
        project<MU, DAG ? -1 : +1>(v, h);
        GaugeIO<P, RECON>::load(gauge, g.stride, q, MU, i, u);
        su3_mul_half<true>(u, h, w);
        FaceIO<R>::store(seg, nf, f, w);
    }
}

// Face contributions of direction MU at output site i (coordinates c).
template <int P, int RECON, int MU, bool DAG>
__device__ __forceinline__ void add_faces(const DslashArgs& A, const char* recv, const HaloSeg& hs, int i,
                                          const int c[4], typename RealT<P>::type acc[24])
{
    typedef typename RealT<P>::type R;
    if (!((A.g.part >> MU) & 1)) return;
    const int nf = hs.nf[MU];
    R h[12], w[12];
    if (c[MU] == A.g.L[MU] - 1) {  // forward hop: U_mu(x) times the neighbour's projection
        FaceIO<R>::load(recv + hs.off[2 * MU], nf, face_index(A.g, MU, c), h);
        if (MU == 3 && A.g.tanti && A.g.tlast) {
#pragma unroll
            for (int k = 0; k < 12; ++k) h[k] = -h[k];
        }
        R u[18];
        GaugeIO<P, RECON>::load(A.gauge, A.g.stride, A.par, MU, i, u);
        su3_mul_half<false>(u, h, w);
        accumulate<MU, DAG ? +1 : -1>(acc, w);
    }
    if (c[MU] == 0) {  // backward hop: the neighbour sent U^dag times its projection
        FaceIO<R>::load(recv + hs.off[2 * MU + 1], nf, face_index(A.g, MU, c), w);
        if (MU == 3 && A.g.tanti && A.g.tfirst) {
#pragma unroll
            for (int k = 0; k < 12; ++k) w[k] = -w[k];
        }
        accumulate<MU, DAG ? -1 : +1>(acc, w);
    }
}

// Face pass: output sites next to a cut boundary add the received faces to
// the interior pass's partial sum (in out) and apply the epilogue.
template <int P, int RECON, bool DAG, int EPI>
__global__ void __launch_bounds__(128) halo_faces_kernel(const DslashArgs A, const char* recv, HaloSeg hs)
{
    typedef typename RealT<P>::type R;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int rhs = blockIdx.y;
    if (i >= A.g.Vh) return;
    int c[4];
    cb_coords(A.g, i, A.par, c);
    if (!on_cut_face(A.g, c)) return;
    R acc[24];
    SpinorIO<P>::load(static_cast<const char*>(A.out) + rhs * A.out_rb, A.g.stride, i, acc);
    const char* rv = recv + rhs * hs.set_bytes;
    add_faces<P, RECON, 0, DAG>(A, rv, hs, i, c, acc);
    add_faces<P, RECON, 1, DAG>(A, rv, hs, i, c, acc);
    add_faces<P, RECON, 2, DAG>(A, rv, hs, i, c, acc);
    add_faces<P, RECON, 3, DAG>(A, rv, hs, i, c, acc);
    double nrm = 0.0;
    dslash_epilogue<P, P, DAG, EPI, false>(A, rhs, i, acc, nrm);
}

// Interior pass: the hopping kernel with the hops across cut boundaries left out.
template <int P, int RECON, bool DAG, int EPI>
__global__ void __launch_bounds__(DSLASH_MAX_BLOCK) halo_interior_kernel(const DslashArgs A)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int rhs = blockIdx.y;
    double nrm = 0.0;
    if (i < A.g.Vh) dslash_site<P, P, RECON, DAG, EPI, false, true>(A, rhs, i, nrm);
}

HaloSeg halo_segments(const lqcd_ctx* c, int P)
{
    HaloSeg hs;
    memset(&hs, 0, sizeof(hs));
    const size_t real = P == P64 ? 8 : 4;
    size_t off = 0;
    for (int mu = 0; mu < 4; ++mu) {
        if (!((c->g.part >> mu) & 1)) continue;
        hs.nf[mu] = (int)(c->volume / c->g.L[mu] / 2);
        for (int side = 0; side < 2; ++side) {
            hs.off[2 * mu + side] = off;
            off += ((size_t)hs.nf[mu] * 12 * real + 255) & ~(size_t)255;
        }
    }
    hs.set_bytes = off;
    return hs;
}

template <int P, int RECON, bool DAG>
cudaError_t pack_t(const lqcd_ctx* c, const char* in, size_t in_rb, char* send, const HaloSeg& hs, int q, int nrhs)
{
    for (int mu = 0; mu < 4; ++mu) {
        if (!((c->g.part >> mu) & 1)) continue;
        dim3 grid((hs.nf[mu] + 127) / 128, 2, nrhs);
        switch (mu) {
        case 0: halo_pack_kernel<P, RECON, 0, DAG><<<grid, 128, 0, c->stream>>>(c->g, c->gauge[P], in, in_rb, send, hs, q); break;
        case 1: halo_pack_kernel<P, RECON, 1, DAG><<<grid, 128, 0, c->stream>>>(c->g, c->gauge[P], in, in_rb, send, hs, q); break;
        case 2: halo_pack_kernel<P, RECON, 2, DAG><<<grid, 128, 0, c->stream>>>(c->g, c->gauge[P], in, in_rb, send, hs, q); break;
        default: halo_pack_kernel<P, RECON, 3, DAG><<<grid, 128, 0, c->stream>>>(c->g, c->gauge[P], in, in_rb, send, hs, q); break;
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <int P, int RECON, bool DAG, int EPI>
cudaError_t passes_t(const lqcd_ctx* c, const DslashArgs& A, const char* recv, const HaloSeg& hs, int stage, int nrhs)
{
    dim3 grid((c->g.Vh + 127) / 128, nrhs);
    if (stage != 2) halo_interior_kernel<P, RECON, DAG, EPI><<<grid, 128, 0, c->stream>>>(A);
    if (stage != 1) halo_faces_kernel<P, RECON, DAG, EPI><<<grid, 128, 0, c->stream>>>(A, recv, hs);
    return cudaGetLastError();
}

template <int P, int RECON>
cudaError_t passes_p(const lqcd_ctx* c, const DslashArgs& A, const char* recv, const HaloSeg& hs, bool dag, int epi,
                     int stage, int nrhs)
{
#define LQ_H(DG, EP) if (dag == DG && epi == EP) return passes_t<P, RECON, DG, EP>(c, A, recv, hs, stage, nrhs)
    LQ_H(false, EPI_NONE); LQ_H(false, EPI_CLOVINV); LQ_H(false, EPI_XPAY);
    LQ_H(true, EPI_NONE); LQ_H(true, EPI_CLOVINV); LQ_H(true, EPI_XPAY);
#undef LQ_H
    return cudaErrorInvalidValue;
}

lqcd_status check_halo(const lqcd_ctx* c, int prec, int nrhs)
{
    if (!c) return fail(LQCD_ERR_INVALID, "null context");
    if (!c->ws) return fail(LQCD_ERR_NOMEM, "no workspace: call lqcd_set_workspace");
    if (!c->cut()) return fail(LQCD_ERR_STATE, "halo: the context is not a sub-domain of a cut lattice");
    if (prec != LQCD_F64 && prec != LQCD_F32) return fail(LQCD_ERR_INVALID, "halo: LQCD_F64 or LQCD_F32 storage only");
    if (!c->holds(prec)) return fail(LQCD_ERR_STATE, "halo: precision not held by this context");
    if (!c->gauge_loaded) return fail(LQCD_ERR_STATE, "halo: no gauge field loaded");
    if (nrhs < 1) return fail(LQCD_ERR_INVALID, "halo: nrhs must be >= 1");
    return LQCD_OK;
}

}  // namespace

}  // namespace lqcd

using namespace lqcd;

extern "C" {

lqcd_status lqcd_halo_layout(const lqcd_ctx* c, lqcd_prec prec, size_t off[8], size_t len[8], size_t* total)
{
    if (!c || !total) return fail(LQCD_ERR_INVALID, "lqcd_halo_layout: null argument");
    if (prec != LQCD_F64 && prec != LQCD_F32) return fail(LQCD_ERR_INVALID, "lqcd_halo_layout: LQCD_F64 or LQCD_F32 only");
    const HaloSeg hs = halo_segments(c, prec);
    const size_t real = prec == LQCD_F64 ? 8 : 4;
    for (int k = 0; k < 8; ++k) {
        const int mu = k / 2;
        if (off) off[k] = hs.off[k];
        if (len) len[k] = (size_t)hs.nf[mu] * 12 * real;
    }
    *total = hs.set_bytes;
    return LQCD_OK;
}

lqcd_status lqcd_halo_pack(lqcd_ctx* c, void* send, const void* in, int parity, int dag, lqcd_prec prec, int nrhs)
{
    try {
        LQ_TRY(check_halo(c, prec, nrhs));
        if (!send || !in) return fail(LQCD_ERR_INVALID, "lqcd_halo_pack: null buffer");
        if (parity != 0 && parity != 1) return fail(LQCD_ERR_INVALID, "lqcd_halo_pack: parity must be 0 or 1");
        DeviceScope dev_scope;
        LQ_TRY(dev_scope.enter(c->device));
        const HaloSeg hs = halo_segments(c, prec);
        const size_t fb = c->field_bytes(prec);
        const char* ip = static_cast<const char*>(in);
        char* sp = static_cast<char*>(send);
        cudaError_t e;
        const int rc = c->recon_of(prec);
        if (prec == LQCD_F64) e = dag ? pack_t<P64, 18, true>(c, ip, fb, sp, hs, parity, nrhs)
                                      : pack_t<P64, 18, false>(c, ip, fb, sp, hs, parity, nrhs);
        else if (rc == 12) e = dag ? pack_t<P32, 12, true>(c, ip, fb, sp, hs, parity, nrhs)
                                   : pack_t<P32, 12, false>(c, ip, fb, sp, hs, parity, nrhs);
        else e = dag ? pack_t<P32, 18, true>(c, ip, fb, sp, hs, parity, nrhs)
                     : pack_t<P32, 18, false>(c, ip, fb, sp, hs, parity, nrhs);
        LQ_CUDA(e);
        c->launches++;
        return LQCD_OK;
    } catch (...) {
        return fail(LQCD_ERR_INVALID, "unexpected exception");
    }
}

lqcd_status lqcd_halo_dslash(lqcd_ctx* c, void* out, const void* in, const void* recv, int parity, int dag, int epi,
                             const void* y, double a, int stage, lqcd_prec prec, int nrhs)
{
    try {
        LQ_TRY(check_halo(c, prec, nrhs));
        if (!out || !in) return fail(LQCD_ERR_INVALID, "lqcd_halo_dslash: null field");
        if (parity != 0 && parity != 1) return fail(LQCD_ERR_INVALID, "lqcd_halo_dslash: parity must be 0 or 1");
        if (epi < 0 || epi > 2) return fail(LQCD_ERR_INVALID, "lqcd_halo_dslash: epi must be 0, 1 or 2");
        if (stage < 0 || stage > 2) return fail(LQCD_ERR_INVALID, "lqcd_halo_dslash: stage must be 0, 1 or 2");
        if (stage != 1 && !recv) return fail(LQCD_ERR_INVALID, "lqcd_halo_dslash: the face pass needs recv");
        if (epi == 2 && !y) return fail(LQCD_ERR_INVALID, "lqcd_halo_dslash: epi 2 needs y");
        if (out == in || (y && out == y)) return fail(LQCD_ERR_INVALID, "lqcd_halo_dslash: out must not alias in or y");
        DeviceScope dev_scope;
        LQ_TRY(dev_scope.enter(c->device));
        const HaloSeg hs = halo_segments(c, prec);
        const size_t fb = c->field_bytes(prec);
        DslashArgs A = base_args(c, prec);
        A.par = parity;
        A.out = out;
        A.out_rb = fb;
        A.in = in;
        A.in_rb = fb;
        A.clov = nullptr;  // a cut context has no clover term (A = 1)
        A.y = y;
        A.y_rb = fb;
        A.a = a;
        A.nrhs = nrhs;
        const int ep = epi == 0 ? EPI_NONE : epi == 1 ? EPI_CLOVINV : EPI_XPAY;
        const char* rv = static_cast<const char*>(recv);
        cudaError_t e;
        if (prec == LQCD_F64) e = passes_p<P64, 18>(c, A, rv, hs, dag != 0, ep, stage, nrhs);
        else if (c->recon_of(prec) == 12) e = passes_p<P32, 12>(c, A, rv, hs, dag != 0, ep, stage, nrhs);
        else e = passes_p<P32, 18>(c, A, rv, hs, dag != 0, ep, stage, nrhs);
        LQ_CUDA(e);
        c->launches += stage == 0 ? 2 : 1;
        c->dslash_count += stage != 2 ? nrhs : 0;
        return LQCD_OK;
    } catch (...) {
        return fail(LQCD_ERR_INVALID, "unexpected exception");
    }
}

lqcd_status lqcd_norm2(lqcd_ctx* c, const void* field, int parity, lqcd_prec prec, int nrhs, double* out)
{
    try {
        if (!c || !field || !out) return fail(LQCD_ERR_INVALID, "lqcd_norm2: null argument");
        if (!c->ws) return fail(LQCD_ERR_NOMEM, "no workspace: call lqcd_set_workspace");
        if (!valid_mode(prec))
            return fail(LQCD_ERR_INVALID, "lqcd_norm2: bad precision");
        if (parity < -1 || parity > 1) return fail(LQCD_ERR_INVALID, "lqcd_norm2: parity must be -1, 0 or 1");
        if (nrhs < 1 || nrhs > c->cfg.max_nrhs) return fail(LQCD_ERR_INVALID, "lqcd_norm2: need 1 <= nrhs <= max_nrhs");
        DeviceScope dev_scope;
        LQ_TRY(dev_scope.enter(c->device));
        const size_t fb = c->field_bytes(prec);
        const int nf = parity < 0 ? 2 : 1;
        LQ_TRY(blas_norm2(c, field, mode_ps(prec), nrhs, nf * fb, nf, SC_TMP + 5));
        std::vector<double> h((size_t)nrhs * SC_PER_RHS);
        LQ_CUDA(cudaMemcpyAsync(h.data(), c->scal, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        LQ_CUDA(cudaStreamSynchronize(c->stream));
        for (int r = 0; r < nrhs; ++r) out[r] = h[(size_t)r * SC_PER_RHS + SC_TMP + 5];
        return LQCD_OK;
    } catch (...) {
        return fail(LQCD_ERR_NOMEM, "lqcd_norm2: host allocation failed");
    }
}

}  // extern "C"
