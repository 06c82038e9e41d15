// Flexible GCR(k) on the full Wilson-clover operator with a right
// preconditioner (identity, SAP or the parallel-transport network).
//
// The paper's outer solver is FGCR: it stores two vectors per iteration
// (z_k and w_k = M z_k), so it is restarted, and it tolerates a
// preconditioner that is not a fixed operator; mixed precision is
// iterative refinement, i.e. the recursion runs in single precision and the
// residual is recomputed in double precision at each restart (Sec. 5).
//
// Here w_k is orthogonalised against the earlier w_j by classical
// Gram-Schmidt: one kernel forms <w_j, w_k>, <w_k, r> and |w_k|^2, the host
// forms c_j = <w_j, w_k>/|w_j|^2 and the step a = <w_k, r>/|w^_k|^2 with
// |w^_k|^2 = |w_k|^2 - sum_j |<w_j, w_k>|^2/|w_j|^2, and one fused kernel
// writes w^_k = w_k - sum_j c_j w_j and r -= a w^_k.  When that estimate
// shows cancellation (|w^_k|^2 < |w_k|^2 / 2, the "twice is enough"
// criterion of Daniel, Gragg, Kaufman and Stewart) a second pass runs first.
// r is orthogonal to the earlier w^_j, so <w^_k, r> = <w_k, r>.  The z_k are
// not orthogonalised: with U the unit upper triangle of the coefficients
// c_jk, the cycle's correction is x += Z U^{-1} a, formed once at the end of
// the cycle.  In exact arithmetic these are the iterates of GCR with
// modified Gram-Schmidt on both w and z.
//
// A cycle ends (FP64 residual, restart) after nkrylov directions, or once
// the FP32 residual has fallen by GCR_CYCLE_REDUCTION from the cycle's start,
// or when a new direction lies numerically in the span of the earlier ones:
// past FP32's resolution of the starting residual the recursion only adds
// rounding, and the rebuilt solution would no longer match it.
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "internal.h"

namespace lqcd {

lqcd_status net_apply_internal(lqcd_net* n, void* z, const void* r, size_t rb);

enum { GCR_KMAX = 24, GCR_NDOT = 2 * GCR_KMAX + 8 };  // the last chunk writes 8 values at 2 GCR_KMAX
constexpr double GCR_CYCLE_REDUCTION = 1e-5;

// out[2j, 2j+1] = <w_j, w_k> (j < k), out[2 KMAX, 2 KMAX + 1] = <w_k, r>,
// out[2 KMAX + 2] = |w_k|^2.  The dots are split over blockIdx.y in chunks
// of GCR_CH basis vectors (chunk c < nch_j: j = c GCR_CH ..; the last chunk
// the dots with r), each with its own partials, ticket and eight outputs, so
// that a thread loads at most GCR_CH + 1 fields per site instead of k + 2 in
// a chain.  FP32 sums per thread, FP64 across threads.
enum { GCR_CH = 4 };

__global__ void gcr_dots_kernel(Geom g, const char* W, size_t fld, int k, const char* wk, const char* r,
                                double* partials, unsigned* tickets, double* out)
{
    const int c = blockIdx.y, nch_j = (k + GCR_CH - 1) / GCR_CH;
    const bool with_r = c == nch_j;
    const int j0 = c * GCR_CH, cnt = with_r ? 0 : min(GCR_CH, k - j0);
    float acc[2 * GCR_CH];
#pragma unroll
    for (int j = 0; j < 2 * GCR_CH; ++j) acc[j] = 0.f;
    const size_t fb = fld / 2;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.Vh; i += gridDim.x * blockDim.x)
        for (int par = 0; par < 2; ++par) {
            float vv[24];
            SpinorIO<P32>::load(wk + par * fb, g.stride, i, vv);
            if (with_r) {
                float rv[24];
                SpinorIO<P32>::load(r + par * fb, g.stride, i, rv);
                float re = 0.f, im = 0.f, nn = 0.f;
#pragma unroll
                for (int q = 0; q < 12; ++q) {
                    re += vv[2 * q] * rv[2 * q] + vv[2 * q + 1] * rv[2 * q + 1];
                    im += vv[2 * q] * rv[2 * q + 1] - vv[2 * q + 1] * rv[2 * q];
                    nn += vv[2 * q] * vv[2 * q] + vv[2 * q + 1] * vv[2 * q + 1];
                }
                acc[0] += re;
                acc[1] += im;
                acc[2] += nn;
                continue;
            }
#pragma unroll
            for (int j = 0; j < GCR_CH; ++j) {
                if (j >= cnt) break;
                float w[24];
                SpinorIO<P32>::load(W + (size_t)(j0 + j) * fld + par * fb, g.stride, i, w);
                float re = 0.f, im = 0.f;
#pragma unroll
                for (int q = 0; q < 12; ++q) {
                    re += w[2 * q] * vv[2 * q] + w[2 * q + 1] * vv[2 * q + 1];
                    im += w[2 * q] * vv[2 * q + 1] - w[2 * q + 1] * vv[2 * q];
                }
                acc[2 * j] += re;
                acc[2 * j + 1] += im;
            }
        }
    double d[2 * GCR_CH];
#pragma unroll
    for (int j = 0; j < 2 * GCR_CH; ++j) d[j] = acc[j];
    block_reduce_finalize<2 * GCR_CH>(d, partials + (size_t)c * gridDim.x * 2 * GCR_CH, tickets + c,
                                      out + (with_r ? 2 * GCR_KMAX : 2 * j0));
}

struct GcrStep {
    float2 c[GCR_KMAX];  // w_k -= sum_j c_j w_j
    float2 a;            // r -= a w_k (after the projection)
    int update_r;
};

// w_k -= sum_j c_j w_j; if update_r: r -= a w_k.  out[0] = |r|^2, out[1] = |w_k|^2.
__global__ void gcr_orth_update_kernel(Geom g, const char* W, size_t fld, int k, char* wk, char* r, GcrStep st,
                                       double* partials, unsigned* ticket, double* out)
{
    // one thread per (parity, float4 chunk, site): the update is elementwise,
    // so six threads share a site, each running the chain of k loads for its
    // chunk (six times the loads in flight of a thread per site)
    double acc[2] = {0.0, 0.0};
    const size_t fb = fld / 2;
    const long n = 12L * g.Vh;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
        const int pq = (int)(e / g.Vh), i = (int)(e - (long)pq * g.Vh);
        const int par = pq / 6, q = pq - 6 * par;
        const size_t off = par * fb + ((size_t)q * g.stride + i) * sizeof(float4);
        float4 a = *reinterpret_cast<const float4*>(wk + off);
        for (int j = 0; j < k; ++j) {
            const float4 w = __ldg(reinterpret_cast<const float4*>(W + j * fld + off));
            const float xr = st.c[j].x, xi = st.c[j].y;
            a.x -= xr * w.x - xi * w.y;
            a.y -= xr * w.y + xi * w.x;
            a.z -= xr * w.z - xi * w.w;
            a.w -= xr * w.w + xi * w.z;
        }
        if (k > 0) *reinterpret_cast<float4*>(wk + off) = a;
        const float nw = a.x * a.x + a.y * a.y + a.z * a.z + a.w * a.w;
        float nr = 0.f;
        if (st.update_r) {
            float4 rv = *reinterpret_cast<const float4*>(r + off);
            rv.x -= st.a.x * a.x - st.a.y * a.y;
            rv.y -= st.a.x * a.y + st.a.y * a.x;
            rv.z -= st.a.x * a.z - st.a.y * a.w;
            rv.w -= st.a.x * a.w + st.a.y * a.z;
            *reinterpret_cast<float4*>(r + off) = rv;
            nr = rv.x * rv.x + rv.y * rv.y + rv.z * rv.z + rv.w * rv.w;
        }
        acc[0] += nr;
        acc[1] += nw;
    }
    block_reduce_finalize<2>(acc, partials, ticket, out);
}

struct GcrCombine {
    float2 beta[GCR_KMAX];
};

// x = sum_{k < m} beta_k z_k
__global__ void gcr_combine_kernel(Geom g, const char* Z, size_t fld, int m, GcrCombine cb, char* x)
{
    const size_t fb = fld / 2;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.Vh; i += gridDim.x * blockDim.x)
        for (int par = 0; par < 2; ++par) {
            float a[24];
#pragma unroll
            for (int q = 0; q < 24; ++q) a[q] = 0.f;
            for (int k = 0; k < m; ++k) {
                float z[24];
                SpinorIO<P32>::load(Z + k * fld + par * fb, g.stride, i, z);
                const float br = cb.beta[k].x, bi = cb.beta[k].y;
#pragma unroll
                for (int q = 0; q < 12; ++q) {
                    a[2 * q] += br * z[2 * q] - bi * z[2 * q + 1];
                    a[2 * q + 1] += br * z[2 * q + 1] + bi * z[2 * q];
                }
            }
            SpinorIO<P32>::store(x + par * fb, g.stride, i, a);
        }
}

namespace {

int gcr_grid(const lqcd_ctx* c, int block)
{
    int nb = (c->g.Vh + block - 1) / block;
    return nb < 2 * 152 ? nb : 2 * 152;
}

}  // namespace

lqcd_status solve_fgcr(lqcd_ctx* c, lqcd_net* net, double* x, const double* b, double tol,
                       const lqcd_solver_params* p, lqcd_solver_stats* st, bool host_io)
{
    const auto t_start = std::chrono::steady_clock::now();
    const int K = p->nkrylov;
    if (K < 1 || K > GCR_KMAX || K > c->cfg.gcr_nkrylov)
        return fail(LQCD_ERR_INVALID, "lqcd_solve: FGCR needs 1 <= nkrylov <= min(24, cfg.gcr_nkrylov)");
    const int mode = p->inner_prec;
    if (mode_ps(mode) != P32) return fail(LQCD_ERR_INVALID, "lqcd_solve: FGCR runs with FP32 vectors (inner_prec F32, F16_LINKS or BF16_LINKS)");
    const bool log = getenv("LQCD_LOG") != nullptr;
    if (p->residual_prec != LQCD_F64) return fail(LQCD_ERR_INVALID, "lqcd_solve: residual_prec must be LQCD_F64");
    const size_t fb64 = c->field_bytes(P64), rb64 = 2 * fb64;
    const size_t fb = c->field_bytes(P32), fld = 2 * fb;
    char* B = vec64_field(c, 0, 0);
    char* X = vec64_field(c, 1, 0);
    char* T1 = vec64_field(c, 2, 0);
    char* T2 = vec64_field(c, 3, 0);
    char* Zb = c->gcr;
    char* Wb = Zb + (size_t)K * fld;
    char* R32 = Wb + (size_t)K * fld;
    char* X32 = R32 + fld;
    double* dev = reinterpret_cast<double*>(X32 + fld);  // scalars of the recursion
    double* dots = dev;                                    // [GCR_NDOT]
    double* upd = dev + 64;                                // [2]
    unsigned* tick = reinterpret_cast<unsigned*>(upd + 4); // [0]: updates, [1 + c]: dot chunk c
    double* parts = reinterpret_cast<double*>(reinterpret_cast<char*>(tick) + 256);
    const size_t canon_rb = (size_t)c->volume * 192;

    c->dslash_count = 0;
    c->launches = 0;
    const double* bdev = b;
    if (host_io) {
        LQ_CUDA(cudaMemcpyAsync(c->staging, b, canon_rb, cudaMemcpyHostToDevice, c->stream));
        bdev = static_cast<const double*>(c->staging);
    }
    LQ_TRY(pack_spinor(c, B, bdev, -1, P64, 1, rb64, canon_rb));
    LQ_CUDA(cudaMemsetAsync(c->scal, 0, SC_PER_RHS * sizeof(double), c->stream));
    LQ_CUDA(cudaMemsetAsync(tick, 0, 64 * sizeof(unsigned), c->stream));
    LQ_TRY(blas_norm2(c, B, P64, 1, rb64, 2, SC_TMP + 0));
    LQ_TRY(blas_zero(c, X, P64, 1, rb64, 2));
    double h[SC_PER_RHS];
    auto read = [&](const double* src, double* dst, int n) -> lqcd_status {
        LQ_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        LQ_CUDA(cudaStreamSynchronize(c->stream));
        return LQCD_OK;
    };
    LQ_TRY(read(c->scal, h, SC_PER_RHS));
    const double bn2 = h[SC_TMP + 0];
    const int block = 256;
    const dim3 grid(gcr_grid(c, block));
    // the elementwise update: one thread per (parity, float4 chunk, site), at most 8 blocks per SM
    const long nupd = (12L * c->g.Vh + block - 1) / block;
    const int gu = (int)(nupd < 8 * 152 ? nupd : 8 * 152);
    bool sap = !net && c->sap_on;
    if (sap) LQ_TRY(sap_check(c, c->sap_bs));
    int iters = 0, restarts = 0, fallback = 0;
    double res = 1.0, res_prev = 0.0;
    lqcd_status status = LQCD_OK;
    typedef std::complex<double> cd;
    std::vector<cd> alpha(K), coef((size_t)K * K);  // coef[j * K + k] = c_jk
    std::vector<double> wn(K);                       // |w^_j|^2
    std::vector<double> hd(GCR_NDOT);
    auto launch_dots = [&](int k, const char* wk) -> lqcd_status {
        const dim3 gd(grid.x, (k + GCR_CH - 1) / GCR_CH + 1);
        gcr_dots_kernel<<<gd, block, 0, c->stream>>>(c->g, Wb, fld, k, wk, R32, parts, tick + 1, dots);
        LQ_CUDA(cudaGetLastError());
        c->launches++;
        return read(dots, hd.data(), GCR_NDOT);
    };
    auto launch_update = [&](int k, char* wk, const cd* cj, cd a, bool update_r, double out[2]) -> lqcd_status {
        GcrStep st;
        memset(&st, 0, sizeof st);
        for (int j = 0; j < k; ++j) st.c[j] = make_float2((float)cj[j].real(), (float)cj[j].imag());
        st.a = make_float2((float)a.real(), (float)a.imag());
        st.update_r = update_r ? 1 : 0;
        gcr_orth_update_kernel<<<gu, block, 0, c->stream>>>(c->g, Wb, fld, k, wk, R32, st, parts, tick, upd);
        LQ_CUDA(cudaGetLastError());
        c->launches++;
        return read(upd, out, 2);
    };
    while (true) {
        // restart: r = b - M x in FP64; stop on the true residual
        LQ_TRY(op_full(c, T1, X, P64, false, 1, rb64));
        LQ_TRY(blas_xmy_norm(c, T2, B, T1, P64, 1, rb64, 2, SC_TMP + 2));
        LQ_TRY(read(c->scal, h, SC_PER_RHS));
        res = bn2 > 0 ? std::sqrt(h[SC_TMP + 2] / bn2) : 0.0;
        if (log) fprintf(stderr, "[lqcd] fgcr iter %d restart, true residual %.3e\n", iters, res);
        if (!std::isfinite(res)) { status = LQCD_ERR_BREAKDOWN; break; }
        if (res <= tol) break;
        // safeguard: a network that does not halve the residual over a whole
        // cycle is replaced by the identity for the rest of the solve (SAP is
        // a fixed convergent splitting and is kept)
        if (net && restarts > 0 && res > 0.5 * res_prev) {
            net = nullptr;
            fallback = 1;
            if (log) fprintf(stderr, "[lqcd] fgcr: preconditioner stagnates, continuing with the identity\n");
        }
        res_prev = res;
        if (iters >= p->maxiter) { status = LQCD_ERR_NOT_CONVERGED; break; }
        restarts++;
        LQ_TRY(convert_field(c, R32, P32, T2, P64, 1, fld, rb64, 2, -1));
        const double r2_cycle = h[SC_TMP + 2];  // |r|^2 at the restart
        int m = 0;  // vectors of this cycle
        for (int k = 0; k < K && iters < p->maxiter; ++k) {
            char* zk = Zb + (size_t)k * fld;
            char* wk = Wb + (size_t)k * fld;
            if (net) LQ_TRY(net_apply_internal(net, zk, R32, fld));
            else if (sap) LQ_TRY(sap_apply(c, zk, R32, c->sap_bs, c->sap_ncycle, c->sap_nmr, vec64_field(c, 4, 0),
                                           vec64_field(c, 5, 0)));
            else LQ_TRY(convert_field(c, zk, P32, R32, P32, 1, fld, fld, 2, -1));
            LQ_TRY(op_full(c, wk, zk, mode, false, 1, fld));
            // classical Gram-Schmidt, a second pass when the first cancels
            std::vector<cd> ck(k, cd(0.0, 0.0)), cj(k);
            double out[2] = {0.0, 0.0};
            cd a(0.0, 0.0);
            double what2 = 0.0, ww0 = 0.0;
            bool used = false;
            for (int pass = 0; pass < 2; ++pass) {
                LQ_TRY(launch_dots(k, wk));
                const double ww = hd[2 * GCR_KMAX + 2];
                if (pass == 0) ww0 = ww;
                what2 = ww;
                for (int j = 0; j < k; ++j) {
                    const cd d(hd[2 * j], hd[2 * j + 1]);
                    cj[j] = d / wn[j];
                    what2 -= std::norm(d) / wn[j];
                }
                const cd wr(hd[2 * GCR_KMAX], hd[2 * GCR_KMAX + 1]);
                // nothing new in w_k (also catches NaN): do not use it
                if (!(what2 > 1e-10 * ww0) || !std::isfinite(ww)) break;
                for (int j = 0; j < k; ++j) ck[j] += cj[j];
                if (pass == 0 && k > 0 && what2 < 0.5 * ww) {
                    LQ_TRY(launch_update(k, wk, cj.data(), cd(0.0, 0.0), false, out));
                    continue;
                }
                a = wr / what2;
                LQ_TRY(launch_update(k, wk, cj.data(), a, true, out));
                used = true;
                break;
            }
            if (!used) {
                // w_k lies in the span of the earlier w_j: end the cycle without it
                if (k == 0) status = LQCD_ERR_BREAKDOWN;
                break;
            }
            if (!std::isfinite(out[0])) { status = LQCD_ERR_BREAKDOWN; break; }
            wn[k] = out[1];
            alpha[k] = a;
            for (int j = 0; j < k; ++j) coef[(size_t)j * K + k] = ck[j];
            m = k + 1;
            ++iters;
            const double r2 = out[0];
            if (log) fprintf(stderr, "[lqcd] fgcr iter %d |r|/|b| %.3e\n", iters, std::sqrt(r2 / bn2));
            if (std::sqrt(r2 / bn2) <= 0.5 * tol) break;
            if (r2 <= GCR_CYCLE_REDUCTION * GCR_CYCLE_REDUCTION * r2_cycle) break;
        }
        if (status != LQCD_OK) break;
        // x += Z U^{-1} a: back substitution with the unit upper triangle
        GcrCombine cb;
        memset(&cb, 0, sizeof cb);
        std::vector<cd> beta(m);
        for (int k = m - 1; k >= 0; --k) {
            cd v = alpha[k];
            for (int j = k + 1; j < m; ++j) v -= coef[(size_t)k * K + j] * beta[j];
            beta[k] = v;
            cb.beta[k] = make_float2((float)v.real(), (float)v.imag());
        }
        gcr_combine_kernel<<<grid, block, 0, c->stream>>>(c->g, Zb, fld, m, cb, X32);
        LQ_CUDA(cudaGetLastError());
        c->launches++;
        LQ_TRY(blas_accumulate_x(c, X, X32, P32, 1, rb64, fld, 2));
    }
    // final true residual (recomputed above at the last restart check) and x
    double* xdev = host_io ? static_cast<double*>(c->staging) : x;
    LQ_TRY(unpack_spinor(c, xdev, X, -1, P64, 1, rb64, canon_rb));
    if (host_io) LQ_CUDA(cudaMemcpyAsync(x, c->staging, canon_rb, cudaMemcpyDeviceToHost, c->stream));
    LQ_CUDA(cudaStreamSynchronize(c->stream));
    st->iterations = iters;
    st->reliable_updates = 0;
    st->restarts = restarts;
    st->dslash_count = c->dslash_count;
    st->kernel_launches = c->launches;
    st->true_residual = res;
    st->preconditioner_fallback = fallback;
    st->precision_fallback = 0;
    st->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    if (status == LQCD_ERR_NOT_CONVERGED) return fail(status, "lqcd_solve: FGCR not converged within maxiter");
    if (status == LQCD_ERR_BREAKDOWN) return fail(status, "lqcd_solve: FGCR breakdown");
    return LQCD_OK;
}

}  // namespace lqcd
