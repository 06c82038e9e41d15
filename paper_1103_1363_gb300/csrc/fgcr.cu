// Flexible GCR(k) on the full Wilson-clover operator with a right
// preconditioner (identity, SAP or the parallel-transport network).
//
// The paper's outer solver is FGCR: it stores two vectors per iteration
// (z_k and w_k = M z_k), so it is restarted, and it tolerates a
// preconditioner that is not a fixed operator; mixed precision is
// iterative refinement, i.e. the recursion runs in single precision and the
// residual is recomputed in double precision at each restart (Sec. 5).
// Here w_k is orthogonalised against the earlier w_j by classical
// Gram-Schmidt applied twice (the same coefficients update z_k), which in
// exact arithmetic gives the same iterates as modified Gram-Schmidt but
// needs two fused launches per pass instead of 2k.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "internal.h"

namespace lqcd {

lqcd_status net_apply_internal(lqcd_net* n, void* z, const void* r, size_t rb);

enum { GCR_KMAX = 24 };

// dots[j] = <w_j, v> (j < k), complex, FP64 accumulation.
__global__ void gcr_multidot_kernel(Geom g, const char* W, size_t fld, int k, const char* v, double* partials,
                                    unsigned* ticket, double* out)
{
    double acc[2 * GCR_KMAX];
#pragma unroll
    for (int j = 0; j < 2 * GCR_KMAX; ++j) acc[j] = 0.0;
    const size_t fb = fld / 2;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.Vh; i += gridDim.x * blockDim.x)
        for (int par = 0; par < 2; ++par) {
            float vv[24];
            SpinorIO<P32>::load(v + par * fb, g.stride, i, vv);
#pragma unroll
            for (int j = 0; j < GCR_KMAX; ++j) {
                if (j >= k) break;
                float w[24];
                SpinorIO<P32>::load(W + j * fld + par * fb, g.stride, i, w);
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
    block_reduce_finalize<2 * GCR_KMAX>(acc, partials, ticket, out);
}

// w_k -= sum_j c_j w_j, z_k -= sum_j c_j z_j with c_j = dots[j] / wnorm[j].
__global__ void gcr_multiaxpy_kernel(Geom g, const char* W, const char* Z, size_t fld, int k, char* wk, char* zk,
                                     const double* dots, const double* wnorm)
{
    __shared__ float cr[GCR_KMAX], ci[GCR_KMAX];
    if (threadIdx.x < k) {
        cr[threadIdx.x] = (float)(dots[2 * threadIdx.x] / wnorm[threadIdx.x]);
        ci[threadIdx.x] = (float)(dots[2 * threadIdx.x + 1] / wnorm[threadIdx.x]);
    }
    __syncthreads();
    const size_t fb = fld / 2;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.Vh; i += gridDim.x * blockDim.x)
        for (int par = 0; par < 2; ++par) {
            float a[24], b[24];
            SpinorIO<P32>::load(wk + par * fb, g.stride, i, a);
            SpinorIO<P32>::load(zk + par * fb, g.stride, i, b);
            for (int j = 0; j < k; ++j) {
                float w[24], z[24];
                SpinorIO<P32>::load(W + j * fld + par * fb, g.stride, i, w);
                SpinorIO<P32>::load(Z + j * fld + par * fb, g.stride, i, z);
                const float xr = cr[j], xi = ci[j];
#pragma unroll
                for (int q = 0; q < 12; ++q) {
                    a[2 * q] -= xr * w[2 * q] - xi * w[2 * q + 1];
                    a[2 * q + 1] -= xr * w[2 * q + 1] + xi * w[2 * q];
                    b[2 * q] -= xr * z[2 * q] - xi * z[2 * q + 1];
                    b[2 * q + 1] -= xr * z[2 * q + 1] + xi * z[2 * q];
                }
            }
            SpinorIO<P32>::store(wk + par * fb, g.stride, i, a);
            SpinorIO<P32>::store(zk + par * fb, g.stride, i, b);
        }
}

// out[0..1] = <w, r>, out[2] = |w|^2
__global__ void gcr_dot3_kernel(Geom g, const char* w, const char* r, size_t fb, double* partials, unsigned* ticket,
                                double* out)
{
    double acc[3] = {0.0, 0.0, 0.0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.Vh; i += gridDim.x * blockDim.x)
        for (int par = 0; par < 2; ++par) {
            float a[24], b[24];
            SpinorIO<P32>::load(w + par * fb, g.stride, i, a);
            SpinorIO<P32>::load(r + par * fb, g.stride, i, b);
            float re = 0.f, im = 0.f, nn = 0.f;
#pragma unroll
            for (int q = 0; q < 12; ++q) {
                re += a[2 * q] * b[2 * q] + a[2 * q + 1] * b[2 * q + 1];
                im += a[2 * q] * b[2 * q + 1] - a[2 * q + 1] * b[2 * q];
                nn += a[2 * q] * a[2 * q] + a[2 * q + 1] * a[2 * q + 1];
            }
            acc[0] += re;
            acc[1] += im;
            acc[2] += nn;
        }
    block_reduce_finalize<3>(acc, partials, ticket, out);
}

// x += a z, r -= a w with a = d3[0..1] / d3[2]; |r|^2 -> out; wnorm_k = d3[2]
__global__ void gcr_update_kernel(Geom g, char* x, char* r, const char* z, const char* w, size_t fb, const double* d3,
                                  double* wnorm_k, double* partials, unsigned* ticket, double* out)
{
    const float ar = (float)(d3[0] / d3[2]), ai = (float)(d3[1] / d3[2]);
    if (blockIdx.x == 0 && threadIdx.x == 0) *wnorm_k = d3[2];
    double acc[1] = {0.0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.Vh; i += gridDim.x * blockDim.x)
        for (int par = 0; par < 2; ++par) {
            float xv[24], rv[24], zv[24], wv[24];
            SpinorIO<P32>::load(x + par * fb, g.stride, i, xv);
            SpinorIO<P32>::load(r + par * fb, g.stride, i, rv);
            SpinorIO<P32>::load(z + par * fb, g.stride, i, zv);
            SpinorIO<P32>::load(w + par * fb, g.stride, i, wv);
            float nn = 0.f;
#pragma unroll
            for (int q = 0; q < 12; ++q) {
                xv[2 * q] += ar * zv[2 * q] - ai * zv[2 * q + 1];
                xv[2 * q + 1] += ar * zv[2 * q + 1] + ai * zv[2 * q];
                rv[2 * q] -= ar * wv[2 * q] - ai * wv[2 * q + 1];
                rv[2 * q + 1] -= ar * wv[2 * q + 1] + ai * wv[2 * q];
                nn += rv[2 * q] * rv[2 * q] + rv[2 * q + 1] * rv[2 * q + 1];
            }
            acc[0] += nn;
            SpinorIO<P32>::store(x + par * fb, g.stride, i, xv);
            SpinorIO<P32>::store(r + par * fb, g.stride, i, rv);
        }
    block_reduce_finalize<1>(acc, partials, ticket, out);
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
    if (p->residual_prec != LQCD_F64 && p->residual_prec != LQCD_F64_DF)
        return fail(LQCD_ERR_INVALID, "lqcd_solve: residual_prec must be LQCD_F64 or LQCD_F64_DF");
    const int pres = p->residual_prec;
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
    double* dots = dev;                                    // [2 GCR_KMAX]
    double* wnorm = dev + 2 * GCR_KMAX;                    // [GCR_KMAX]
    double* d3 = wnorm + GCR_KMAX;                         // [3]
    double* rr = d3 + 4;                                   // [1]
    unsigned* tick = reinterpret_cast<unsigned*>(rr + 4);  // [1]
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
    LQ_CUDA(cudaMemsetAsync(tick, 0, sizeof(unsigned), c->stream));
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
    bool sap = !net && c->sap_on;
    if (sap) LQ_TRY(sap_check(c, c->sap_bs));
    int iters = 0, restarts = 0, fallback = 0;
    double res = 1.0, res_prev = 0.0;
    lqcd_status status = LQCD_OK;
    while (true) {
        // restart: r = b - M x with FP64 accuracy; stop on the true residual,
        // confirmed with native FP64 arithmetic when double-float was used
        LQ_TRY(op_full(c, T1, X, pres, false, 1, rb64));
        LQ_TRY(blas_xmy_norm(c, T2, B, T1, P64, 1, rb64, 2, SC_TMP + 2));
        LQ_TRY(read(c->scal, h, SC_PER_RHS));
        res = bn2 > 0 ? std::sqrt(h[SC_TMP + 2] / bn2) : 0.0;
        if (res <= tol && pres != P64) {
            LQ_TRY(op_full(c, T1, X, P64, false, 1, rb64));
            LQ_TRY(blas_xmy_norm(c, T2, B, T1, P64, 1, rb64, 2, SC_TMP + 2));
            LQ_TRY(read(c->scal, h, SC_PER_RHS));
            res = bn2 > 0 ? std::sqrt(h[SC_TMP + 2] / bn2) : 0.0;
        }
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
        LQ_TRY(blas_zero(c, X32, P32, 1, fld, 2));
        for (int k = 0; k < K && iters < p->maxiter; ++k) {
            char* zk = Zb + (size_t)k * fld;
            char* wk = Wb + (size_t)k * fld;
            if (net) LQ_TRY(net_apply_internal(net, zk, R32, fld));
            else if (sap) LQ_TRY(sap_apply(c, zk, R32, c->sap_bs, c->sap_ncycle, c->sap_nmr, vec64_field(c, 4, 0),
                                           vec64_field(c, 5, 0)));
            else LQ_TRY(convert_field(c, zk, P32, R32, P32, 1, fld, fld, 2, -1));
            LQ_TRY(op_full(c, wk, zk, mode, false, 1, fld));
            for (int pass = 0; pass < 2 && k > 0; ++pass) {
                gcr_multidot_kernel<<<grid, block, 0, c->stream>>>(c->g, Wb, fld, k, wk, parts, tick, dots);
                LQ_CUDA(cudaGetLastError());
                gcr_multiaxpy_kernel<<<grid, block, 0, c->stream>>>(c->g, Wb, Zb, fld, k, wk, zk, dots, wnorm);
                LQ_CUDA(cudaGetLastError());
                c->launches += 2;
            }
            gcr_dot3_kernel<<<grid, block, 0, c->stream>>>(c->g, wk, R32, fb, parts, tick, d3);
            LQ_CUDA(cudaGetLastError());
            gcr_update_kernel<<<grid, block, 0, c->stream>>>(c->g, X32, R32, zk, wk, fb, d3, wnorm + k, parts, tick, rr);
            LQ_CUDA(cudaGetLastError());
            c->launches += 2;
            ++iters;
            double r2 = 0.0;
            LQ_TRY(read(rr, &r2, 1));
            if (log) fprintf(stderr, "[lqcd] fgcr iter %d |r|/|b| %.3e\n", iters, std::sqrt(r2 / bn2));
            if (!std::isfinite(r2)) { status = LQCD_ERR_BREAKDOWN; break; }
            if (std::sqrt(r2 / bn2) <= 0.5 * tol) break;
        }
        if (status != LQCD_OK) break;
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
    st->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    if (status == LQCD_ERR_NOT_CONVERGED) return fail(status, "lqcd_solve: FGCR not converged within maxiter");
    if (status == LQCD_ERR_BREAKDOWN) return fail(status, "lqcd_solve: FGCR breakdown");
    return LQCD_OK;
}

}  // namespace lqcd
