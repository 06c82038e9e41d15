// Flexible GMRES with deflated restarts (FGMRES-DR) on the full
// Wilson-clover operator, right preconditioned (identity, SAP or the
// network).  Sec. 7 of the paper uses it with SAP when the Krylov space
// that fits in memory is too small for FGCR: at a restart it keeps
// approximate eigenvectors of the smallest eigenvalues (Morgan's deflated
// restart) instead of discarding the space.
//
// Recursion in FP32 on full fields: z_j = P(v_j), w = M z_j, classical
// Gram-Schmidt against v_0..v_{nv-1} with a second pass when the first
// cancels (|w^|^2 < |w|^2 / 2), v_nv = w^/|w^|, so that M Z = V Hbar with V
// orthonormal.  The host keeps Hbar in FP64 and solves min |c - Hbar y| by
// Householder reflections added one column at a time.  A cycle ends after
// nkrylov vectors, or once the least-squares residual has fallen by 1e-5 from
// the cycle's start (FP32's resolution), then x += Z y and the residual
// b - M x is recomputed in FP64.
//
// Deflated restart (ndefl = k > 0): the harmonic Ritz pairs of the
// preconditioned operator on span(V), Hbar^H Hbar g = theta Hsq^H g, give
// the k vectors G_k of smallest |theta|; with P_k an orthonormal basis of
// [G_k; 0] and q the residual coefficients c - Hbar y orthogonalised against
// P_k, the kept basis is V <- V P_k, Z <- Z P_k (in place on the device),
// Hbar <- [P_k q]^H Hbar P_k.  The (k+1)-th basis vector is then formed from
// the FP64 residual itself (its part orthogonal to the kept v's), which in
// exact arithmetic is V q; so every cycle restarts from the true residual.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "dense.h"
#include "internal.h"

namespace lqcd {

lqcd_status net_apply_internal(lqcd_net* n, void* z, const void* r, size_t rb);

namespace {

// Dots with the basis in chunks of ARN_CHUNK vectors per blockIdx.y: a thread
// loads at most ARN_CHUNK + 1 fields per site (short chains of loads, many
// blocks), at the cost of |w|^2 formed once per chunk.
enum { ARN_CHUNK = 4, ARN_NV = 2 * ARN_CHUNK + 1, ARN_MAXCH = 32, DEFL_MAX = 16 };
constexpr double CYCLE_REDUCTION = 1e-5;

int arn_grid(const lqcd_ctx* c, int block)
{
    const int nb = (c->g.Vh + block - 1) / block;
    return nb < 2 * 152 ? nb : 2 * 152;
}

}  // namespace

// Dot products of w with a chunk of basis vectors per blockIdx.y:
// out[ch * ARN_NV + 2i, +1] = <V_{ARN_CHUNK ch + i}, w>, out[ch * ARN_NV + 2 ARN_CHUNK] = |w|^2.
__global__ void arn_dots_kernel(Geom g, const char* V, size_t fld, int n, const char* w, double* partials,
                                size_t part_stride, unsigned* tickets, double* out)
{
    const int ch = blockIdx.y;
    const int j0 = ch * ARN_CHUNK;
    const int cnt = min(ARN_CHUNK, n - j0);
    float acc[ARN_NV];
#pragma unroll
    for (int j = 0; j < ARN_NV; ++j) acc[j] = 0.f;
    const size_t fb = fld / 2;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.Vh; i += gridDim.x * blockDim.x)
        for (int par = 0; par < 2; ++par) {
            float wv[24];
            SpinorIO<P32>::load(w + par * fb, g.stride, i, wv);
#pragma unroll
            for (int j = 0; j < ARN_CHUNK; ++j) {
                if (j >= cnt) break;
                float v[24];
                SpinorIO<P32>::load(V + (size_t)(j0 + j) * fld + par * fb, g.stride, i, v);
                float re = 0.f, im = 0.f;
#pragma unroll
                for (int q = 0; q < 12; ++q) {
                    re += v[2 * q] * wv[2 * q] + v[2 * q + 1] * wv[2 * q + 1];
                    im += v[2 * q] * wv[2 * q + 1] - v[2 * q + 1] * wv[2 * q];
                }
                acc[2 * j] += re;
                acc[2 * j + 1] += im;
            }
            float nn = 0.f;
#pragma unroll
            for (int q = 0; q < 24; ++q) nn += wv[q] * wv[q];
            acc[2 * ARN_CHUNK] += nn;
        }
    double d[ARN_NV];
#pragma unroll
    for (int j = 0; j < ARN_NV; ++j) d[j] = acc[j];
    block_reduce_finalize<ARN_NV>(d, partials + ch * part_stride, tickets + ch, out + ch * ARN_NV);
}

// w -= sum_{j < n} coef_j V_j; out[0] = |w|^2 afterwards.
__global__ void arn_update_kernel(Geom g, const char* V, size_t fld, int n, const float2* coef, char* w,
                                  double* partials, unsigned* ticket, double* out)
{
    double acc[1] = {0.0};
    const size_t fb = fld / 2;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.Vh; i += gridDim.x * blockDim.x)
        for (int par = 0; par < 2; ++par) {
            float a[24];
            SpinorIO<P32>::load(w + par * fb, g.stride, i, a);
            for (int j = 0; j < n; ++j) {
                float v[24];
                SpinorIO<P32>::load(V + (size_t)j * fld + par * fb, g.stride, i, v);
                const float2 c = __ldg(coef + j);
#pragma unroll
                for (int q = 0; q < 12; ++q) {
                    a[2 * q] -= c.x * v[2 * q] - c.y * v[2 * q + 1];
                    a[2 * q + 1] -= c.x * v[2 * q + 1] + c.y * v[2 * q];
                }
            }
            SpinorIO<P32>::store(w + par * fb, g.stride, i, a);
            float nn = 0.f;
#pragma unroll
            for (int q = 0; q < 24; ++q) nn += a[q] * a[q];
            acc[0] += nn;
        }
    block_reduce_finalize<1>(acc, partials, ticket, out);
}

__global__ void arn_scale_kernel(Geom g, char* v, size_t fld, float s)
{
    const size_t fb = fld / 2;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.Vh; i += gridDim.x * blockDim.x)
        for (int par = 0; par < 2; ++par) {
            float a[24];
            SpinorIO<P32>::load(v + par * fb, g.stride, i, a);
#pragma unroll
            for (int q = 0; q < 24; ++q) a[q] *= s;
            SpinorIO<P32>::store(v + par * fb, g.stride, i, a);
        }
}

// out_l = sum_{j < n} in_j P[j + l n] for l < kout (fields fld bytes apart).
// One thread per float4 of a field (two complex numbers); in place (out ==
// in) is safe: a thread reads all its inputs before writing its outputs.
template <int KO>
__global__ void arn_lincomb_kernel(Geom g, char* out, const char* in, size_t fld, int n, int kout, const float2* P)
{
    const size_t fb = fld / 2;
    const long per_par = 6L * g.stride;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < 2 * per_par; e += (long)gridDim.x * blockDim.x) {
        const int par = (int)(e / per_par);
        const long r = e - par * per_par;
        if ((int)(r % g.stride) >= g.Vh) continue;  // padding sites
        const size_t off = par * fb + (size_t)r * sizeof(float4);
        float2 acc[KO][2];
#pragma unroll
        for (int l = 0; l < KO; ++l) acc[l][0] = acc[l][1] = make_float2(0.f, 0.f);
        for (int j = 0; j < n; ++j) {
            const float4 v = *reinterpret_cast<const float4*>(in + (size_t)j * fld + off);
#pragma unroll
            for (int l = 0; l < KO; ++l) {
                if (l >= kout) break;
                const float2 c = __ldg(P + j + (size_t)l * n);
                acc[l][0].x += c.x * v.x - c.y * v.y;
                acc[l][0].y += c.x * v.y + c.y * v.x;
                acc[l][1].x += c.x * v.z - c.y * v.w;
                acc[l][1].y += c.x * v.w + c.y * v.z;
            }
        }
#pragma unroll
        for (int l = 0; l < KO; ++l) {
            if (l >= kout) break;
            *reinterpret_cast<float4*>(out + (size_t)l * fld + off) =
                make_float4(acc[l][0].x, acc[l][0].y, acc[l][1].x, acc[l][1].y);
        }
    }
}

lqcd_status solve_fgmres_dr(lqcd_ctx* c, lqcd_net* net, double* x, const double* b, double tol,
                            const lqcd_solver_params* p, lqcd_solver_stats* st, bool host_io)
{
    typedef dense::cd cd;
    const auto t_start = std::chrono::steady_clock::now();
    const int m = p->nkrylov, k = p->ndefl;
    if (m < 2 || m > c->cfg.gcr_nkrylov || m + 1 > ARN_CHUNK * ARN_MAXCH)
        return fail(LQCD_ERR_INVALID, "lqcd_solve: FGMRES-DR needs 2 <= nkrylov <= cfg.gcr_nkrylov");
    if (k < 0 || k > DEFL_MAX || k >= m) return fail(LQCD_ERR_INVALID, "lqcd_solve: FGMRES-DR needs 0 <= ndefl <= 16, < nkrylov");
    const int mode = p->inner_prec;
    if (mode_ps(mode) != P32)
        return fail(LQCD_ERR_INVALID, "lqcd_solve: FGMRES-DR runs with FP32 vectors (inner_prec F32, F16_LINKS or BF16_LINKS)");
    if (p->residual_prec != LQCD_F64) return fail(LQCD_ERR_INVALID, "lqcd_solve: residual_prec must be LQCD_F64");
    const bool log = getenv("LQCD_LOG") != nullptr;
    const size_t fb64 = c->field_bytes(P64), rb64 = 2 * fb64;
    const size_t fb = c->field_bytes(P32), fld = 2 * fb;
    char* B = vec64_field(c, 0, 0);
    char* X = vec64_field(c, 1, 0);
    char* T1 = vec64_field(c, 2, 0);
    char* T2 = vec64_field(c, 3, 0);
    char* Vb = c->gcr;                         // m + 1 basis vectors
    char* Zb = Vb + (size_t)(m + 1) * fld;     // m preconditioned vectors
    char* R32 = Zb + (size_t)m * fld;
    char* X32 = R32 + fld;
    char* sc = X32 + fld;                       // scalars
    double* dots = reinterpret_cast<double*>(sc);                   // [ARN_MAXCH * ARN_NV]
    double* upd = dots + ARN_MAXCH * ARN_NV;                         // [4]
    unsigned* tick = reinterpret_cast<unsigned*>(upd + 4);          // [ARN_MAXCH + 1]
    float2* coef = reinterpret_cast<float2*>(sc + 16384);           // [(m + 1) * DEFL_MAX]
    double* parts = reinterpret_cast<double*>(sc + 65536);
    const int block = 256;
    const int gx = arn_grid(c, block);
    const size_t part_stride = (size_t)gx * ARN_NV;
    if (65536 + part_stride * ARN_MAXCH * sizeof(double) > GCR_SCALAR_BYTES)
        return fail(LQCD_ERR_NOMEM, "lqcd_solve: FGMRES-DR scalar area too small");
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
    LQ_CUDA(cudaMemsetAsync(tick, 0, (ARN_MAXCH + 1) * sizeof(unsigned), c->stream));
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
    const double bn = std::sqrt(bn2);
    bool sap = !net && c->sap_on;
    if (sap) LQ_TRY(sap_check(c, c->sap_bs));

    auto vec = [&](int j) { return Vb + (size_t)j * fld; };
    auto zvec = [&](int j) { return Zb + (size_t)j * fld; };
    std::vector<double> hd((size_t)ARN_MAXCH * ARN_NV);
    // dots of w with V_0..V_{n-1} (and |w|^2): d[j], ww
    auto launch_dots = [&](int n, const char* w, std::vector<cd>& d, double& ww) -> lqcd_status {
        const int nch = n > 0 ? (n + ARN_CHUNK - 1) / ARN_CHUNK : 1;
        arn_dots_kernel<<<dim3(gx, nch), block, 0, c->stream>>>(c->g, Vb, fld, n, w, parts, part_stride, tick, dots);
        LQ_CUDA(cudaGetLastError());
        c->launches++;
        LQ_TRY(read(dots, hd.data(), nch * ARN_NV));
        d.assign(n, cd(0.0, 0.0));
        for (int j = 0; j < n; ++j) {
            const int ch = j / ARN_CHUNK, i = j % ARN_CHUNK;
            d[j] = cd(hd[ch * ARN_NV + 2 * i], hd[ch * ARN_NV + 2 * i + 1]);
        }
        ww = hd[2 * ARN_CHUNK];
        return LQCD_OK;
    };
    std::vector<float2> hcoef;
    auto upload = [&](const std::vector<float2>& v) -> lqcd_status {
        LQ_CUDA(cudaMemcpyAsync(coef, v.data(), v.size() * sizeof(float2), cudaMemcpyHostToDevice, c->stream));
        return LQCD_OK;
    };
    // w -= sum_j d_j V_j; returns |w|^2
    auto launch_update = [&](int n, char* w, const std::vector<cd>& d, double& nw2) -> lqcd_status {
        hcoef.resize(n > 0 ? n : 1);
        for (int j = 0; j < n; ++j) hcoef[j] = make_float2((float)d[j].real(), (float)d[j].imag());
        LQ_TRY(upload(hcoef));
        arn_update_kernel<<<gx, block, 0, c->stream>>>(c->g, Vb, fld, n, coef, w, parts, tick + ARN_MAXCH, upd);
        LQ_CUDA(cudaGetLastError());
        c->launches++;
        double o[1];
        LQ_TRY(read(upd, o, 1));
        nw2 = o[0];
        return LQCD_OK;
    };
    // orthogonalise w (slot of V_n) against V_0..V_{n-1}: coefficients h, |w^|
    auto orthogonalise = [&](int n, char* w, std::vector<cd>& hcol, double& wnorm) -> lqcd_status {
        std::vector<cd> d;
        double ww = 0.0, nw2 = 0.0;
        LQ_TRY(launch_dots(n, w, d, ww));
        hcol = d;
        LQ_TRY(launch_update(n, w, d, nw2));
        if (n > 0 && nw2 < 0.5 * ww) {  // cancellation: a second pass
            double ww2 = 0.0;
            LQ_TRY(launch_dots(n, w, d, ww2));
            for (int j = 0; j < n; ++j) hcol[j] += d[j];
            LQ_TRY(launch_update(n, w, d, nw2));
        }
        wnorm = std::sqrt(nw2);
        return LQCD_OK;
    };
    auto scale = [&](char* v, double s) -> lqcd_status {
        arn_scale_kernel<<<gx, block, 0, c->stream>>>(c->g, v, fld, (float)s);
        LQ_CUDA(cudaGetLastError());
        c->launches++;
        return LQCD_OK;
    };
    auto lincomb = [&](char* out, const char* in, int n, int kout, const std::vector<cd>& P) -> lqcd_status {
        hcoef.resize((size_t)n * kout);
        for (size_t i = 0; i < hcoef.size(); ++i) hcoef[i] = make_float2((float)P[i].real(), (float)P[i].imag());
        LQ_TRY(upload(hcoef));
        const long elems = 2L * 6 * c->g.stride;
        const int grid = (int)std::min<long>((elems + 255) / 256, 4L * 152 * 8);
        if (kout == 1)
            arn_lincomb_kernel<1><<<grid, 256, 0, c->stream>>>(c->g, out, in, fld, n, kout, coef);
        else
            arn_lincomb_kernel<DEFL_MAX><<<grid, 256, 0, c->stream>>>(c->g, out, in, fld, n, kout, coef);
        LQ_CUDA(cudaGetLastError());
        c->launches++;
        return LQCD_OK;
    };

    const int ldh = m + 1;
    std::vector<cd> H((size_t)ldh * m), cvec(ldh);
    std::vector<cd> Hdefl;  // (k + 1) x k block kept by the last deflated restart
    bool have_defl = false;
    dense::Lsq ls;
    int iters = 0, restarts = 0, fallback = 0;
    double res = 1.0, res_prev = 0.0;
    lqcd_status status = LQCD_OK;
    while (true) {
        // FP64 residual of the current x; convergence on it
        LQ_TRY(op_full(c, T1, X, P64, false, 1, rb64));
        LQ_TRY(blas_xmy_norm(c, T2, B, T1, P64, 1, rb64, 2, SC_TMP + 2));
        LQ_TRY(read(c->scal, h, SC_PER_RHS));
        res = bn2 > 0 ? std::sqrt(h[SC_TMP + 2] / bn2) : 0.0;
        if (log) fprintf(stderr, "[lqcd] fgmres-dr iter %d restart, true residual %.3e\n", iters, res);
        if (!std::isfinite(res)) { status = LQCD_ERR_BREAKDOWN; break; }
        if (res <= tol) break;
        if (net && restarts > 0 && res > 0.5 * res_prev) {  // the network stagnates: identity from here
            net = nullptr;
            fallback = 1;
            have_defl = false;
        }
        res_prev = res;
        if (iters >= p->maxiter) { status = LQCD_ERR_NOT_CONVERGED; break; }
        restarts++;
        LQ_TRY(convert_field(c, R32, P32, T2, P64, 1, fld, rb64, 2, -1));
        std::fill(H.begin(), H.end(), cd(0.0, 0.0));
        std::fill(cvec.begin(), cvec.end(), cd(0.0, 0.0));
        int nz = 0, nv = 0;
        double rcycle = 0.0;
        if (have_defl) {
            // kept: V_0..V_{k-1}, Z_0..Z_{k-1}, Hbar (k+1) x k; v_k from the residual
            LQ_TRY(convert_field(c, vec(k), P32, R32, P32, 1, fld, fld, 2, -1));
            std::vector<cd> d;
            double vn = 0.0;
            LQ_TRY(orthogonalise(k, vec(k), d, vn));
            if (!(vn > 0.0) || !std::isfinite(vn)) { status = LQCD_ERR_BREAKDOWN; break; }
            LQ_TRY(scale(vec(k), 1.0 / vn));
            for (int j = 0; j < k; ++j) cvec[j] = d[j];
            cvec[k] = vn;
            for (int jj = 0; jj < k; ++jj)
                for (int i = 0; i <= k; ++i) H[i + (size_t)jj * ldh] = Hdefl[i + (size_t)jj * (k + 1)];
            nz = k;
            nv = k + 1;
            rcycle = std::sqrt(h[SC_TMP + 2]);
        } else {
            const double rn = std::sqrt(h[SC_TMP + 2]);
            LQ_TRY(convert_field(c, vec(0), P32, R32, P32, 1, fld, fld, 2, -1));
            LQ_TRY(scale(vec(0), 1.0 / rn));
            cvec[0] = rn;
            nz = 0;
            nv = 1;
            rcycle = rn;
        }
        ls.reset(cvec.data(), nv);
        for (int jj = 0; jj < nz; ++jj) ls.add_column(&H[(size_t)jj * ldh], nv);
        bool lucky = false;
        while (nz < m && iters < p->maxiter) {
            const int j = nz;
            char* zj = zvec(j);
            char* w = vec(nv);
            if (net) LQ_TRY(net_apply_internal(net, zj, vec(j), fld));
            else if (sap) LQ_TRY(sap_apply(c, zj, vec(j), c->sap_bs, c->sap_ncycle, c->sap_nmr, vec64_field(c, 4, 0),
                                           vec64_field(c, 5, 0)));
            else LQ_TRY(convert_field(c, zj, P32, vec(j), P32, 1, fld, fld, 2, -1));
            LQ_TRY(op_full(c, w, zj, mode, false, 1, fld));
            std::vector<cd> hcol;
            double wn = 0.0;
            LQ_TRY(orthogonalise(nv, w, hcol, wn));
            if (!std::isfinite(wn)) { status = LQCD_ERR_BREAKDOWN; break; }
            for (int i = 0; i < nv; ++i) H[i + (size_t)j * ldh] = hcol[i];
            H[nv + (size_t)j * ldh] = wn;
            ls.add_column(&H[(size_t)j * ldh], nv + 1);
            ++nz;
            ++iters;
            double hn = 0.0;
            for (int i = 0; i < nv; ++i) hn += std::norm(hcol[i]);
            if (!(wn > 1e-10 * std::sqrt(hn + wn * wn))) {  // invariant subspace: the solution is in it
                lucky = true;
                ++nv;
                break;
            }
            LQ_TRY(scale(w, 1.0 / wn));
            ++nv;
            const double est = ls.residual();
            if (log) fprintf(stderr, "[lqcd] fgmres-dr iter %d |r|/|b| %.3e\n", iters, est / bn);
            if (est <= 0.5 * tol * bn || est <= CYCLE_REDUCTION * rcycle) break;
        }
        if (status != LQCD_OK) break;
        // x += Z y
        const std::vector<cd> y = ls.solve();
        LQ_TRY(lincomb(X32, Zb, nz, 1, y));
        LQ_TRY(blas_accumulate_x(c, X, X32, P32, 1, rb64, fld, 2));
        // deflated restart: keep the k harmonic Ritz vectors of smallest |theta|
        have_defl = false;
        if (k > 0 && nz > k && !lucky && nv == nz + 1) {
            std::vector<cd> theta(k), G((size_t)nz * k);
            if (dense::harmonic_ritz(nz, H.data(), ldh, k, theta.data(), G.data())) {
                const int rows = nz + 1;
                std::vector<cd> Pk((size_t)rows * (k + 1), cd(0.0, 0.0));  // [P_k q]
                for (int jj = 0; jj < k; ++jj)
                    for (int i = 0; i < nz; ++i) Pk[i + (size_t)jj * rows] = G[i + (size_t)jj * nz];
                std::vector<cd> cls(rows);
                for (int i = 0; i < rows; ++i) {
                    cd s = cvec[i];
                    for (int jj = 0; jj < nz; ++jj) s -= H[i + (size_t)jj * ldh] * y[jj];
                    cls[i] = s;
                }
                for (int i = 0; i < rows; ++i) Pk[i + (size_t)k * rows] = cls[i];
                dense::orthonormalize(rows, k + 1, Pk.data(), rows);
                // Hdefl = [P_k q]^H Hbar P_k[:nz]
                std::vector<cd> HP((size_t)rows * k, cd(0.0, 0.0));
                for (int jj = 0; jj < k; ++jj)
                    for (int i = 0; i < rows; ++i) {
                        cd s(0.0, 0.0);
                        for (int l = 0; l < nz; ++l) s += H[i + (size_t)l * ldh] * Pk[l + (size_t)jj * rows];
                        HP[i + (size_t)jj * rows] = s;
                    }
                Hdefl.assign((size_t)(k + 1) * k, cd(0.0, 0.0));
                for (int jj = 0; jj < k; ++jj)
                    for (int a = 0; a <= k; ++a) {
                        cd s(0.0, 0.0);
                        for (int i = 0; i < rows; ++i) s += std::conj(Pk[i + (size_t)a * rows]) * HP[i + (size_t)jj * rows];
                        Hdefl[a + (size_t)jj * (k + 1)] = s;
                    }
                // V_0..V_{k-1} <- V P_k, Z_0..Z_{k-1} <- Z P_k[:nz], in place
                std::vector<cd> Pv((size_t)rows * k), Pz((size_t)nz * k);
                for (int jj = 0; jj < k; ++jj) {
                    for (int i = 0; i < rows; ++i) Pv[i + (size_t)jj * rows] = Pk[i + (size_t)jj * rows];
                    for (int i = 0; i < nz; ++i) Pz[i + (size_t)jj * nz] = Pk[i + (size_t)jj * rows];
                }
                LQ_TRY(lincomb(Vb, Vb, rows, k, Pv));
                LQ_TRY(lincomb(Zb, Zb, nz, k, Pz));
                have_defl = true;
            } else if (log) {
                fprintf(stderr, "[lqcd] fgmres-dr: harmonic Ritz step failed, plain restart\n");
            }
        }
    }
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
    if (status == LQCD_ERR_NOT_CONVERGED) return fail(status, "lqcd_solve: FGMRES-DR not converged within maxiter");
    if (status == LQCD_ERR_BREAKDOWN) return fail(status, "lqcd_solve: FGMRES-DR breakdown");
    return LQCD_OK;
}

}  // namespace lqcd
