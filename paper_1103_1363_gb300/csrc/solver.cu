// Krylov solvers: CG on the normal equations of the even-odd Schur
// complement (or of the full operator), in FP64 or in a lower inner
// precision with FP64 reliable updates.
//
// The paper solves M phi = b with CG on M^dag M and on the Schur
// complement of the even-odd split (Sec. 5), and does mixed precision by
// iterative refinement: the cheap recursion runs in single precision and
// the residual is recomputed in double precision at restarts (Sec. 5,
// FGCR paragraph).  Here the inner recursion (FP32, FP16 or BF16 storage,
// FP32 arithmetic) is a CG whose residual is replaced by the FP64 true
// residual of the normal equations every `reliable_interval` iterations
// (or when it has dropped by `reliable_delta`), with the low-precision
// solution folded into the FP64 one at each replacement.
//
// Iterations run in blocks of `check_interval`.  A block reads and writes
// only block-relative scalar slots on the device (alpha, beta never leave
// the GPU), so it can be captured once as a CUDA graph and replayed; the
// host reads |r|^2 once per block to decide convergence and replacements.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "internal.h"

namespace lqcd {

namespace {

struct Cg {
    lqcd_ctx* c;
    int R;          // right-hand sides
    int Pi, PA;     // inner storage precision, accumulation precision
    bool eo;
    size_t fb64, rb64, fbi, rbi, fba, rba;
    char *B, *X, *T1, *BH, *RH, *T2;  // FP64 full fields (rhs stride rb64)
    char *Pv, *Qv;                    // inner precision full fields (rhs stride rbi)
    char *XLO, *RV;                   // accumulation precision full fields (rhs stride rba)
    int nf;                           // 1 (odd parity only) or 2 (full lattice)
    size_t o64, oi, oa;               // byte offset of the solved parity in each field
    long reliable = 0, checks = 0;
};

const void* clov_or_null(lqcd_ctx* c, int P, int parity, bool inverse)
{
    if (c->csw == 0.0) return nullptr;
    const int pg = mode_pg(P);
    const char* base = static_cast<const char*>(inverse ? c->clovinv[pg] : c->clov[pg]);
    return base + parity * c->clov_parity_bytes(pg);
}

// One inner CG iteration j of a block: q = K p, x += alpha p, r -= alpha K^dag q
// with K = Mhat (eo) or M (full), |r|^2 into block slot j + 1.
lqcd_status cg_iteration(Cg& s, int j)
{
    lqcd_ctx* c = s.c;
    const int P = s.Pi;
    if (s.eo) {
        // D1: t_e = A_ee^{-1} H_eo p_o
        DslashArgs A = base_args(c, P);
        A.skip = c->skip;
        A.par = 0;
        A.out = s.Qv;
        A.out_rb = s.rbi;
        A.in = s.Pv + s.fbi;
        A.in_rb = s.rbi;
        A.clov = clov_or_null(c, P, 0, true);
        A.a = 1.0;
        LQ_TRY(launch_dslash(c, A, P, false, EPI_CLOVINV, false, s.R));
        // D2: q_o = A_oo p_o - kappa^2 H_oe t_e, |q|^2 -> pap slot j
        DslashArgs B = base_args(c, P);
        B.skip = c->skip;
        B.par = 1;
        B.out = s.Qv + s.fbi;
        B.out_rb = s.rbi;
        B.in = s.Qv;
        B.in_rb = s.rbi;
        B.clov = clov_or_null(c, P, 1, false);
        B.y = s.Pv + s.fbi;
        B.y_rb = s.rbi;
        B.a = -c->kappa * c->kappa;
        B.red = c->scal + pap_slot(j) + 1;
        LQ_TRY(launch_dslash(c, B, P, false, EPI_XPAY, true, s.R));
        // D3: t_e = A_ee^{-1} H_eo^dag q_o
        A.in = s.Qv + s.fbi;
        LQ_TRY(launch_dslash(c, A, P, true, EPI_CLOVINV, false, s.R));
        // D4: s = A_oo q_o - kappa^2 H_oe^dag t_e; x += alpha p; r -= alpha s
        DslashArgs D = base_args(c, P);
        D.skip = c->skip;
        D.par = 1;
        D.in = s.Qv;
        D.in_rb = s.rbi;
        D.clov = clov_or_null(c, P, 1, false);
        D.y = s.Qv + s.fbi;
        D.y_rb = s.rbi;
        D.a = -c->kappa * c->kappa;
        D.x = s.XLO + s.fba;
        D.r = s.RV + s.fba;
        D.acc_rb = s.rba;
        D.p = s.Pv + s.fbi;
        D.p_rb = s.rbi;
        D.s_num = rr_slot(j);
        D.s_num2 = rr_slot(j) + 1;
        D.s_den = pap_slot(j);
        D.s_den2 = pap_slot(j) + 1;
        D.red = c->scal + rr_slot(j + 1) + 1;
        LQ_TRY(launch_dslash(c, D, P, true, EPI_CG, true, s.R));
    } else {
        // q = M p on both parities, |q|^2 per parity -> pap slot j (+0, +1)
        for (int par = 0; par < 2; ++par) {
            DslashArgs A = base_args(c, P);
            A.skip = c->skip;
            A.par = par;
            A.out = s.Qv + par * s.fbi;
            A.out_rb = s.rbi;
            A.in = s.Pv + (1 - par) * s.fbi;
            A.in_rb = s.rbi;
            A.clov = clov_or_null(c, P, par, false);
            A.y = s.Pv + par * s.fbi;
            A.y_rb = s.rbi;
            A.a = -c->kappa;
            A.red = c->scal + pap_slot(j) + par;
            LQ_TRY(launch_dslash(c, A, P, false, EPI_XPAY, true, s.R));
        }
        // s = M^dag q fused with the x, r update, |r|^2 per parity -> rr slot j + 1
        for (int par = 0; par < 2; ++par) {
            DslashArgs D = base_args(c, P);
            D.skip = c->skip;
            D.par = par;
            D.in = s.Qv + (1 - par) * s.fbi;
            D.in_rb = s.rbi;
            D.clov = clov_or_null(c, P, par, false);
            D.y = s.Qv + par * s.fbi;
            D.y_rb = s.rbi;
            D.a = -c->kappa;
            D.x = s.XLO + par * s.fba;
            D.r = s.RV + par * s.fba;
            D.acc_rb = s.rba;
            D.p = s.Pv + par * s.fbi;
            D.p_rb = s.rbi;
            D.s_num = rr_slot(j);
            D.s_num2 = rr_slot(j) + 1;
            D.s_den = pap_slot(j);
            D.s_den2 = pap_slot(j) + 1;
            D.red = c->scal + rr_slot(j + 1) + par;
            LQ_TRY(launch_dslash(c, D, P, true, EPI_CG, true, s.R));
        }
    }
    return LQCD_OK;
}

// x_hi += x_lo, x_lo = 0
lqcd_status fold_x(Cg& s)
{
    return blas_accumulate_x(s.c, s.X + s.o64, s.XLO + s.oa, s.PA, s.R, s.rb64, s.rba, s.nf);
}

// FP64 residual of the solved system: T2 = bhat - K x_hi (|T2|^2 -> SC_TMP + 2)
lqcd_status true_system_residual(Cg& s)
{
    lqcd_ctx* c = s.c;
    if (s.eo) {
        LQ_TRY(op_schur(c, s.T1 + s.fb64, s.X + s.fb64, s.T2, P64, false, s.R, s.rb64, s.rb64, -1));
        LQ_TRY(blas_xmy_norm(c, s.T2 + s.fb64, s.BH + s.fb64, s.T1 + s.fb64, P64, s.R, s.rb64, 1, SC_TMP + 2));
    } else {
        LQ_TRY(op_full(c, s.T1, s.X, P64, false, s.R, s.rb64));
        LQ_TRY(blas_xmy_norm(c, s.T2, s.B, s.T1, P64, s.R, s.rb64, 2, SC_TMP + 2));
    }
    return LQCD_OK;
}

// Reliable update at block slot j: fold x, recompute r = K^dag (bhat - K x_hi)
// in FP64, replace the inner r and its norm in slot j.
lqcd_status reliable_update(Cg& s, int j)
{
    lqcd_ctx* c = s.c;
    LQ_TRY(fold_x(s));
    LQ_TRY(true_system_residual(s));
    if (s.eo) {
        LQ_TRY(op_schur(c, s.RH + s.fb64, s.T2 + s.fb64, s.T1, P64, true, s.R, s.rb64, s.rb64, -1));
        LQ_TRY(convert_field(c, s.RV + s.fba, s.PA, s.RH + s.fb64, P64, s.R, s.rba, s.rb64, 1, rr_slot(j) + 1));
    } else {
        LQ_TRY(op_full(c, s.RH, s.T2, P64, true, s.R, s.rb64));
        LQ_TRY(convert_field(c, s.RV, s.PA, s.RH, P64, s.R, s.rba, s.rb64, 1, rr_slot(j)));
        LQ_TRY(convert_field(c, s.RV + s.fba, s.PA, s.RH + s.fb64, P64, s.R, s.rba, s.rb64, 1, rr_slot(j) + 1));
    }
    return LQCD_OK;
}

// n iterations with block-relative slots; optional reliable update before
// the last direction update; ends by moving slot n to slot 0.
lqcd_status run_block(Cg& s, int n, bool ru_at_end)
{
    for (int j = 0; j < n; ++j) {
        LQ_TRY(cg_iteration(s, j));
        if (ru_at_end && j == n - 1) LQ_TRY(reliable_update(s, j + 1));
        LQ_TRY(blas_cg_p_update(s.c, s.Pv + s.oi, mode_ps(s.Pi), s.RV + s.oa, s.PA, s.R, s.rbi, s.rba, s.nf, rr_slot(j + 1),
                                rr_slot(j)));
    }
    LQ_TRY(blas_copy_scalar(s.c, rr_slot(0), rr_slot(n), s.R));
    LQ_TRY(blas_copy_scalar(s.c, rr_slot(0) + 1, rr_slot(n) + 1, s.R));
    return LQCD_OK;
}

lqcd_status read_scalars(lqcd_ctx* c, int R, std::vector<double>& h)
{
    h.assign((size_t)R * SC_PER_RHS, 0.0);
    LQ_CUDA(cudaMemcpyAsync(h.data(), c->scal, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    LQ_CUDA(cudaStreamSynchronize(c->stream));
    return LQCD_OK;
}

bool is_device(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// A captured iteration block (graph), keyed by (length, reliable update).
struct BlockGraph {
    int n = -1;
    bool ru = false;
    cudaGraphExec_t exec = nullptr;
    long launches = 0;  // kernel nodes in the graph
    long dslash = 0;    // hopping applications in the graph
};

}  // namespace

lqcd_status solve(lqcd_ctx* c, double* x, const double* b, double tol, int R, const lqcd_solver_params* p,
                  lqcd_solver_stats* st)
{
    const auto t_start = std::chrono::steady_clock::now();
    if (p->solver == LQCD_SOLVER_FGCR) {
        if (R != 1) return fail(LQCD_ERR_INVALID, "lqcd_solve: FGCR solves one right-hand side per call");
        const bool hio = !is_device(b);
        if (hio != !is_device(x)) return fail(LQCD_ERR_INVALID, "lqcd_solve: x and b must both be host or both device");
        return solve_fgcr(c, c->precond, x, b, tol, p, st, hio);
    }
    if (p->solver != LQCD_SOLVER_CG_EO && p->solver != LQCD_SOLVER_CG_FULL)
        return fail(LQCD_ERR_INVALID, "lqcd_solve: unknown solver");
    if (p->check_interval < 1 || p->check_interval > SC_RING - 2)
        return fail(LQCD_ERR_INVALID, "lqcd_solve: check_interval must be in [1, 30]");
    if (p->maxiter < 1) return fail(LQCD_ERR_INVALID, "lqcd_solve: maxiter must be >= 1");
    c->dslash_count = 0;
    c->launches = 0;
    Cg s;
    s.c = c;
    s.R = R;
    s.Pi = p->inner_prec;
    s.PA = s.Pi == P64 ? P64 : P32;
    s.eo = p->solver == LQCD_SOLVER_CG_EO;
    s.nf = s.eo ? 1 : 2;
    s.fb64 = c->field_bytes(P64);
    s.rb64 = 2 * s.fb64;
    s.fbi = c->field_bytes(s.Pi);
    s.rbi = 2 * s.fbi;
    s.fba = c->field_bytes(s.PA);
    s.rba = 2 * s.fba;
    s.B = vec64_field(c, 0, 0);
    s.X = vec64_field(c, 1, 0);
    s.T1 = vec64_field(c, 2, 0);
    s.BH = vec64_field(c, 3, 0);
    s.RH = vec64_field(c, 4, 0);
    s.T2 = vec64_field(c, 5, 0);
    s.Pv = c->veclo;
    s.Qv = c->veclo + (size_t)R * s.rbi;
    s.XLO = c->vecacc;
    s.RV = c->vecacc + (size_t)R * s.rba;
    s.o64 = s.eo ? s.fb64 : 0;
    s.oi = s.eo ? s.fbi : 0;
    s.oa = s.eo ? s.fba : 0;
    const size_t canon_rb = (size_t)c->volume * 192;
    const bool host_io = !is_device(b);
    if (host_io != !is_device(x)) return fail(LQCD_ERR_INVALID, "lqcd_solve: x and b must both be host or both device");
    if (host_io && c->staging_bytes < (size_t)R * canon_rb) return fail(LQCD_ERR_NOMEM, "lqcd_solve: staging too small");

    // ---- set-up: pack b, scalars to zero
    const double* bdev = b;
    if (host_io) {
        LQ_CUDA(cudaMemcpyAsync(c->staging, b, (size_t)R * canon_rb, cudaMemcpyHostToDevice, c->stream));
        bdev = static_cast<const double*>(c->staging);
    }
    LQ_TRY(pack_spinor(c, s.B, bdev, -1, P64, R, s.rb64, canon_rb));
    LQ_CUDA(cudaMemsetAsync(c->scal, 0, (size_t)R * SC_PER_RHS * sizeof(double), c->stream));
    LQ_CUDA(cudaMemsetAsync(c->skip, 0, (size_t)R * sizeof(int), c->stream));
    LQ_TRY(blas_norm2(c, s.B, P64, R, s.rb64, 2, SC_TMP + 0));
    LQ_TRY(blas_zero(c, s.X, P64, R, s.rb64, 2));
    LQ_TRY(blas_zero(c, s.XLO, s.PA, R, s.rba, 2));
    if (s.eo) {
        // bhat_o = b_o + kappa H_oe A_ee^{-1} b_e
        const char* src_e = s.B;
        if (c->csw != 0.0) {
            LQ_TRY(clover_apply_launch(c, s.T1, s.B, 0, 1, P64, R, s.rb64));
            src_e = s.T1;
        }
        LQ_TRY(op_hop(c, s.BH + s.fb64, src_e, 1, P64, false, EPI_XPAY, false, nullptr, s.B + s.fb64, c->kappa, R,
                      s.rb64, -1));
        // r0 = Mhat^dag bhat_o (x0 = 0)
        LQ_TRY(op_schur(c, s.RH + s.fb64, s.BH + s.fb64, s.T2, P64, true, R, s.rb64, s.rb64, -1));
        LQ_TRY(convert_field(c, s.RV + s.fba, s.PA, s.RH + s.fb64, P64, R, s.rba, s.rb64, 1, rr_slot(0) + 1));
        LQ_TRY(convert_field(c, s.Pv + s.fbi, mode_ps(s.Pi), s.RV + s.fba, s.PA, R, s.rbi, s.rba, 1, -1));
    } else {
        LQ_TRY(op_full(c, s.RH, s.B, P64, true, R, s.rb64));
        LQ_TRY(convert_field(c, s.RV, s.PA, s.RH, P64, R, s.rba, s.rb64, 1, rr_slot(0)));
        LQ_TRY(convert_field(c, s.RV + s.fba, s.PA, s.RH + s.fb64, P64, R, s.rba, s.rb64, 1, rr_slot(0) + 1));
        LQ_TRY(convert_field(c, s.Pv, mode_ps(s.Pi), s.RV, s.PA, R, s.rbi, s.rba, 2, -1));
    }
    std::vector<double> h;
    LQ_TRY(read_scalars(c, R, h));
    std::vector<double> bn2(R), rr0(R), target(R), rrmax(R);
    std::vector<int> done(R, 0);
    double worst_res = 0.0;
    for (int r = 0; r < R; ++r) {
        bn2[r] = h[r * SC_PER_RHS + SC_TMP + 0];
        rr0[r] = h[r * SC_PER_RHS + rr_slot(0)] + h[r * SC_PER_RHS + rr_slot(0) + 1];
        target[r] = rr0[r] * tol * tol;
        rrmax[r] = rr0[r];
        if (bn2[r] == 0.0 || rr0[r] == 0.0) done[r] = 1;  // b = 0 (x = 0) or exact already
    }

    // ---- iterate in blocks
    const bool mixed = s.Pi != P64;
    const int ru_every = mixed ? p->reliable_interval : 0;
    const double delta2 = p->reliable_delta * p->reliable_delta;
    const bool graphs = p->use_graph && c->stream != nullptr;
    const bool log = getenv("LQCD_LOG") != nullptr;  // residual history on stderr
    std::vector<BlockGraph> cache;
    int k = 0, since_ru = 0;
    bool ru_next = false;
    lqcd_status status = LQCD_OK;
    int nrestart = 0;
    while (true) {
        int ndone = 0;
        for (int r = 0; r < R; ++r) ndone += done[r];
        if (ndone == R) break;
        if (k >= p->maxiter) {
            status = LQCD_ERR_NOT_CONVERGED;
            break;
        }
        int n = p->check_interval;
        if (n > p->maxiter - k) n = p->maxiter - k;
        bool ru = false;
        if (ru_every > 0 && since_ru + n >= ru_every) {
            n = ru_every - since_ru;
            if (n < 1) n = 1;
            ru = true;
        }
        if (ru_next && mixed) {
            ru = true;
            ru_next = false;
        }
        if (graphs) {
            BlockGraph* gph = nullptr;
            for (auto& e : cache)
                if (e.n == n && e.ru == ru) gph = &e;
            if (!gph) {
                cudaGraph_t graph;
                LQ_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
                const long saved = c->dslash_count, saved_l = c->launches;
                lqcd_status cs = run_block(s, n, ru);
                cudaError_t ce = cudaStreamEndCapture(c->stream, &graph);
                BlockGraph e;
                e.dslash = c->dslash_count - saved;
                e.launches = c->launches - saved_l;
                c->dslash_count = saved;
                c->launches = saved_l;
                if (cs != LQCD_OK) return cs;
                LQ_CUDA(ce);
                e.n = n;
                e.ru = ru;
                cudaError_t ie = cudaGraphInstantiate(&e.exec, graph, 0);
                cudaGraphDestroy(graph);
                LQ_CUDA(ie);
                cache.push_back(e);
                gph = &cache.back();
            }
            LQ_CUDA(cudaGraphLaunch(gph->exec, c->stream));
            c->dslash_count += gph->dslash;
            c->launches += gph->launches;
        } else {
            LQ_TRY(run_block(s, n, ru));
        }
        if (ru) {
            s.reliable++;
            since_ru = 0;
        } else {
            since_ru += n;
        }
        k += n;
        LQ_TRY(read_scalars(c, R, h));
        bool any_candidate = false;
        for (int r = 0; r < R; ++r) {
            if (done[r]) continue;
            const double rr = h[r * SC_PER_RHS + rr_slot(0)] + h[r * SC_PER_RHS + rr_slot(0) + 1];
            if (log) fprintf(stderr, "[lqcd] rhs %d iter %d |r|^2/|r0|^2 %.3e%s\n", r, k, rr / rr0[r], ru ? " (reliable update)" : "");
            if (!std::isfinite(rr) || rr > 1e30 * rr0[r]) {
                for (auto& e : cache) cudaGraphExecDestroy(e.exec);
                char msg[160];
                snprintf(msg, sizeof msg, "lqcd_solve: residual not finite or diverged (rhs %d, iteration %d, |r|^2 = %g)", r, k, rr);
                return fail(LQCD_ERR_BREAKDOWN, msg);
            }
            if (ru) rrmax[r] = rr;
            if (rr > rrmax[r]) rrmax[r] = rr;
            if (mixed && rr < delta2 * rrmax[r]) ru_next = true;
            if (rr <= target[r]) any_candidate = true;
        }
        if (any_candidate) {
            // true residual of the full system for every rhs (x is folded, r untouched)
            LQ_TRY(fold_x(s));
            LQ_TRY(true_system_residual(s));
            LQ_TRY(read_scalars(c, R, h));
            s.checks++;
            nrestart++;
            std::vector<int> skip(R, 0);
            for (int r = 0; r < R; ++r) {
                if (done[r]) { skip[r] = 1; continue; }
                const double rr = h[r * SC_PER_RHS + rr_slot(0)] + h[r * SC_PER_RHS + rr_slot(0) + 1];
                if (rr > target[r]) continue;
                const double res = std::sqrt(h[r * SC_PER_RHS + SC_TMP + 2] / bn2[r]);
                if (log) fprintf(stderr, "[lqcd] rhs %d iter %d true residual %.3e\n", r, k, res);
                if (res <= 0.5 * tol) {
                    done[r] = 1;
                    skip[r] = 1;
                } else {
                    double f = (0.25 * tol / res);
                    f *= f;
                    if (f > 0.5) f = 0.5;
                    if (f < 1e-6) f = 1e-6;
                    target[r] = rr * f;
                    if (mixed) ru_next = true;
                }
            }
            LQ_CUDA(cudaMemcpyAsync(c->skip, skip.data(), R * sizeof(int), cudaMemcpyHostToDevice, c->stream));
            LQ_CUDA(cudaStreamSynchronize(c->stream));
        }
    }
    for (auto& e : cache) cudaGraphExecDestroy(e.exec);

    // ---- finish: fold x, reconstruct x_e, FP64 true residual, unpack
    LQ_TRY(fold_x(s));
    if (s.eo) {
        // x_e = A_ee^{-1} (b_e + kappa H_eo x_o)
        LQ_TRY(op_hop(c, s.T1, s.X + s.fb64, 0, P64, false, EPI_XPAY, false, nullptr, s.B, c->kappa, R, s.rb64, -1));
        if (c->csw != 0.0) {
            LQ_TRY(clover_apply_launch(c, s.X, s.T1, 0, 1, P64, R, s.rb64));
        } else {
            LQ_TRY(convert_field(c, s.X, P64, s.T1, P64, R, s.rb64, s.rb64, 1, -1));
        }
    }
    LQ_TRY(op_full(c, s.T1, s.X, P64, false, R, s.rb64));
    LQ_TRY(blas_xmy_norm(c, s.T2, s.B, s.T1, P64, R, s.rb64, 2, SC_TMP + 3));
    double* xdev = host_io ? static_cast<double*>(c->staging) : x;
    LQ_TRY(unpack_spinor(c, xdev, s.X, -1, P64, R, s.rb64, canon_rb));
    if (host_io) LQ_CUDA(cudaMemcpyAsync(x, c->staging, (size_t)R * canon_rb, cudaMemcpyDeviceToHost, c->stream));
    LQ_TRY(read_scalars(c, R, h));
    for (int r = 0; r < R; ++r) {
        const double res = bn2[r] > 0 ? std::sqrt(h[r * SC_PER_RHS + SC_TMP + 3] / bn2[r]) : 0.0;
        if (res > worst_res) worst_res = res;
        if (!std::isfinite(res)) status = LQCD_ERR_BREAKDOWN;
        else if (res > tol && status == LQCD_OK) status = LQCD_ERR_NOT_CONVERGED;
    }
    st->iterations = k;
    st->reliable_updates = (int)s.reliable;
    st->restarts = nrestart;
    st->dslash_count = c->dslash_count;
    st->kernel_launches = c->launches;
    st->true_residual = worst_res;
    st->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    if (status == LQCD_ERR_NOT_CONVERGED) return fail(status, "lqcd_solve: not converged within maxiter");
    if (status == LQCD_ERR_BREAKDOWN) return fail(status, "lqcd_solve: breakdown");
    return LQCD_OK;
}

}  // namespace lqcd
