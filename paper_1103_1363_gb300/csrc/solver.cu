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

static const void* clov_or_null(lqcd_ctx* c, int P, int parity, bool inverse)
{
    if (c->csw == 0.0) return nullptr;
    const int pg = mode_pg(P);
    const char* base = static_cast<const char*>(inverse ? c->clovinv[pg] : c->clov[pg]);
    return base + parity * c->clov_parity_bytes(pg);
}

// The four hopping launches of an even-odd CG iteration j (block-relative
// scalar slots):
//   D1: t_e = A_ee^{-1} H_eo p_o
//   D2: q_o = A_oo p_o - kappa^2 H_oe t_e,               |q_o|^2 -> pap slot j
//   D3: t_e = A_ee^{-1} H_eo^dag q_o
//   D4: s = A_oo q_o - kappa^2 H_oe^dag t_e; x += alpha p; r -= alpha s,
//       alpha = |r|^2 / |q|^2 from slots j,                |r|^2 -> rr slot j + 1
// (D1, D3: EPI_CLOVINV; D2: EPI_XPAY with the norm; D4: EPI_CG, dagger for D3, D4.)
void eo_stage_args(const Cg& s, int j, DslashArgs d[4])
{
    lqcd_ctx* c = s.c;
    const int P = s.Pi;
    DslashArgs A = base_args(c, P);
    A.skip = c->skip;
    A.par = 0;
    A.out = s.Qv;
    A.out_rb = s.rbi;
    A.in = s.Pv + s.fbi;
    A.in_rb = s.rbi;
    A.clov = clov_or_null(c, P, 0, true);
    A.a = 1.0;
    d[0] = A;
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
    d[1] = B;
    A.in = s.Qv + s.fbi;
    d[2] = A;
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
    d[3] = D;
}

namespace {

// One inner CG iteration j of a block: q = K p, x += alpha p, r -= alpha K^dag q
// with K = Mhat (eo) or M (full), |r|^2 into block slot j + 1.
lqcd_status cg_iteration(Cg& s, int j)
{
    lqcd_ctx* c = s.c;
    const int P = s.Pi;
    if (s.eo) {
        DslashArgs d[4];
        eo_stage_args(s, j, d);
        LQ_TRY(launch_dslash(c, d[0], P, false, EPI_CLOVINV, false, s.R));
        LQ_TRY(launch_dslash(c, d[1], P, false, EPI_XPAY, true, s.R));
        LQ_TRY(launch_dslash(c, d[2], P, true, EPI_CLOVINV, false, s.R));
        LQ_TRY(launch_dslash(c, d[3], P, true, EPI_CG, true, s.R));
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

// RV_o = Mhat^dag d_o for an FP64 odd field d (stride rb64), |RV_o|^2 into
// slot.  Only the defect d needs FP64 (it comes from a cancellation); the
// map applied to it does not, so a mixed solve with FP32 links at hand
// applies Mhat^dag in FP32 to d rounded to FP32, which is as accurate as
// rounding the FP64 product into the FP32 vector.  T1 is the scratch.
lqcd_status normal_residual_eo(Cg& s, const char* d_odd, int slot)
{
    lqcd_ctx* c = s.c;
    if (s.PA == P32 && c->holds(P32)) {
        char* d32 = s.T1;                         // R fields at stride rba
        char* tmp = s.T1 + (size_t)s.R * s.rba;   // R even scratch fields
        LQ_TRY(convert_field(c, d32, P32, d_odd, P64, s.R, s.rba, s.rb64, 1, -1));
        return op_schur(c, s.RV + s.fba, d32, tmp, LQCD_F32, true, s.R, s.rba, s.rba, slot);
    }
    LQ_TRY(op_schur(c, s.RH + s.fb64, d_odd, s.T1, P64, true, s.R, s.rb64, s.rb64, -1));
    return convert_field(c, s.RV + s.fba, s.PA, s.RH + s.fb64, P64, s.R, s.rba, s.rb64, 1, slot);
}

// Reliable update at block slot j: fold x, recompute r = K^dag (bhat - K x_hi)
// with the defect bhat - K x_hi in FP64, replace the inner r and its norm in
// slot j.
lqcd_status reliable_update(Cg& s, int j)
{
    lqcd_ctx* c = s.c;
    LQ_TRY(fold_x(s));
    LQ_TRY(true_system_residual(s));
    if (s.eo) {
        LQ_TRY(normal_residual_eo(s, s.T2 + s.fb64, rr_slot(j) + 1));
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

// A captured iteration block (graph) for a set of runs, keyed by
// (length, reliable update, which runs are active).
struct BlockGraph {
    int n = -1;
    bool ru = false;
    unsigned long long mask = 0;
    cudaGraphExec_t exec = nullptr;
    std::vector<long> launches;  // kernel nodes per run
    std::vector<long> dslash;    // hopping applications per run
};

// State of one CG solve (one lattice, nrhs right-hand sides).
struct CgRun {
    Cg s;
    lqcd_ctx* c = nullptr;
    double* x = nullptr;
    const double* b = nullptr;
    double tol = 0.0;
    bool host_io = false;
    int maxiter = 0;
    std::vector<double> h, bn2, rr0, target, rrmax;
    std::vector<int> done;
    bool mixed = false, log = false, ru_next = false;
    int ru_every = 0;
    // stagnation of a 16-bit inner iteration: |r|^2 at consecutive reliable
    // updates; after three that do not halve it the inner storage becomes FP32
    std::vector<double> rr_last_ru;
    int stalls = 0;
    bool fell_back = false, rebuild_graphs = false;
    double delta2 = 0.0;
    int k = 0, since_ru = 0, nrestart = 0;
    lqcd_status status = LQCD_OK;
    std::chrono::steady_clock::time_point t_start;
    bool finished() const
    {
        if (status != LQCD_OK) return true;
        for (int d : done)
            if (!d) return false;
        return true;
    }
};

lqcd_status cg_setup(CgRun& run, lqcd_ctx* c, double* x, const double* b, double tol, int R,
                     const lqcd_solver_params* p)
{
    run.t_start = std::chrono::steady_clock::now();
    if (p->solver != LQCD_SOLVER_CG_EO && p->solver != LQCD_SOLVER_CG_FULL)
        return fail(LQCD_ERR_INVALID, "lqcd_solve: unknown solver");
    if (p->check_interval < 1 || p->check_interval > SC_RING - 2)
        return fail(LQCD_ERR_INVALID, "lqcd_solve: check_interval must be in [1, 30]");
    if (p->maxiter < 1) return fail(LQCD_ERR_INVALID, "lqcd_solve: maxiter must be >= 1");
    c->dslash_count = 0;
    c->launches = 0;
    run.c = c;
    run.x = x;
    run.b = b;
    run.tol = tol;
    run.maxiter = p->maxiter;
    Cg& s = run.s;
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
    if (p->residual_prec != LQCD_F64) return fail(LQCD_ERR_INVALID, "lqcd_solve: residual_prec must be LQCD_F64");
    const size_t canon_rb = (size_t)c->volume * 192;
    run.host_io = !is_device(b);
    if (run.host_io != !is_device(x)) return fail(LQCD_ERR_INVALID, "lqcd_solve: x and b must both be host or both device");
    if (run.host_io && c->staging_bytes < (size_t)R * canon_rb) return fail(LQCD_ERR_NOMEM, "lqcd_solve: staging too small");

    // pack b, scalars to zero
    const double* bdev = b;
    if (run.host_io) {
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
        LQ_TRY(normal_residual_eo(s, s.BH + s.fb64, rr_slot(0) + 1));
        LQ_TRY(convert_field(c, s.Pv + s.fbi, mode_ps(s.Pi), s.RV + s.fba, s.PA, R, s.rbi, s.rba, 1, -1));
    } else {
        LQ_TRY(op_full(c, s.RH, s.B, P64, true, R, s.rb64));
        LQ_TRY(convert_field(c, s.RV, s.PA, s.RH, P64, R, s.rba, s.rb64, 1, rr_slot(0)));
        LQ_TRY(convert_field(c, s.RV + s.fba, s.PA, s.RH + s.fb64, P64, R, s.rba, s.rb64, 1, rr_slot(0) + 1));
        LQ_TRY(convert_field(c, s.Pv, mode_ps(s.Pi), s.RV, s.PA, R, s.rbi, s.rba, 2, -1));
    }
    LQ_TRY(read_scalars(c, R, run.h));
    run.bn2.assign(R, 0.0);
    run.rr0.assign(R, 0.0);
    run.target.assign(R, 0.0);
    run.rrmax.assign(R, 0.0);
    run.rr_last_ru.assign(R, 0.0);
    run.done.assign(R, 0);
    for (int r = 0; r < R; ++r) {
        run.bn2[r] = run.h[r * SC_PER_RHS + SC_TMP + 0];
        run.rr0[r] = run.h[r * SC_PER_RHS + rr_slot(0)] + run.h[r * SC_PER_RHS + rr_slot(0) + 1];
        run.target[r] = run.rr0[r] * tol * tol;
        run.rrmax[r] = run.rr0[r];
        if (run.bn2[r] == 0.0 || run.rr0[r] == 0.0) run.done[r] = 1;  // b = 0 (x = 0) or exact already
    }
    run.mixed = s.Pi != P64;
    run.ru_every = run.mixed ? p->reliable_interval : 0;
    run.delta2 = p->reliable_delta * p->reliable_delta;
    run.log = getenv("LQCD_LOG") != nullptr;  // residual history on stderr
    return LQCD_OK;
}

// After a block of n iterations: read |r|^2, detect breakdown, check
// candidates on the FP64 true residual, mark converged right-hand sides.
// A 16-bit inner iteration that has stopped making progress between
// reliable updates (on ill-conditioned systems 11 or 8 bits of the search
// directions cannot resolve the remaining residual) continues with FP32
// inner storage: the same links (FP32 copy), p restarted from r.
lqcd_status fall_back_to_f32(CgRun& run)
{
    lqcd_ctx* c = run.c;
    Cg& s = run.s;
    run.stalls = 0;
    if (run.fell_back || s.Pi == P64 || s.Pi == LQCD_F32 || mode_ps(s.Pi) == P64 || !c->holds(P32)) return LQCD_OK;
    if (run.log) fprintf(stderr, "[lqcd] iter %d: inner iteration stagnates, continuing with FP32 storage\n", run.k);
    s.Pi = LQCD_F32;
    s.fbi = c->field_bytes(s.Pi);
    s.rbi = 2 * s.fbi;
    s.Qv = c->veclo + (size_t)s.R * s.rbi;
    s.oi = s.eo ? s.fbi : 0;
    if (s.eo) LQ_TRY(convert_field(c, s.Pv + s.fbi, P32, s.RV + s.fba, s.PA, s.R, s.rbi, s.rba, 1, -1));
    else LQ_TRY(convert_field(c, s.Pv, P32, s.RV, s.PA, s.R, s.rbi, s.rba, 2, -1));
    run.fell_back = true;
    run.rebuild_graphs = true;
    return LQCD_OK;
}

lqcd_status cg_check(CgRun& run, int n, bool ru)
{
    lqcd_ctx* c = run.c;
    Cg& s = run.s;
    const int R = s.R;
    if (ru) {
        s.reliable++;
        run.since_ru = 0;
    } else {
        run.since_ru += n;
    }
    run.k += n;
    LQ_TRY(read_scalars(c, R, run.h));
    bool any_candidate = false, any_stall = false;
    for (int r = 0; r < R; ++r) {
        if (run.done[r]) continue;
        const double rr = run.h[r * SC_PER_RHS + rr_slot(0)] + run.h[r * SC_PER_RHS + rr_slot(0) + 1];
        if (run.log)
            fprintf(stderr, "[lqcd] rhs %d iter %d |r|^2/|r0|^2 %.3e%s\n", r, run.k, rr / run.rr0[r],
                    ru ? " (reliable update)" : "");
        if (!std::isfinite(rr) || rr > 1e30 * run.rr0[r]) {
            char msg[160];
            snprintf(msg, sizeof msg, "lqcd_solve: residual not finite or diverged (rhs %d, iteration %d, |r|^2 = %g)",
                     r, run.k, rr);
            run.status = fail(LQCD_ERR_BREAKDOWN, msg);
            return run.status;
        }
        if (ru) {
            run.rrmax[r] = rr;
            if (run.rr_last_ru[r] > 0.0 && rr > 0.5 * run.rr_last_ru[r]) any_stall = true;
            run.rr_last_ru[r] = rr;
        }
        if (rr > run.rrmax[r]) run.rrmax[r] = rr;
        if (run.mixed && rr < run.delta2 * run.rrmax[r]) run.ru_next = true;
        if (rr <= run.target[r]) any_candidate = true;
    }
    if (ru) {
        run.stalls = any_stall ? run.stalls + 1 : 0;
        if (run.stalls >= 3) LQ_TRY(fall_back_to_f32(run));
    }
    if (!any_candidate) return LQCD_OK;
    // true residual of the full system for every rhs (x is folded, r untouched)
    LQ_TRY(fold_x(s));
    LQ_TRY(true_system_residual(s));
    LQ_TRY(read_scalars(c, R, run.h));
    s.checks++;
    run.nrestart++;
    std::vector<int> skip(R, 0);
    for (int r = 0; r < R; ++r) {
        if (run.done[r]) {
            skip[r] = 1;
            continue;
        }
        const double rr = run.h[r * SC_PER_RHS + rr_slot(0)] + run.h[r * SC_PER_RHS + rr_slot(0) + 1];
        if (rr > run.target[r]) continue;
        const double res = std::sqrt(run.h[r * SC_PER_RHS + SC_TMP + 2] / run.bn2[r]);
        if (run.log) fprintf(stderr, "[lqcd] rhs %d iter %d true residual %.3e\n", r, run.k, res);
        if (res <= 0.5 * run.tol) {
            run.done[r] = 1;
            skip[r] = 1;
        } else {
            double f = (0.25 * run.tol / res);
            f *= f;
            if (f > 0.5) f = 0.5;
            if (f < 1e-6) f = 1e-6;
            run.target[r] = rr * f;
            if (run.mixed) run.ru_next = true;
        }
    }
    LQ_CUDA(cudaMemcpyAsync(c->skip, skip.data(), R * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    LQ_CUDA(cudaStreamSynchronize(c->stream));
    return LQCD_OK;
}

// Fold x, reconstruct x_e, FP64 true residual, unpack, stats.
lqcd_status cg_finish(CgRun& run, lqcd_solver_stats* st)
{
    lqcd_ctx* c = run.c;
    Cg& s = run.s;
    const int R = s.R;
    const size_t canon_rb = (size_t)c->volume * 192;
    lqcd_status status = run.status;
    if (status == LQCD_OK && !run.finished()) status = LQCD_ERR_NOT_CONVERGED;
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
    double* xdev = run.host_io ? static_cast<double*>(c->staging) : run.x;
    LQ_TRY(unpack_spinor(c, xdev, s.X, -1, P64, R, s.rb64, canon_rb));
    if (run.host_io)
        LQ_CUDA(cudaMemcpyAsync(run.x, c->staging, (size_t)R * canon_rb, cudaMemcpyDeviceToHost, c->stream));
    LQ_TRY(read_scalars(c, R, run.h));
    double worst = 0.0;
    for (int r = 0; r < R; ++r) {
        const double res = run.bn2[r] > 0 ? std::sqrt(run.h[r * SC_PER_RHS + SC_TMP + 3] / run.bn2[r]) : 0.0;
        if (res > worst || !std::isfinite(res)) worst = res;
        if (!std::isfinite(res)) status = LQCD_ERR_BREAKDOWN;
        else if (res > run.tol && status == LQCD_OK) status = LQCD_ERR_NOT_CONVERGED;
    }
    st->iterations = run.k;
    st->reliable_updates = (int)s.reliable;
    st->precision_fallback = run.fell_back ? 1 : 0;
    st->restarts = run.nrestart;
    st->dslash_count = c->dslash_count;
    st->kernel_launches = c->launches;
    st->true_residual = worst;
    st->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - run.t_start).count();
    if (status == LQCD_ERR_NOT_CONVERGED) return fail(status, "lqcd_solve: not converged within maxiter");
    if (status == LQCD_ERR_BREAKDOWN) return fail(status, "lqcd_solve: breakdown");
    return LQCD_OK;
}

// One block of n iterations of every active run as persistent launches (one
// per inner precision present: a 16-bit run that fell back to FP32 forms its
// own group); with a reliable update at its end a launch stops before the
// last direction update, and the update, the direction update and the slot
// copy follow as separate launches (as in run_block).  Inside the launch the
// |r|^2 slots are a ring of two: the block's final |r|^2 is in slot n mod 2.
lqcd_status run_block_persistent(std::vector<CgRun*>& runs, unsigned long long mask, int n, bool ru,
                                 const lqcd_solver_params* p)
{
    lqcd_ctx* c0 = runs[0]->c;
    char* w = c0->persist;
    double* partials = reinterpret_cast<double*>(w);
    unsigned* tickets = reinterpret_cast<unsigned*>(w + (size_t)PERSIST_MAXPAIRS * PERSIST_MAX_TILES * sizeof(double));
    int* abort_word = reinterpret_cast<int*>(tickets + PERSIST_MAXPAIRS + 2);
    unsigned long long todo = mask;
    while (todo) {
        int mode = -1, recon = -1, pairs = 0;
        PersistArgs P;
        memset(&P, 0, sizeof(P));
        std::vector<size_t> members;
        for (size_t i = 0; i < runs.size(); ++i) {
            if (!(todo >> i & 1)) continue;
            Cg& s = runs[i]->s;
            if (!s.eo) return fail(LQCD_ERR_INVALID, "persistent CG: even-odd CG only");
            const int rc = s.c->recon_of(mode_pg(s.Pi));
            if (mode < 0) {
                mode = s.Pi;
                recon = rc;
            }
            if (s.Pi != mode || rc != recon) continue;  // a later group
            if ((int)members.size() == PERSIST_MAXL) return fail(LQCD_ERR_INVALID, "persistent CG: at most 8 lattices");
            if (pairs + s.R > PERSIST_MAXPAIRS)
                return fail(LQCD_ERR_INVALID, "persistent CG: at most 64 right-hand sides");
            members.push_back(i);
            pairs += s.R;
        }
        pairs = 0;
        int ntiles = 0;
        for (size_t m : members) {
            todo &= ~(1ull << m);
            Cg& s = runs[m]->s;
            lqcd_ctx* c = s.c;
            PersistLattice& L = P.lat[P.nlat++];
            for (int jj = 0; jj < 2; ++jj) {
                eo_stage_args(s, jj, L.d[jj]);
                L.d[jj][3].red = c->scal + rr_slot((jj + 1) & 1) + 1;  // the ring of two
                for (int k = 0; k < 4; ++k) {
                    L.d[jj][k].nrhs = s.R;
                    L.d[jj][k].partials = partials + (size_t)pairs * PERSIST_MAX_TILES;
                    L.d[jj][k].part_rs = PERSIST_MAX_TILES;
                    L.d[jj][k].tickets = tickets + pairs;
                }
            }
            L.g = c->g;
            L.R = s.R;
            L.pair0 = pairs;
            const long per = (long)PERSIST_THREADS * PERSIST_MAX_TILES;
            L.spt = (int)((c->g.Vh + per - 1) / per);
            L.ntiles = (c->g.Vh + PERSIST_THREADS * L.spt - 1) / (PERSIST_THREADS * L.spt);
            for (int r = 0; r < s.R; ++r) {
                P.tile0[P.npairs] = ntiles;
                P.pair_lat[P.npairs] = (unsigned char)(P.nlat - 1);
                P.pair_rhs[P.npairs] = (unsigned char)r;
                P.npairs++;
                ntiles += L.ntiles;
            }
            L.p = s.Pv + s.fbi;
            L.p_rb = s.rbi;
            L.r = s.RV + s.fba;
            L.r_rb = s.rba;
            L.scal = c->scal;
            L.skip = c->skip;
            pairs += s.R;
            c->dslash_count += 4L * n * s.R;
            c->launches++;
        }
        P.tile0[P.npairs] = ntiles;
        int grid = 0;
        LQ_TRY(persist_grid(mode, recon, ntiles, &grid));
        P.niter = n;
        P.last_p = ru ? 0 : 1;
        P.copy_slots = ru ? 0 : 1;
        P.partials = partials;
        P.tickets = tickets;
        P.bar = tickets + PERSIST_MAXPAIRS;
        P.abort = abort_word;
        P.errw = c0->errw;
        P.wait_ns = p->persistent_wait_us > 0 ? 1000ull * (unsigned long long)p->persistent_wait_us : 2000000000ull;
        // tickets, barrier words and abort word start at zero (an aborted launch leaves them set)
        LQ_CUDA(cudaMemsetAsync(tickets, 0, (PERSIST_MAXPAIRS + 3) * sizeof(unsigned), c0->stream));
        LQ_TRY(launch_persist(c0, P, mode, recon, grid));
        int aborted = 0;
        LQ_CUDA(cudaMemcpyAsync(&aborted, abort_word, sizeof(int), cudaMemcpyDeviceToHost, c0->stream));
        LQ_CUDA(cudaStreamSynchronize(c0->stream));
        if (aborted) return fail(LQCD_ERR_TIMEOUT, "persistent CG: a grid-barrier wait expired");
    }
    if (ru) {
        const int jn = n & 1, jp = (n - 1) & 1;
        for (size_t i = 0; i < runs.size(); ++i) {
            if (!(mask >> i & 1)) continue;
            Cg& s = runs[i]->s;
            LQ_TRY(reliable_update(s, jn));
            LQ_TRY(blas_cg_p_update(s.c, s.Pv + s.oi, mode_ps(s.Pi), s.RV + s.oa, s.PA, s.R, s.rbi, s.rba, s.nf,
                                    rr_slot(jn), rr_slot(jp)));
            if (jn) {
                LQ_TRY(blas_copy_scalar(s.c, rr_slot(0), rr_slot(1), s.R));
                LQ_TRY(blas_copy_scalar(s.c, rr_slot(0) + 1, rr_slot(1) + 1, s.R));
            }
        }
    }
    return LQCD_OK;
}

void destroy_graphs(std::vector<BlockGraph>& cache)
{
    for (auto& e : cache)
        if (e.exec) cudaGraphExecDestroy(e.exec);
    cache.clear();
}

// Streams and events that fork the runs of a batch into parallel branches
// of a captured graph (one branch per run after the first).
struct Fork {
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;  // [0]: the fork point; [i]: run i's join
    ~Fork()
    {
        for (auto s : streams)
            if (s) cudaStreamDestroy(s);
        for (auto e : events)
            if (e) cudaEventDestroy(e);
    }
    lqcd_status init(size_t n)
    {
        streams.assign(n, nullptr);
        events.assign(n, nullptr);
        for (size_t i = 0; i < n; ++i) {
            LQ_CUDA(cudaEventCreateWithFlags(&events[i], cudaEventDisableTiming));
            if (i > 0) LQ_CUDA(cudaStreamCreateWithFlags(&streams[i], cudaStreamNonBlocking));
        }
        return LQCD_OK;
    }
};

// Iterate every unfinished run in lockstep blocks until all finish or hit
// maxiter; with graphs, one graph holds the block of every active run.  The
// runs of a batch (distinct contexts, hence disjoint memory) are captured as
// parallel branches, so that the lattices' kernels run side by side: the
// small lattices of an uneven batch do not fill the GPU one after another.
lqcd_status iterate(std::vector<CgRun*>& runs, const lqcd_solver_params* p)
{
    lqcd_ctx* c0 = runs[0]->c;
    const bool persistent = p->persistent != 0;
    const bool graphs = !persistent && p->use_graph && c0->stream != nullptr;
    bool branches = graphs && runs.size() > 1;
    for (size_t i = 0; i < runs.size() && branches; ++i)
        for (size_t j = 0; j < i; ++j)
            if (runs[i]->c == runs[j]->c) branches = false;
    Fork fork;
    if (branches) LQ_TRY(fork.init(runs.size()));
    std::vector<BlockGraph> cache;
    while (true) {
        NvtxRange nvtx_range("cg iteration block");
        unsigned long long mask = 0;
        int kmax = 0, since = 0, ru_every = 0;
        bool ru_next = false;
        for (size_t i = 0; i < runs.size(); ++i) {
            CgRun& r = *runs[i];
            if (r.finished() || r.k >= r.maxiter) continue;
            mask |= 1ull << i;
            kmax = r.k > kmax ? r.k : kmax;
            since = r.since_ru;
            ru_every = r.ru_every;
            ru_next = ru_next || (r.ru_next && r.mixed);
        }
        if (!mask) break;
        int maxiter = p->maxiter;
        int n = p->check_interval;
        if (n > maxiter - kmax) n = maxiter - kmax;
        if (n < 1) break;
        bool ru = false;
        if (ru_every > 0 && since + n >= ru_every) {
            n = ru_every - since;
            if (n < 1) n = 1;
            ru = true;
        }
        if (ru_next) ru = true;
        for (auto* r : runs) r->ru_next = false;
        if (persistent) {
            lqcd_status ps = run_block_persistent(runs, mask, n, ru, p);
            if (ps != LQCD_OK) return ps;
        } else if (graphs) {
            BlockGraph* gph = nullptr;
            for (auto& e : cache)
                if (e.n == n && e.ru == ru && e.mask == mask) gph = &e;
            if (!gph) {
                BlockGraph e;
                e.n = n;
                e.ru = ru;
                e.mask = mask;
                e.launches.assign(runs.size(), 0);
                e.dslash.assign(runs.size(), 0);
                cudaGraph_t graph;
                LQ_CUDA(cudaStreamBeginCapture(c0->stream, cudaStreamCaptureModeThreadLocal));
                lqcd_status cs = LQCD_OK;
                cudaError_t fe = cudaSuccess;
                if (branches) fe = cudaEventRecord(fork.events[0], c0->stream);
                for (size_t i = 0; i < runs.size() && cs == LQCD_OK && fe == cudaSuccess; ++i) {
                    if (!(mask >> i & 1)) continue;
                    lqcd_ctx* c = runs[i]->c;
                    const bool branch = branches && i > 0;
                    if (branch) {  // run i on a branch of its own: fork from c0's stream ...
                        fe = cudaStreamWaitEvent(fork.streams[i], fork.events[0], 0);
                        if (fe != cudaSuccess) break;
                        c->stream = fork.streams[i];
                    }
                    const long d0 = c->dslash_count, l0 = c->launches;
                    cs = run_block(runs[i]->s, n, ru);
                    e.dslash[i] = c->dslash_count - d0;
                    e.launches[i] = c->launches - l0;
                    c->dslash_count = d0;
                    c->launches = l0;
                    if (branch) {  // ... and join back into it
                        if (cs == LQCD_OK) {
                            fe = cudaEventRecord(fork.events[i], fork.streams[i]);
                            if (fe == cudaSuccess) fe = cudaStreamWaitEvent(c0->stream, fork.events[i], 0);
                        }
                        c->stream = c0->stream;
                    }
                }
                cudaError_t ce = cudaStreamEndCapture(c0->stream, &graph);
                if (fe != cudaSuccess && ce == cudaSuccess) ce = fe;
                if (cs != LQCD_OK) { destroy_graphs(cache); return cs; }
                if (ce != cudaSuccess) { destroy_graphs(cache); return cuda_fail(ce, "cudaStreamEndCapture"); }
                cudaError_t ie = cudaGraphInstantiate(&e.exec, graph, 0);
                cudaGraphDestroy(graph);
                if (ie != cudaSuccess) { destroy_graphs(cache); return cuda_fail(ie, "cudaGraphInstantiate"); }
                cache.push_back(e);
                gph = &cache.back();
            }
            cudaError_t le = cudaGraphLaunch(gph->exec, c0->stream);
            if (le != cudaSuccess) { destroy_graphs(cache); return cuda_fail(le, "cudaGraphLaunch"); }
            for (size_t i = 0; i < runs.size(); ++i) {
                runs[i]->c->dslash_count += gph->dslash[i];
                runs[i]->c->launches += gph->launches[i];
            }
        } else {
            for (size_t i = 0; i < runs.size(); ++i)
                if (mask >> i & 1) {
                    lqcd_status bs = run_block(runs[i]->s, n, ru);
                    if (bs != LQCD_OK) return bs;
                }
        }
        bool rebuild = false;
        for (size_t i = 0; i < runs.size(); ++i)
            if (mask >> i & 1) {
                lqcd_status cs = cg_check(*runs[i], n, ru);
                if (cs != LQCD_OK && runs[i]->status == LQCD_OK) { destroy_graphs(cache); return cs; }
                rebuild = rebuild || runs[i]->rebuild_graphs;
                runs[i]->rebuild_graphs = false;
            }
        if (rebuild) destroy_graphs(cache);  // captured with the old inner precision
    }
    destroy_graphs(cache);
    return LQCD_OK;
}

}  // namespace

lqcd_status solve(lqcd_ctx* c, double* x, const double* b, double tol, int R, const lqcd_solver_params* p,
                  lqcd_solver_stats* st)
{
    if (p->solver == LQCD_SOLVER_FGCR || p->solver == LQCD_SOLVER_FGMRES_DR) {
        if (R != 1) return fail(LQCD_ERR_INVALID, "lqcd_solve: FGCR / FGMRES-DR solve one right-hand side per call");
        const bool hio = !is_device(b);
        if (hio != !is_device(x)) return fail(LQCD_ERR_INVALID, "lqcd_solve: x and b must both be host or both device");
        if (p->solver == LQCD_SOLVER_FGMRES_DR) return solve_fgmres_dr(c, c->precond, x, b, tol, p, st, hio);
        return solve_fgcr(c, c->precond, x, b, tol, p, st, hio);
    }
    CgRun run;
    LQ_TRY(cg_setup(run, c, x, b, tol, R, p));
    std::vector<CgRun*> runs{&run};
    lqcd_status is = iterate(runs, p);
    if (is != LQCD_OK && run.status == LQCD_OK) return is;
    return cg_finish(run, st);
}

// Several lattices solved together: set-up per lattice, then lockstep
// iteration blocks (one CUDA graph for all lattices with use_graph), then
// the per-lattice finish.  Every context runs on the stream of ctxs[0]
// during the call.
lqcd_status solve_batch(lqcd_ctx* const* ctxs, int n, double* const* x, const double* const* b, const double* tol,
                        const lqcd_solver_params* p, lqcd_solver_stats* st)
{
    if (n < 1 || n > 64) return fail(LQCD_ERR_INVALID, "lqcd_solve_batch: 1..64 lattices");
    if (p->solver == LQCD_SOLVER_FGCR) return fail(LQCD_ERR_INVALID, "lqcd_solve_batch: CG solvers only");
    std::vector<cudaStream_t> saved(n);
    for (int i = 0; i < n; ++i) {
        saved[i] = ctxs[i]->stream;
        ctxs[i]->stream = ctxs[0]->stream;
    }
    std::vector<CgRun> runs(n);
    std::vector<CgRun*> ptrs;
    lqcd_status status = LQCD_OK;
    for (int i = 0; i < n && status == LQCD_OK; ++i) {
        status = cg_setup(runs[i], ctxs[i], x[i], b[i], tol[i], 1, p);
        ptrs.push_back(&runs[i]);
    }
    if (status == LQCD_OK) status = iterate(ptrs, p);
    lqcd_status worst = status;
    if (status == LQCD_OK || status == LQCD_ERR_BREAKDOWN) {
        for (int i = 0; i < n; ++i) {
            lqcd_status fs = cg_finish(runs[i], &st[i]);
            if (fs != LQCD_OK && worst == LQCD_OK) worst = fs;
        }
    }
    for (int i = 0; i < n; ++i) ctxs[i]->stream = saved[i];
    return worst;
}

}  // namespace lqcd
