// C ABI entry points (include/lqcd.h): context and workspace management,
// gauge and clover set-up, packing, operator application.
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

namespace lqcd {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

lqcd_status fail(lqcd_status st, const std::string& msg)
{
    g_last_error = msg;
    return st;
}

lqcd_status cuda_fail(cudaError_t e, const char* where)
{
    g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
    return LQCD_ERR_CUDA;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Is p a device-accessible pointer (device or managed memory)?
static bool is_device_ptr(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

DslashArgs base_args(lqcd_ctx* c, int P)
{
    DslashArgs A;
    memset(&A, 0, sizeof(A));
    A.g = c->g;
    A.gauge = c->gauge[mode_pg(P)];
    A.partials = c->partials;
    A.part_rs = c->part_rs;
    A.tickets = c->tickets;
    A.scal = c->scal;
    A.scal_rs = SC_PER_RHS;
    A.red_rs = SC_PER_RHS;
    return A;
}

// ---- kernel timing: event pairs around each hopping-term launch
struct Profiler {
    struct Rec { int P; cudaEvent_t a, b; double bytes, flops; };
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
    ~Profiler()
    {
        for (auto e : pool) cudaEventDestroy(e);
        for (auto& r : pending) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    }
};

// Compulsory bytes of one launch per output site: every right-hand side's
// input spinor and epilogue vectors, and the 8 links and the clover entry
// once (shared by all right-hand sides).
static double launch_bytes_per_site(const lqcd_ctx* c, const DslashArgs& A, int mode, int epi, int nrhs)
{
    const int pg = mode_pg(mode), ps = mode_ps(mode);
    const double S = (double)spinor_field_bytes(ps, 1);
    const double L = (double)gauge_link_bytes(pg, c->recon_of(pg));
    const double Cl = A.clov ? (double)clover_site_bytes(pg) : 0.0;
    const double Acc = (double)spinor_field_bytes(AccumPrec(ps), 1);
    double per_rhs = S;
    switch (epi) {
    case EPI_NONE: per_rhs += S; break;
    case EPI_CLOVINV: per_rhs += S; break;
    case EPI_XPAY: per_rhs += 2 * S; break;
    default: per_rhs += 2 * S + 4 * Acc; break;  // y, p read; x, r read and written
    }
    return nrhs * per_rhs + 8 * L + (epi == EPI_NONE ? 0.0 : Cl);
}

lqcd_status launch_dslash(lqcd_ctx* c, const DslashArgs& A0, int P, bool dag, int epi, bool red, int nrhs)
{
    DslashArgs A = A0;
    if (red || epi == EPI_CG) A.sites_per_thread = c->tuned_spt[P][dag ? 1 : 0];
    int block = c->tuned_block[P][dag ? 1 : 0][red ? 1 : 0];
    if (block <= 0) block = c->block;
    const int rc = c->recon_of(mode_pg(P));
    Profiler* pr = c->prof;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (pr && pr->on) cudaStreamIsCapturing(c->stream, &cap);
    const bool timed = pr && pr->on && cap == cudaStreamCaptureStatusNone;
    Profiler::Rec rec{};
    if (timed) {
        rec.P = P;
        rec.a = pr->get();
        rec.b = pr->get();
        if (!rec.a || !rec.b) return fail(LQCD_ERR_CUDA, "profiler: cudaEventCreate failed");
        LQ_CUDA(cudaEventRecord(rec.a, c->stream));
    }
    cudaError_t e;
    switch (P) {
    case P64: e = dslash_dispatch_f64(A, rc, dag, epi, red, nrhs, block, c->stream); break;
    case P32: e = dslash_dispatch_f32(A, rc, dag, epi, red, nrhs, block, c->stream); break;
    case P16: e = dslash_dispatch_f16(A, rc, dag, epi, red, nrhs, block, c->stream); break;
    case PB16: e = dslash_dispatch_bf16(A, rc, dag, epi, red, nrhs, block, c->stream); break;
    case MODE_F16_LINKS: e = dslash_dispatch_f16links(A, rc, dag, epi, red, nrhs, block, c->stream); break;
    case MODE_BF16_LINKS: e = dslash_dispatch_bf16links(A, rc, dag, epi, red, nrhs, block, c->stream); break;
    case MODE_F16_SPINORS: e = dslash_dispatch_f16spinors(A, rc, dag, epi, red, nrhs, block, c->stream); break;
    case MODE_BF16_SPINORS: e = dslash_dispatch_bf16spinors(A, rc, dag, epi, red, nrhs, block, c->stream); break;
    default: return fail(LQCD_ERR_INVALID, "launch_dslash: bad precision mode");
    }
    LQ_CUDA(e);
    if (timed) {
        LQ_CUDA(cudaEventRecord(rec.b, c->stream));
        rec.bytes = launch_bytes_per_site(c, A, P, epi, nrhs) * c->g.Vh;
        rec.flops = 1320.0 * c->g.Vh * nrhs;
        pr->pending.push_back(rec);
    }
    c->dslash_count += nrhs;
    c->launches++;
    return LQCD_OK;
}

// out_p = epi(H_{p,1-p} in): thin wrapper filling DslashArgs.
lqcd_status op_hop(lqcd_ctx* c, void* out, const void* in, int parity, int P, bool dag, int epi, bool red,
                   const void* clov, const void* y, double a, int nrhs, size_t rb, int red_slot)
{
    DslashArgs A = base_args(c, P);
    A.par = parity;
    A.out = out;
    A.out_rb = rb;
    A.in = in;
    A.in_rb = rb;
    A.clov = clov;
    A.y = y;
    A.y_rb = rb;
    A.a = a;
    A.red = red ? c->scal + red_slot : nullptr;
    return launch_dslash(c, A, P, dag, epi, red, nrhs);
}

static const void* clover_ptr(lqcd_ctx* c, int P, int parity, bool inverse)
{
    if (c->clover_state == 0 || c->csw == 0.0) return nullptr;
    const int pg = mode_pg(P);
    const char* base = static_cast<const char*>(inverse ? c->clovinv[pg] : c->clov[pg]);
    return base + parity * c->clov_parity_bytes(pg);
}

// out_o = Mhat in_o = A_oo in_o - kappa^2 H_oe A_ee^{-1} H_eo in_o (dag: Mhat^dag)
lqcd_status op_schur(lqcd_ctx* c, void* out_o, const void* in_o, void* tmp_e, int P, bool dag, int nrhs, size_t rb,
                     size_t tmp_rb, int red_slot)
{
    DslashArgs A = base_args(c, P);
    A.par = 0;
    A.out = tmp_e;
    A.out_rb = tmp_rb;
    A.in = in_o;
    A.in_rb = rb;
    A.clov = clover_ptr(c, P, 0, true);
    A.a = 1.0;
    LQ_TRY(launch_dslash(c, A, P, dag, EPI_CLOVINV, false, nrhs));
    DslashArgs B = base_args(c, P);
    B.par = 1;
    B.out = out_o;
    B.out_rb = rb;
    B.in = tmp_e;
    B.in_rb = tmp_rb;
    B.clov = clover_ptr(c, P, 1, false);
    B.y = in_o;
    B.y_rb = rb;
    B.a = -c->kappa * c->kappa;
    B.red = red_slot >= 0 ? c->scal + red_slot : nullptr;
    return launch_dslash(c, B, P, dag, EPI_XPAY, red_slot >= 0, nrhs);
}

// out = M in on full fields (even then odd): out_p = A_pp in_p - kappa H_{p,1-p} in_{1-p}
lqcd_status op_full(lqcd_ctx* c, void* out, const void* in, int P, bool dag, int nrhs, size_t rb)
{
    const size_t fb = c->field_bytes(P);
    for (int par = 0; par < 2; ++par) {
        DslashArgs A = base_args(c, P);
        A.par = par;
        A.out = static_cast<char*>(out) + par * fb;
        A.out_rb = rb;
        A.in = static_cast<const char*>(in) + (1 - par) * fb;
        A.in_rb = rb;
        A.clov = clover_ptr(c, P, par, false);
        A.y = static_cast<const char*>(in) + par * fb;
        A.y_rb = rb;
        A.a = -c->kappa;
        LQ_TRY(launch_dslash(c, A, P, dag, EPI_XPAY, false, nrhs));
    }
    return LQCD_OK;
}

}  // namespace lqcd

using namespace lqcd;

#define LQ_GUARD_BEGIN try {
#define LQ_GUARD_END                                                      \
    }                                                                     \
    catch (const std::bad_alloc&) { return fail(LQCD_ERR_NOMEM, "host allocation failed"); } \
    catch (...) { return fail(LQCD_ERR_INVALID, "unexpected exception"); }

static lqcd_status check_ready(const lqcd_ctx* c)
{
    if (!c) return fail(LQCD_ERR_INVALID, "null context");
    if (!c->ws) return fail(LQCD_ERR_NOMEM, "no workspace: call lqcd_set_workspace");
    return LQCD_OK;
}


extern "C" {

const char* lqcd_last_error(void) { return g_last_error.c_str(); }

lqcd_status lqcd_create(const lqcd_config* cfg, void* stream, lqcd_ctx** out)
{
    LQ_GUARD_BEGIN
    if (!cfg || !out) return fail(LQCD_ERR_INVALID, "lqcd_create: null argument");
    *out = nullptr;
    long V = 1;
    for (int m = 0; m < 4; ++m) {
        if (cfg->dims[m] < 2 || (cfg->dims[m] & 1)) return fail(LQCD_ERR_INVALID, "lqcd_create: dims must be even and >= 2");
        V *= cfg->dims[m];
    }
    if (V / 2 > (1L << 30)) return fail(LQCD_ERR_INVALID, "lqcd_create: lattice too large");
    if (cfg->recon != 12 && cfg->recon != 18) return fail(LQCD_ERR_INVALID, "lqcd_create: recon must be 12 or 18");
    if (cfg->max_nrhs < 1 || cfg->max_nrhs > 64) return fail(LQCD_ERR_INVALID, "lqcd_create: max_nrhs must be in [1, 64]");
    if (cfg->gcr_nkrylov < 0 || cfg->gcr_nkrylov > 256)
        return fail(LQCD_ERR_INVALID, "lqcd_create: gcr_nkrylov must be in [0, 256]");
    int part = 0;
    for (int m = 0; m < 4; ++m) {
        const int pm = cfg->part[m] < 1 ? 1 : cfg->part[m];
        if (cfg->coord[m] < 0 || cfg->coord[m] >= pm)
            return fail(LQCD_ERR_INVALID, "lqcd_create: need 0 <= coord < part in every direction");
        if (pm > 1) part |= 1 << m;
    }
    lqcd_ctx* c = new lqcd_ctx();
    memset(c, 0, sizeof(*c));
    c->cfg = *cfg;
    c->cfg.prec_mask |= 1;  // F64 always held
    c->stream = static_cast<cudaStream_t>(stream);
    c->volume = V;
    for (int m = 0; m < 4; ++m) c->g.L[m] = cfg->dims[m];
    c->g.Lxh = cfg->dims[0] / 2;
    c->g.Vh = (int)(V / 2);
    c->g.stride = (c->g.Vh + 127) / 128 * 128;
    c->g.tanti = cfg->t_antiperiodic ? 1 : 0;
    c->g.part = part;
    c->g.tfirst = (part >> 3) & 1 ? (cfg->coord[3] == 0) : 1;
    c->g.tlast = (part >> 3) & 1 ? (cfg->coord[3] == cfg->part[3] - 1) : 1;
    c->block = DSLASH_MAX_BLOCK;
    if (const char* eb = getenv("LQCD_DSLASH_BLOCK")) {  // experiments: threads per dslash block
        const int b = atoi(eb);
        if (b >= 32 && b <= DSLASH_MAX_BLOCK && b % 32 == 0) c->block = b;
    }
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        cudaGetLastError();
        c->device = 0;
    }
    // workspace carve-up
    size_t off = 0;
    auto take = [&](lqcd_ctx::Slot& s, size_t bytes) {
        s.off = off;
        s.bytes = align256(bytes);
        off += s.bytes;
    };
    const int R = cfg->max_nrhs;
    for (int P = 0; P < 4; ++P) {
        if (!c->holds(P)) continue;
        take(c->s_gauge[P], 8 * c->gauge_parity_mu_bytes(P));
        take(c->s_clov[P], 2 * c->clov_parity_bytes(P));
        take(c->s_clovinv[P], 2 * c->clov_parity_bytes(P));
    }
    c->staging_bytes = (size_t)R * V * 192;
    const size_t slice = (size_t)V / cfg->dims[3] * 576;
    if (c->staging_bytes < slice) c->staging_bytes = slice;
    take(c->s_staging, c->staging_bytes);
    c->part_rs = (size_t)c->g.Vh / 32 + 64;
    take(c->s_partials, (size_t)R * c->part_rs * sizeof(double));
    take(c->s_tickets, (size_t)R * sizeof(unsigned));
    take(c->s_scal, (size_t)R * SC_PER_RHS * sizeof(double));
    take(c->s_errw, sizeof(int));
    take(c->s_skip, (size_t)R * sizeof(int));
    const size_t full64 = 2 * c->field_bytes(P64);
    take(c->s_vec64, (size_t)NV64 * R * full64);
    take(c->s_veclo, (size_t)NVLO * R * full64);
    take(c->s_vecacc, (size_t)NVACC * R * full64);
    // FGCR: z_0..z_{k-1}, w_0..w_{k-1}, r, x (FP32 full fields) + scalars and reduction partials
    // FGCR: 2K + 2 FP32 full fields; FGMRES-DR: V (K + 1), Z (K), r, x: 2K + 3;
    // then the scalars of the recursions (reduction partials, coefficients)
    c->gcr_bytes = cfg->gcr_nkrylov > 0 ? (size_t)(2 * cfg->gcr_nkrylov + 3) * 2 * c->field_bytes(P32) + GCR_SCALAR_BYTES
                                        : 0;
    take(c->s_gcr, c->gcr_bytes);
    take(c->s_persist, PERSIST_SCRATCH_BYTES);
    c->need = off;
    *out = c;
    return LQCD_OK;
    LQ_GUARD_END
}

lqcd_status lqcd_destroy(lqcd_ctx* c)
{
    if (c) delete c->prof;
    delete c;
    return LQCD_OK;
}

lqcd_status lqcd_profile_enable(lqcd_ctx* c, int enable)
{
    LQ_GUARD_BEGIN
    if (!c) return fail(LQCD_ERR_INVALID, "null context");
    if (!c->prof) c->prof = new Profiler();
    c->prof->on = enable != 0;
    return LQCD_OK;
    LQ_GUARD_END
}

lqcd_status lqcd_profile_read(lqcd_ctx* c, lqcd_profile_entry out[LQCD_NPREC])
{
    LQ_GUARD_BEGIN
    if (!c || !out) return fail(LQCD_ERR_INVALID, "lqcd_profile_read: null argument");
    for (int P = 0; P < LQCD_NPREC; ++P) out[P] = lqcd_profile_entry{0, 0.0, 0.0, 0.0};
    if (!c->prof) return LQCD_OK;
    LQ_CUDA(cudaStreamSynchronize(c->stream));
    for (auto& r : c->prof->pending) {
        float ms = 0.f;
        LQ_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
        out[r.P].launches += 1;
        out[r.P].ms += ms;
        out[r.P].bytes += r.bytes;
        out[r.P].flops += r.flops;
        c->prof->pool.push_back(r.a);
        c->prof->pool.push_back(r.b);
    }
    c->prof->pending.clear();
    return LQCD_OK;
    LQ_GUARD_END
}

lqcd_status lqcd_set_stream(lqcd_ctx* c, void* stream)
{
    if (!c) return fail(LQCD_ERR_INVALID, "null context");
    c->stream = static_cast<cudaStream_t>(stream);
    return LQCD_OK;
}

lqcd_status lqcd_workspace_size(const lqcd_ctx* c, size_t* bytes)
{
    if (!c || !bytes) return fail(LQCD_ERR_INVALID, "lqcd_workspace_size: null argument");
    *bytes = c->need;
    return LQCD_OK;
}

lqcd_status lqcd_set_workspace(lqcd_ctx* c, void* ptr, size_t bytes)
{
    LQ_GUARD_BEGIN
    if (!c || !ptr) return fail(LQCD_ERR_INVALID, "lqcd_set_workspace: null argument");
    if (bytes < c->need) return fail(LQCD_ERR_NOMEM, "lqcd_set_workspace: workspace smaller than lqcd_workspace_size");
    if (reinterpret_cast<uintptr_t>(ptr) & 255) return fail(LQCD_ERR_INVALID, "lqcd_set_workspace: base must be 256-byte aligned");
    if (!is_device_ptr(ptr)) return fail(LQCD_ERR_INVALID, "lqcd_set_workspace: not a device pointer");
    cudaPointerAttributes attr;
    LQ_CUDA(cudaPointerGetAttributes(&attr, ptr));
    c->device = attr.device;
    DeviceScope dev_scope;
    LQ_TRY(dev_scope.enter(c->device));
    c->ws = static_cast<char*>(ptr);
    c->ws_bytes = bytes;
    auto at = [&](const lqcd_ctx::Slot& s) -> char* { return s.bytes ? c->ws + s.off : nullptr; };
    for (int P = 0; P < 4; ++P) {
        c->gauge[P] = at(c->s_gauge[P]);
        c->clov[P] = at(c->s_clov[P]);
        c->clovinv[P] = at(c->s_clovinv[P]);
    }
    c->staging = at(c->s_staging);
    c->partials = reinterpret_cast<double*>(at(c->s_partials));
    c->tickets = reinterpret_cast<unsigned*>(at(c->s_tickets));
    c->scal = reinterpret_cast<double*>(at(c->s_scal));
    c->errw = reinterpret_cast<int*>(at(c->s_errw));
    c->skip = reinterpret_cast<int*>(at(c->s_skip));
    c->vec64 = at(c->s_vec64);
    c->veclo = at(c->s_veclo);
    c->vecacc = at(c->s_vecacc);
    c->gcr = at(c->s_gcr);
    c->persist = at(c->s_persist);
    LQ_CUDA(cudaMemsetAsync(c->tickets, 0, c->s_tickets.bytes, c->stream));
    LQ_CUDA(cudaMemsetAsync(c->errw, 0, c->s_errw.bytes, c->stream));
    LQ_CUDA(cudaMemsetAsync(c->skip, 0, c->s_skip.bytes, c->stream));
    LQ_CUDA(cudaMemsetAsync(c->scal, 0, c->s_scal.bytes, c->stream));
    c->gauge_loaded = 0;
    c->clover_state = 0;
    return LQCD_OK;
    LQ_GUARD_END
}

lqcd_status lqcd_field_bytes(const lqcd_ctx* c, lqcd_prec prec, size_t* bytes)
{
    if (!c || !bytes) return fail(LQCD_ERR_INVALID, "lqcd_field_bytes: null argument");
    if (!valid_mode(prec)) return fail(LQCD_ERR_INVALID, "lqcd_field_bytes: bad precision");
    *bytes = c->field_bytes(prec);
    return LQCD_OK;
}

lqcd_status lqcd_gauge_load(lqcd_ctx* c, const double* links)
{
    LQ_GUARD_BEGIN
    LQ_TRY(check_ready(c));
    if (!links) return fail(LQCD_ERR_INVALID, "lqcd_gauge_load: null links");
    DeviceScope dev_scope;
    LQ_TRY(dev_scope.enter(c->device));
    const int Lt = c->g.L[3];
    const size_t per_t = (size_t)c->volume / Lt * 72;  // doubles per t slice
    if (is_device_ptr(links)) {
        for (int P = 0; P < 4; ++P)
            if (c->holds(P)) LQ_TRY(gauge_pack(c, links, 0, Lt, P));
    } else {
        int nt = (int)(c->staging_bytes / (per_t * sizeof(double)));
        if (nt < 1) return fail(LQCD_ERR_NOMEM, "lqcd_gauge_load: staging too small");
        for (int t0 = 0; t0 < Lt; t0 += nt) {
            const int t1 = t0 + nt < Lt ? t0 + nt : Lt;
            LQ_CUDA(cudaMemcpyAsync(c->staging, links + (size_t)t0 * per_t, (size_t)(t1 - t0) * per_t * sizeof(double),
                                    cudaMemcpyHostToDevice, c->stream));
            for (int P = 0; P < 4; ++P)
                if (c->holds(P)) LQ_TRY(gauge_pack(c, static_cast<const double*>(c->staging), t0, t1, P));
        }
        LQ_CUDA(cudaStreamSynchronize(c->stream));  // staging is reused by the next call
    }
    c->gauge_loaded = 1;
    c->clover_state = 0;
    c->csw = 0.0;
    return LQCD_OK;
    LQ_GUARD_END
}

lqcd_status lqcd_clover_compute(lqcd_ctx* c, double kappa, double csw)
{
    LQ_GUARD_BEGIN
    LQ_TRY(check_ready(c));
    if (!c->gauge_loaded) return fail(LQCD_ERR_STATE, "lqcd_clover_compute: no gauge field loaded");
    if (!(kappa > 0.0) || !(csw >= 0.0)) return fail(LQCD_ERR_INVALID, "lqcd_clover_compute: need kappa > 0, csw >= 0");
    if (c->cut() && csw != 0.0)
        return fail(LQCD_ERR_STATE, "lqcd_clover_compute: the clover leaves of a sub-domain need its neighbours' links "
                                    "(csw = 0 only)");
    DeviceScope dev_scope;
    LQ_TRY(dev_scope.enter(c->device));
    c->kappa = kappa;
    c->csw = csw;
    if (csw == 0.0) {
        c->clover_state = 1;
        return LQCD_OK;
    }
    LQ_CUDA(cudaMemsetAsync(c->errw, 0, sizeof(int), c->stream));
    LQ_TRY(clover_build(c, kappa, csw));
    int err = 0;
    LQ_CUDA(cudaMemcpyAsync(&err, c->errw, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    LQ_CUDA(cudaStreamSynchronize(c->stream));
    c->clover_state = 1;
    if (err & ERRW_CLOVER_SINGULAR) return fail(LQCD_ERR_CLOVER_SINGULAR, "lqcd_clover_compute: singular clover block");
    return LQCD_OK;
    LQ_GUARD_END
}

static lqcd_status check_prec(const lqcd_ctx* c, int prec)
{
    if (!valid_mode(prec)) return fail(LQCD_ERR_INVALID, "bad precision");
    if (!c->holds(mode_pg(prec))) return fail(LQCD_ERR_STATE, "precision not held by this context (cfg.prec_mask)");
    return LQCD_OK;
}

static lqcd_status pack_common(lqcd_ctx* c, void* internal, double* canonical, int parity, int prec, int nrhs,
                               bool unpack)
{
    LQ_TRY(check_ready(c));
    LQ_TRY(check_prec(c, prec));
    if (!internal || !canonical) return fail(LQCD_ERR_INVALID, "pack: null pointer");
    if (parity < -1 || parity > 1) return fail(LQCD_ERR_INVALID, "pack: parity must be -1, 0 or 1");
    if (nrhs < 1) return fail(LQCD_ERR_INVALID, "pack: nrhs must be >= 1");
    if (!is_device_ptr(internal)) return fail(LQCD_ERR_INVALID, "pack: internal field must be device memory");
    DeviceScope dev_scope;
    LQ_TRY(dev_scope.enter(c->device));
    const size_t canon_rb = (size_t)c->volume * 192;
    const size_t int_rb = (parity < 0 ? 2 : 1) * c->field_bytes(prec);
    if (is_device_ptr(canonical)) {
        return unpack ? unpack_spinor(c, canonical, internal, parity, mode_ps(prec), nrhs, int_rb, canon_rb)
                      : pack_spinor(c, internal, canonical, parity, mode_ps(prec), nrhs, int_rb, canon_rb);
    }
    // host canonical: go through the staging area in chunks of right-hand sides
    const int per = (int)(c->staging_bytes / canon_rb);
    if (per < 1) return fail(LQCD_ERR_NOMEM, "pack: staging too small");
    for (int r0 = 0; r0 < nrhs; r0 += per) {
        const int n = nrhs - r0 < per ? nrhs - r0 : per;
        char* in = static_cast<char*>(internal) + r0 * int_rb;
        if (unpack) {
            LQ_TRY(unpack_spinor(c, static_cast<double*>(c->staging), in, parity, mode_ps(prec), n, int_rb, canon_rb));
            LQ_CUDA(cudaMemcpyAsync(canonical + (size_t)r0 * canon_rb / 8, c->staging, n * canon_rb,
                                    cudaMemcpyDeviceToHost, c->stream));
        } else {
            LQ_CUDA(cudaMemcpyAsync(c->staging, canonical + (size_t)r0 * canon_rb / 8, n * canon_rb,
                                    cudaMemcpyHostToDevice, c->stream));
            LQ_TRY(pack_spinor(c, in, static_cast<const double*>(c->staging), parity, mode_ps(prec), n, int_rb, canon_rb));
        }
        LQ_CUDA(cudaStreamSynchronize(c->stream));
    }
    return LQCD_OK;
}

lqcd_status lqcd_pack(lqcd_ctx* c, void* internal, const double* canonical, int parity, lqcd_prec prec, int nrhs)
{
    LQ_GUARD_BEGIN
    return pack_common(c, internal, const_cast<double*>(canonical), parity, prec, nrhs, false);
    LQ_GUARD_END
}

lqcd_status lqcd_unpack(lqcd_ctx* c, double* canonical, const void* internal, int parity, lqcd_prec prec, int nrhs)
{
    LQ_GUARD_BEGIN
    return pack_common(c, const_cast<void*>(internal), canonical, parity, prec, nrhs, true);
    LQ_GUARD_END
}

lqcd_status lqcd_dslash(lqcd_ctx* c, void* out, const void* in, int parity, double kappa, double csw, int op_flags,
                        lqcd_prec prec, int nrhs)
{
    LQ_GUARD_BEGIN
    LQ_TRY(check_ready(c));
    LQ_TRY(check_prec(c, prec));
    if (!out || !in) return fail(LQCD_ERR_INVALID, "lqcd_dslash: null field");
    if (c->cut()) return fail(LQCD_ERR_STATE, "lqcd_dslash: not on a sub-domain of a cut lattice (use lqcd_halo_*)");
    if (out == in) return fail(LQCD_ERR_INVALID, "lqcd_dslash: out must not alias in");
    if (nrhs < 1) return fail(LQCD_ERR_INVALID, "lqcd_dslash: nrhs must be >= 1");
    if (!c->gauge_loaded) return fail(LQCD_ERR_STATE, "lqcd_dslash: no gauge field loaded");
    const int op = op_flags & 0xff;
    const bool dag = (op_flags & LQCD_DAG) != 0;
    if ((op_flags & ~(0xff | LQCD_DAG)) != 0 || op > LQCD_OP_FULL) return fail(LQCD_ERR_INVALID, "lqcd_dslash: bad op_flags");
    DeviceScope dev_scope;
    LQ_TRY(dev_scope.enter(c->device));
    const size_t fb = c->field_bytes(prec);
    if (op == LQCD_OP_HOP) {
        if (parity != 0 && parity != 1) return fail(LQCD_ERR_INVALID, "lqcd_dslash: parity must be 0 or 1");
        return op_hop(c, out, in, parity, prec, dag, EPI_NONE, false, nullptr, nullptr, 1.0, nrhs, fb, -1);
    }
    // operators with kappa / csw: must match the clover state
    const double have_csw = c->clover_state ? c->csw : 0.0;
    if (csw != have_csw) return fail(LQCD_ERR_STATE, "lqcd_dslash: csw differs from lqcd_clover_compute");
    if (csw != 0.0 && kappa != c->kappa) return fail(LQCD_ERR_STATE, "lqcd_dslash: kappa differs from lqcd_clover_compute");
    if (!(kappa > 0.0)) return fail(LQCD_ERR_INVALID, "lqcd_dslash: kappa must be > 0");
    if (nrhs > c->cfg.max_nrhs) return fail(LQCD_ERR_INVALID, "lqcd_dslash: nrhs exceeds cfg.max_nrhs");
    const double saved = c->kappa;
    c->kappa = kappa;
    lqcd_status st;
    if (op == LQCD_OP_SCHUR) {
        if (parity != 1) {
            c->kappa = saved;
            return fail(LQCD_ERR_INVALID, "lqcd_dslash: the Schur operator acts on odd sites (parity 1)");
        }
        // the even intermediate lives in the context's FP64 scratch vectors
        st = op_schur(c, out, in, vec64_field(c, 5, 0), prec, dag, nrhs, fb, fb, -1);
    } else {
        st = op_full(c, out, in, prec, dag, nrhs, 2 * fb);
    }
    c->kappa = saved;
    return st;
    LQ_GUARD_END
}

lqcd_status lqcd_training_pair(lqcd_ctx* c, float* r, float* e, const double* xstar, const double* x, int nrhs)
{
    LQ_GUARD_BEGIN
    LQ_TRY(check_ready(c));
    if (!r || !e || !xstar) return fail(LQCD_ERR_INVALID, "lqcd_training_pair: null field");
    if (c->cut()) return fail(LQCD_ERR_STATE, "lqcd_training_pair: not on a sub-domain of a cut lattice (use lqcd_halo_*)");
    if (nrhs < 1) return fail(LQCD_ERR_INVALID, "lqcd_training_pair: nrhs must be >= 1");
    if (!c->gauge_loaded || !c->clover_state)
        return fail(LQCD_ERR_STATE, "lqcd_training_pair: load the gauge field and call lqcd_clover_compute first");
    if (!is_device_ptr(r) || !is_device_ptr(e) || !is_device_ptr(xstar) || (x && !is_device_ptr(x)))
        return fail(LQCD_ERR_INVALID, "lqcd_training_pair: every field must be device memory");
    DeviceScope dev_scope;
    LQ_TRY(dev_scope.enter(c->device));
    const size_t canon_rb = (size_t)c->volume * 192, canon32_rb = (size_t)c->volume * 96;
    const size_t full_rb = 2 * c->field_bytes(P64);
    char* e_int = vec64_field(c, 0, 0);  // max_nrhs full FP64 fields each
    char* r_int = vec64_field(c, 1, 0);
    for (int r0 = 0; r0 < nrhs; r0 += c->cfg.max_nrhs) {
        const int n = nrhs - r0 < c->cfg.max_nrhs ? nrhs - r0 : c->cfg.max_nrhs;
        const double* xs = xstar + (size_t)r0 * canon_rb / sizeof(double);
        const double* xx = x ? x + (size_t)r0 * canon_rb / sizeof(double) : nullptr;
        LQ_TRY(pack_difference(c, e_int, xs, xx, n, full_rb, canon_rb));
        LQ_TRY(op_full(c, r_int, e_int, P64, false, n, full_rb));
        LQ_TRY(unpack_spinor_f32(c, e + (size_t)r0 * canon32_rb / sizeof(float), e_int, n, full_rb, canon32_rb));
        LQ_TRY(unpack_spinor_f32(c, r + (size_t)r0 * canon32_rb / sizeof(float), r_int, n, full_rb, canon32_rb));
    }
    return LQCD_OK;
    LQ_GUARD_END
}

lqcd_status lqcd_clover_apply(lqcd_ctx* c, void* out, const void* in, int parity, int inverse, lqcd_prec prec, int nrhs)
{
    LQ_GUARD_BEGIN
    LQ_TRY(check_ready(c));
    LQ_TRY(check_prec(c, prec));
    if (!out || !in) return fail(LQCD_ERR_INVALID, "lqcd_clover_apply: null field");
    if (parity != 0 && parity != 1) return fail(LQCD_ERR_INVALID, "lqcd_clover_apply: parity must be 0 or 1");
    if (nrhs < 1) return fail(LQCD_ERR_INVALID, "lqcd_clover_apply: nrhs must be >= 1");
    if (!c->clover_state || c->csw == 0.0) return fail(LQCD_ERR_STATE, "lqcd_clover_apply: no clover term computed");
    DeviceScope dev_scope;
    LQ_TRY(dev_scope.enter(c->device));
    return clover_apply_launch(c, out, in, parity, inverse ? 1 : 0, prec, nrhs, c->field_bytes(prec));
    LQ_GUARD_END
}

lqcd_status lqcd_sync(lqcd_ctx* c)
{
    LQ_GUARD_BEGIN
    LQ_TRY(check_ready(c));
    DeviceScope dev_scope;
    LQ_TRY(dev_scope.enter(c->device));
    int err = 0;
    LQ_CUDA(cudaMemcpyAsync(&err, c->errw, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    LQ_CUDA(cudaStreamSynchronize(c->stream));
    if (err) LQ_CUDA(cudaMemsetAsync(c->errw, 0, sizeof(int), c->stream));  // reported once
    if (err & ERRW_CLOVER_SINGULAR) return fail(LQCD_ERR_CLOVER_SINGULAR, "singular clover block");
    if (err & ERRW_BREAKDOWN) return fail(LQCD_ERR_BREAKDOWN, "solver breakdown");
    if (err & ERRW_TIMEOUT) return fail(LQCD_ERR_TIMEOUT, "a bounded device wait expired");
    return LQCD_OK;
    LQ_GUARD_END
}

lqcd_status lqcd_solve_batch(lqcd_ctx* const* ctxs, int n, double* const* x, const double* const* b,
                             const double* tol, const lqcd_solver_params* params, lqcd_solver_stats* stats)
{
    NvtxRange nvtx_range("lqcd_solve_batch");
    LQ_GUARD_BEGIN
    if (!ctxs || !x || !b || !tol || !stats || n < 1) return fail(LQCD_ERR_INVALID, "lqcd_solve_batch: bad argument");
    lqcd_solver_params p;
    if (params) p = *params;
    else lqcd_solver_params_default(&p);
    for (int i = 0; i < n; ++i) {
        lqcd_ctx* c = ctxs[i];
        LQ_TRY(check_ready(c));
        if (!x[i] || !b[i] || !(tol[i] > 0.0)) return fail(LQCD_ERR_INVALID, "lqcd_solve_batch: bad vector or tol");
        if (!c->gauge_loaded || !c->clover_state) return fail(LQCD_ERR_STATE, "lqcd_solve_batch: gauge and clover first");
        if (c->device != ctxs[0]->device) return fail(LQCD_ERR_INVALID, "lqcd_solve_batch: contexts on different GPUs");
        if (c->cut()) return fail(LQCD_ERR_STATE, "lqcd_solve_batch: not on a sub-domain of a cut lattice");
        LQ_TRY(check_prec(c, p.inner_prec));
        memset(&stats[i], 0, sizeof(stats[i]));
    }
    DeviceScope dev_scope;
    LQ_TRY(dev_scope.enter(ctxs[0]->device));
    return solve_batch(ctxs, n, x, b, tol, &p, stats);
    LQ_GUARD_END
}

lqcd_status lqcd_tune(lqcd_ctx* c, lqcd_prec prec, int best_block[4], int best_sites[2])
{
    NvtxRange nvtx_range("lqcd_tune");
    LQ_GUARD_BEGIN
    LQ_TRY(check_ready(c));
    LQ_TRY(check_prec(c, prec));
    if (!c->gauge_loaded) return fail(LQCD_ERR_STATE, "lqcd_tune: no gauge field loaded");
    if (c->cut()) return fail(LQCD_ERR_STATE, "lqcd_tune: not on a sub-domain of a cut lattice (use lqcd_halo_*)");
    DeviceScope dev_scope;
    LQ_TRY(dev_scope.enter(c->device));
    // scratch: two full fields of the FP64-sized solver vectors, filled with
    // a non-zero byte pattern (finite in every storage format)
    const size_t fb = c->field_bytes(prec);
    char* in = vec64_field(c, 0, 0);
    char* out = vec64_field(c, 1, 0);
    LQ_CUDA(cudaMemsetAsync(in, 0x3c, 2 * fb, c->stream));
    cudaEvent_t e0, e1;
    LQ_CUDA(cudaEventCreate(&e0));
    LQ_CUDA(cudaEventCreate(&e1));
    lqcd_status st = LQCD_OK;
    // time of 5 launches after one warm-up of the current setting
    auto time_launches = [&](int dag, int red, float& ms) {
        ms = 0.f;
        for (int rep = 0; rep < 6 && st == LQCD_OK; ++rep) {  // rep 0 warms up
            if (cudaEventRecord(e0, c->stream) != cudaSuccess) st = fail(LQCD_ERR_CUDA, "lqcd_tune: event");
            if (st == LQCD_OK)
                st = op_hop(c, out + fb, in, 1, prec, dag != 0, EPI_XPAY, red != 0, nullptr, in + fb, -0.1, 1, fb,
                            red ? SC_TMP + 7 : -1);
            if (st == LQCD_OK && cudaEventRecord(e1, c->stream) != cudaSuccess) st = fail(LQCD_ERR_CUDA, "lqcd_tune: event");
            if (st == LQCD_OK && cudaEventSynchronize(e1) != cudaSuccess) st = fail(LQCD_ERR_CUDA, "lqcd_tune: sync");
            float t = 0.f;
            if (st == LQCD_OK && rep > 0 && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess) ms += t;
        }
    };
    const int cands[5] = {128, 96, 64, 32, DSLASH_STAGED};  // the default first: it wins ties
    // the staged kernel competes in the plain classes where it applies
    const bool staged_ok = mode_pg(prec) == P32 && c->recon_of(P32) == 12 && staged_supported(c->g);
    const int spts[4] = {0, 1, 4, 16};       // sites per thread of reducing launches (0: one wave of blocks)
    // reducing launches (fused norms, fused CG updates) write one partial sum
    // per block, so they are tuned apart from the plain ones, and for them
    // the sites per thread as well
    for (int dag = 0; dag < 2 && st == LQCD_OK; ++dag)
        for (int red = 0; red < 2 && st == LQCD_OK; ++red) {
            float best = 1e30f;
            int best_b = c->block;
            if (red) c->tuned_spt[prec][dag] = 0;
            for (int ci = 0; ci < 5 && st == LQCD_OK; ++ci) {
                if (ci == 4 && (red || !staged_ok)) break;
                c->tuned_block[prec][dag][red] = cands[ci];
                float ms = 0.f;
                time_launches(dag, red, ms);
                // a smaller block has to be faster by 2 % to replace the larger one
                if (st == LQCD_OK && ms < 0.98f * best) {
                    best = ms;
                    best_b = cands[ci];
                }
            }
            c->tuned_block[prec][dag][red] = best_b;
            if (best_block) best_block[2 * dag + red] = best_b;
            if (red) {
                int best_s = 0;
                for (int si = 1; si < 4 && st == LQCD_OK; ++si) {
                    c->tuned_spt[prec][dag] = spts[si];
                    float ms = 0.f;
                    time_launches(dag, red, ms);
                    if (st == LQCD_OK && ms < 0.98f * best) {
                        best = ms;
                        best_s = spts[si];
                    }
                }
                c->tuned_spt[prec][dag] = best_s;
                if (best_sites) best_sites[dag] = best_s;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
    LQ_GUARD_END
}

static_assert(DSLASH_STAGED == LQCD_BLOCK_STAGED, "the staged kernel's block-size code is part of the ABI");

lqcd_status lqcd_tune_set(lqcd_ctx* c, lqcd_prec prec, const int block[4], const int sites[2])
{
    LQ_GUARD_BEGIN
    LQ_TRY(check_ready(c));
    LQ_TRY(check_prec(c, prec));
    if (!block) return fail(LQCD_ERR_INVALID, "lqcd_tune_set: null block");
    for (int k = 0; k < 4; ++k) {
        const int b = block[k];
        const bool plain = (k & 1) == 0;
        if (!(b == 32 || b == 64 || b == 96 || b == 128 || (plain && b == DSLASH_STAGED)))
            return fail(LQCD_ERR_INVALID, "lqcd_tune_set: block must be 32, 64, 96, 128 or (plain classes) "
                                          "LQCD_BLOCK_STAGED");
    }
    if (sites)
        for (int d = 0; d < 2; ++d)
            if (sites[d] < 0 || sites[d] > 64) return fail(LQCD_ERR_INVALID, "lqcd_tune_set: sites per thread out of range");
    for (int dag = 0; dag < 2; ++dag)
        for (int red = 0; red < 2; ++red) c->tuned_block[prec][dag][red] = block[2 * dag + red];
    if (sites)
        for (int d = 0; d < 2; ++d) c->tuned_spt[prec][d] = sites[d];
    return LQCD_OK;
    LQ_GUARD_END
}

lqcd_status lqcd_set_preconditioner(lqcd_ctx* c, lqcd_net* net)
{
    if (!c) return fail(LQCD_ERR_INVALID, "null context");
    c->precond = net;
    if (net) c->sap_on = 0;
    return LQCD_OK;
}

lqcd_status lqcd_solver_params_default(lqcd_solver_params* p)
{
    if (!p) return fail(LQCD_ERR_INVALID, "null params");
    p->solver = LQCD_SOLVER_CG_EO;
    p->inner_prec = LQCD_F32;
    p->maxiter = 100000;
    p->reliable_interval = 50;
    p->reliable_delta = 0.1;
    p->check_interval = 10;
    p->nkrylov = 20;
    p->use_graph = 0;
    p->ndefl = 0;
    p->persistent = 0;
    p->persistent_wait_us = 0;
    p->residual_prec = LQCD_F64;
    return LQCD_OK;
}

lqcd_status lqcd_solve(lqcd_ctx* c, double* x, const double* b, double tol, int nrhs, const lqcd_solver_params* params,
                       lqcd_solver_stats* stats)
{
    NvtxRange nvtx_range("lqcd_solve");
    LQ_GUARD_BEGIN
    LQ_TRY(check_ready(c));
    if (!x || !b) return fail(LQCD_ERR_INVALID, "lqcd_solve: null vector");
    if (c->cut()) return fail(LQCD_ERR_STATE, "lqcd_solve: not on a sub-domain of a cut lattice (use lqcd_halo_*)");
    if (nrhs < 1 || nrhs > c->cfg.max_nrhs) return fail(LQCD_ERR_INVALID, "lqcd_solve: nrhs out of range");
    if (!(tol > 0.0)) return fail(LQCD_ERR_INVALID, "lqcd_solve: tol must be > 0");
    if (!c->gauge_loaded) return fail(LQCD_ERR_STATE, "lqcd_solve: no gauge field loaded");
    if (!c->clover_state) return fail(LQCD_ERR_STATE, "lqcd_solve: call lqcd_clover_compute first (csw = 0 allowed)");
    lqcd_solver_params p;
    if (params) p = *params;
    else lqcd_solver_params_default(&p);
    LQ_TRY(check_prec(c, p.inner_prec));
    DeviceScope dev_scope;
    LQ_TRY(dev_scope.enter(c->device));
    lqcd_solver_stats st;
    memset(&st, 0, sizeof(st));
    lqcd_status r = solve(c, x, b, tol, nrhs, &p, &st);
    if (stats) *stats = st;
    return r;
    LQ_GUARD_END
}

}  // extern "C"
