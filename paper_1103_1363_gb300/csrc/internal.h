// Host-side internals shared by the library's translation units: the
// context, its workspace carve-up, error reporting and the launchers each
// unit exports.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stddef.h>
#include <stdint.h>
#include <string>

#include "../../include/lqcd.h"
#include "core.cuh"
#include "dslash_impl.cuh"

namespace lqcd {

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
lqcd_status fail(lqcd_status st, const std::string& msg);
lqcd_status cuda_fail(cudaError_t e, const char* where);
#define LQ_CUDA(call)                                                   \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) return ::lqcd::cuda_fail(e_, #call);    \
    } while (0)
#define LQ_TRY(call)                                        \
    do {                                                    \
        lqcd_status s_ = (call);                            \
        if (s_ != LQCD_OK) return s_;                       \
    } while (0)

// Makes a device current for the lifetime of the object and gives the
// calling thread its previous current device back on destruction, so that
// an entry point never leaves the caller on another GPU.
// A named NVTX range over a host-side phase (a solve, an iteration block, a
// network step) for timeline tools; without a tool attached the calls do
// nothing but test for one.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

struct DeviceScope {
    int prev = -1;
    lqcd_status enter(int device)
    {
        int cur = -1;
        LQ_CUDA(cudaGetDevice(&cur));
        if (cur != device) {
            LQ_CUDA(cudaSetDevice(device));
            prev = cur;
        }
        return LQCD_OK;
    }
    ~DeviceScope()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
    DeviceScope() = default;
    DeviceScope(const DeviceScope&) = delete;
    DeviceScope& operator=(const DeviceScope&) = delete;
};

// device error word bits
enum { ERRW_CLOVER_SINGULAR = 1, ERRW_BREAKDOWN = 2, ERRW_TIMEOUT = 4 };

// Scalar slots per right-hand side (doubles).  The CG keeps rings of
// |r|^2 and |M p|^2 values, one (even, odd) pair per iteration, so that
// every kernel reads the slots of its own iteration and the host never
// has to intervene between kernels.
enum {
    SC_RING = 32,       // iterations held by each ring
    SC_RR = 0,          // |r|^2 ring: slots SC_RR + 2*(k % SC_RING) + parity
    SC_PAP = 64,        // |M p|^2 ring: slots SC_PAP + 2*(k % SC_RING) + parity
    SC_TMP = 128,       // scratch reductions [128, 160)
    SC_PER_RHS = 160
};
inline int rr_slot(int k) { return SC_RR + 2 * (k % SC_RING); }
inline int pap_slot(int k) { return SC_PAP + 2 * (k % SC_RING); }

// dslash launch (dispatch by precision); block = threads per block
cudaError_t dslash_dispatch_f64(const DslashArgs&, int, bool, int, bool, int, int, cudaStream_t);
cudaError_t dslash_dispatch_f32(const DslashArgs&, int, bool, int, bool, int, int, cudaStream_t);
cudaError_t dslash_dispatch_f16(const DslashArgs&, int, bool, int, bool, int, int, cudaStream_t);
cudaError_t dslash_dispatch_bf16(const DslashArgs&, int, bool, int, bool, int, int, cudaStream_t);
cudaError_t dslash_dispatch_f16links(const DslashArgs&, int, bool, int, bool, int, int, cudaStream_t);
cudaError_t dslash_dispatch_bf16links(const DslashArgs&, int, bool, int, bool, int, int, cudaStream_t);
cudaError_t dslash_dispatch_f16spinors(const DslashArgs&, int, bool, int, bool, int, int, cudaStream_t);
cudaError_t dslash_dispatch_bf16spinors(const DslashArgs&, int, bool, int, bool, int, int, cudaStream_t);

struct Profiler;  // api.cu: CUDA-event timing of hopping-term launches

// ---- persistent even-odd CG (persistent.cu)
// Work of a stage: every (lattice, rhs) pair is cut into tiles of
// PERSIST_THREADS x spt sites (spt sites per thread, so that a pair has at
// most PERSIST_MAX_TILES tiles); the tiles of all pairs are spread over the
// grid in one pass.
enum { PERSIST_THREADS = 128, PERSIST_MAXL = 8, PERSIST_MAXPAIRS = 64, PERSIST_MAX_TILES = 1024,
       PERSIST_MAX_GRID = 2048 };
// workspace bytes of the persistent launch's reduction partials (one per
// tile), tickets, barrier words and abort word (in the first context of a solve)
enum : size_t {
    PERSIST_SCRATCH_BYTES = (size_t)PERSIST_MAXPAIRS * PERSIST_MAX_TILES * sizeof(double) + 4096
};

// One lattice's part of a persistent iteration block.  Inside the block
// the |r|^2 slots form a ring of two (iteration j reads slot j mod 2 and
// writes (j + 1) mod 2) and |Mhat p|^2 uses one slot, so the stage
// arguments of even and odd iterations are fixed and set by the host.
struct PersistLattice {
    DslashArgs d[2][4];    // [j mod 2][stage]: the four hopping stages of an iteration
    Geom g;
    int R;                 // right-hand sides
    int pair0;             // index of the lattice's first (lattice, rhs) reduction slot
    int spt;               // sites per thread of the lattice's tiles
    int ntiles;            // tiles per right-hand side
    char* p;               // p_o (inner storage), rhs stride p_rb
    size_t p_rb;
    const char* r;         // r_o (FP32 accumulation), rhs stride r_rb
    size_t r_rb;
    double* scal;          // per-rhs scalar slots (stride SC_PER_RHS)
    const int* skip;       // per-rhs converged flags
};

struct PersistArgs {
    int nlat;
    int npairs;
    int tile0[PERSIST_MAXPAIRS + 1];        // first tile of each pair; tile0[npairs] = all tiles
    unsigned char pair_lat[PERSIST_MAXPAIRS];
    unsigned char pair_rhs[PERSIST_MAXPAIRS];
    int niter;             // iterations of the block
    int last_p;            // 1: the block's last iteration also updates p (no reliable update follows)
    int copy_slots;        // 1: at the end, |r|^2 slot 0 <- slot niter
    double* partials;      // [pair][gridDim.x]
    unsigned* tickets;     // [pair]
    unsigned* bar;         // [0] arrivals, [1] generation
    int* abort;            // raised by a block whose barrier wait expired
    int* errw;             // error word of the first context
    unsigned long long wait_ns;
    PersistLattice lat[PERSIST_MAXL];
};
bool persist_supported(int mode);
// blocks of the persistent launch for ntiles tiles in all
lqcd_status persist_grid(int mode, int recon, int ntiles, int* grid);
lqcd_status launch_persist(lqcd_ctx* c0, const PersistArgs& P, int mode, int recon, int grid);

}  // namespace lqcd

struct lqcd_ctx {
    lqcd::Profiler* prof;    // null unless lqcd_profile_enable was called
    lqcd_net* precond;       // FGCR right preconditioner (null: identity or SAP)
    int sap_on;              // FGCR right preconditioner is SAP (sap_bs, sap_ncycle, sap_nmr)
    int sap_bs[4], sap_ncycle, sap_nmr;
    lqcd_config cfg;
    lqcd::Geom g;
    cudaStream_t stream;
    long volume;  // V
    int device;

    // workspace carve-up (offsets fixed at create, pointers at set_workspace)
    char* ws;
    size_t ws_bytes;
    size_t need;
    struct Slot { size_t off, bytes; };
    Slot s_gauge[4], s_clov[4], s_clovinv[4];
    Slot s_staging, s_partials, s_tickets, s_scal, s_errw, s_skip, s_vec64, s_veclo, s_vecacc, s_gcr, s_persist;
    void* gauge[4];          // per precision copy, layout [parity][mu][chunk][stride]
    void* clov[4];           // A, layout [parity][chunk][stride] (parity stride clov_pb[p])
    void* clovinv[4];
    void* staging;
    size_t staging_bytes;
    double* partials;        // per rhs: part_rs doubles
    size_t part_rs;
    unsigned* tickets;       // per rhs, SC_PER_RHS tickets (one per scalar slot)
    double* scal;            // per rhs SC_PER_RHS doubles
    int* errw;               // device error word
    int* skip;               // per rhs converged flags
    char* vec64;             // FP64 solver vectors: NV64 full fields x max_nrhs
    char* veclo;             // inner-precision vectors (sized for F32 and below)
    char* vecacc;            // accumulation vectors (x_lo, r): FP64-sized
    char* gcr;               // FGCR Krylov vectors
    size_t gcr_bytes;
    char* persist;           // persistent CG launch: reduction partials, tickets, barrier and abort words

    // state
    int gauge_loaded;
    int clover_state;        // 0 none, 1 built
    double kappa, csw;
    int block;               // threads per block of the dslash kernels
    long dslash_count;
    long launches;           // kernels launched by this context (all kinds)
    // tuned threads per block: [precision mode][dag][launch reduces into a scalar] (0 = default)
    int tuned_block[lqcd::NMODES][2][2];
    // tuned sites per thread of the reducing launches: [precision mode][dag] (0 = one wave of blocks)
    int tuned_spt[lqcd::NMODES][2];

    // bytes of one single-parity spinor field of precision mode m
    size_t field_bytes(int m) const { return lqcd::spinor_field_bytes(lqcd::mode_ps(m), g.stride); }
    size_t clov_parity_bytes(int P) const { return (size_t)g.stride * lqcd::clover_site_bytes(P); }
    size_t gauge_parity_mu_bytes(int P) const
    {
        return (size_t)g.stride * lqcd::gauge_link_bytes(P, P == lqcd::P64 ? 18 : cfg.recon);
    }
    int recon_of(int P) const { return P == lqcd::P64 ? 18 : cfg.recon; }
    // is this context a sub-domain of a cut lattice?
    bool cut() const { return g.part != 0; }
    // does the context hold links and clover for storage precision P (0..3)?
    bool holds(int P) const { return P == lqcd::P64 || (cfg.prec_mask >> P) & 1; }
};

namespace lqcd {

// bytes after the FP32 fields of the FGCR / FGMRES-DR region: reduction
// partials, dot products and coefficient arrays of the recursions
enum : size_t { GCR_SCALAR_BYTES = (size_t)4 << 20 };

// number of full (both-parity) FP64 fields per rhs in vec64
enum { NV64 = 6 };
// inner-precision full fields per rhs in veclo
enum { NVLO = 3 };
// accumulation full fields per rhs in vecacc
enum { NVACC = 2 };

// field helpers: full field = even then odd
inline char* vec64_field(lqcd_ctx* c, int which, int rhs)
{
    return c->vec64 + ((size_t)which * c->cfg.max_nrhs + rhs) * 2 * c->field_bytes(P64);
}

// ---- launchers exported by the translation units (all asynchronous on s)
// fields.cu
lqcd_status pack_spinor(lqcd_ctx* c, void* internal, const double* canon_dev, int parity, int P, int nrhs,
                        size_t internal_rb, size_t canon_rb);
lqcd_status unpack_spinor(lqcd_ctx* c, double* canon_dev, const void* internal, int parity, int P, int nrhs,
                          size_t internal_rb, size_t canon_rb);
// full FP64 internal fields = canonical a - b (b null: a); and full FP64
// internal fields -> canonical FP32 complex spinors
lqcd_status pack_difference(lqcd_ctx* c, void* internal, const double* a, const double* b, int nrhs,
                            size_t internal_rb, size_t canon_rb);
lqcd_status unpack_spinor_f32(lqcd_ctx* c, float* canon, const void* internal, int nrhs, size_t internal_rb,
                              size_t canon_rb);
lqcd_status gauge_pack(lqcd_ctx* c, const double* canon_dev_slice, int t0, int t1, int P);
lqcd_status convert_field(lqcd_ctx* c, void* out, int Pout, const void* in, int Pin, int nrhs, size_t out_rb,
                          size_t in_rb, int nf, int norm_slot /* -1: no norm */);
// clover.cu
lqcd_status clover_build(lqcd_ctx* c, double kappa, double csw);
// blas.cu
// nf: 1 = single-parity fields, 2 = full fields (even then odd)
lqcd_status blas_norm2(lqcd_ctx* c, const void* x, int P, int nrhs, size_t rb, int nf, int slot);
lqcd_status blas_xmy_norm(lqcd_ctx* c, void* out, const void* b, const void* a, int P, int nrhs, size_t rb, int nf,
                          int slot);
lqcd_status blas_cg_p_update(lqcd_ctx* c, void* p, int Pp, const void* r, int Pr, int nrhs, size_t p_rb,
                             size_t r_rb, int nf, int s_num, int s_den);
lqcd_status blas_accumulate_x(lqcd_ctx* c, void* xhi, const void* xlo, int Plo, int nrhs, size_t hi_rb,
                              size_t lo_rb, int nf);
lqcd_status blas_zero(lqcd_ctx* c, void* x, int P, int nrhs, size_t rb, int nf);
lqcd_status blas_copy_scalar(lqcd_ctx* c, int dst_slot, int src_slot, int nrhs);
lqcd_status clover_apply_launch(lqcd_ctx* c, void* out, const void* in, int parity, int inverse, int P,
                                int nrhs, size_t rb);
// operators (api.cu)
lqcd_status op_hop(lqcd_ctx* c, void* out, const void* in, int parity, int P, bool dag, int epi, bool red,
                   const void* clov, const void* y, double a, int nrhs, size_t rb, int red_slot);
lqcd_status op_schur(lqcd_ctx* c, void* out_o, const void* in_o, void* tmp_e, int P, bool dag, int nrhs,
                     size_t rb, size_t tmp_rb, int red_slot /* -1: no reduction */);
lqcd_status op_full(lqcd_ctx* c, void* out, const void* in, int P, bool dag, int nrhs, size_t rb);
DslashArgs base_args(lqcd_ctx* c, int P);
lqcd_status launch_dslash(lqcd_ctx* c, const DslashArgs& A, int P, bool dag, int epi, bool red, int nrhs);
// solver.cu
lqcd_status solve(lqcd_ctx* c, double* x, const double* b, double tol, int nrhs, const lqcd_solver_params* p,
                  lqcd_solver_stats* st);
lqcd_status solve_batch(lqcd_ctx* const* ctxs, int n, double* const* x, const double* const* b, const double* tol,
                        const lqcd_solver_params* p, lqcd_solver_stats* st);
// fgcr.cu
// sap.cu: z = SAP(r) on FP32 full internal fields; rho_buf and dlt_buf are
// two FP32 full fields of scratch (block residuals and corrections)
lqcd_status sap_check(const lqcd_ctx* c, const int bs[4]);
lqcd_status sap_apply(lqcd_ctx* c, void* z, const void* r, const int bs[4], int ncycle, int nmr, char* rho_buf,
                      char* dlt_buf);
lqcd_status solve_fgcr(lqcd_ctx* c, lqcd_net* net, double* x, const double* b, double tol,
                       const lqcd_solver_params* p, lqcd_solver_stats* st, bool host_io);
// fgmres.cu
lqcd_status solve_fgmres_dr(lqcd_ctx* c, lqcd_net* net, double* x, const double* b, double tol,
                            const lqcd_solver_params* p, lqcd_solver_stats* st, bool host_io);

}  // namespace lqcd
