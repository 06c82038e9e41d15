// Schur-operator application whose scratch lives in a fixed device array.
//
// The even-odd Schur operator needs an even-parity intermediate field
// between its two hopping sweeps.  lqcd_dslash takes it from the solver
// vectors of the context's workspace; lqcd_dslash_schur_static takes it from
// the array below, which the CUDA module carries in every GPU that loads the
// library.  The call allocates nothing and leaves the workspace untouched,
// so it can run between the steps of a caller's own solver without
// clobbering the library's solver vectors.  It is for callers that cannot
// allocate device memory where they apply the operator: a fixed memory
// budget, an allocator that must not grow, or code running where cudaMalloc
// is not allowed.
#include "internal.h"

namespace lqcd {

// 32 MiB: one FP64 even field of up to 174762 sites (V/2), one FP32 field
// of up to 349525 sites, nrhs fields of the requested precision in total.
static constexpr size_t STATIC_SCRATCH_BYTES = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_schur_scratch[STATIC_SCRATCH_BYTES];

// Device address of g_schur_scratch on the current device.  In host code
// the symbol is only a host-side stand-in; kernels must be given the address
// cudaGetSymbolAddress returns.  It is looked up on every call (cheap once
// the module is loaded on the device), so that no address outlives a device
// reset or a recreated primary context.
static lqcd_status static_scratch(void** out)
{
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_schur_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_schur_scratch)");
    *out = p;
    return LQCD_OK;
}

}  // namespace lqcd

using namespace lqcd;

extern "C" lqcd_status lqcd_dslash_schur_static(lqcd_ctx* c, void* out, const void* in, double kappa, double csw,
                                                int dag, lqcd_prec prec, int nrhs)
{
    try {
        if (!c) return fail(LQCD_ERR_INVALID, "null context");
        if (!c->ws) return fail(LQCD_ERR_NOMEM, "no workspace: call lqcd_set_workspace");
        if (!valid_mode(prec)) return fail(LQCD_ERR_INVALID, "bad precision");
        if (!c->holds(mode_pg(prec))) return fail(LQCD_ERR_STATE, "precision not held by this context");
        if (!out || !in) return fail(LQCD_ERR_INVALID, "lqcd_dslash_schur_static: null field");
        if (out == in) return fail(LQCD_ERR_INVALID, "lqcd_dslash_schur_static: out must not alias in");
        if (nrhs < 1) return fail(LQCD_ERR_INVALID, "lqcd_dslash_schur_static: nrhs must be >= 1");
        if (!c->gauge_loaded) return fail(LQCD_ERR_STATE, "lqcd_dslash_schur_static: no gauge field loaded");
        if (c->cut()) return fail(LQCD_ERR_STATE, "lqcd_dslash_schur_static: not on a sub-domain of a cut lattice");
        const double have_csw = c->clover_state ? c->csw : 0.0;
        if (csw != have_csw) return fail(LQCD_ERR_STATE, "lqcd_dslash_schur_static: csw differs from lqcd_clover_compute");
        if (csw != 0.0 && kappa != c->kappa) return fail(LQCD_ERR_STATE, "lqcd_dslash_schur_static: kappa differs from lqcd_clover_compute");
        if (!(kappa > 0.0)) return fail(LQCD_ERR_INVALID, "lqcd_dslash_schur_static: kappa must be > 0");
        const size_t fb = c->field_bytes(prec);
        if ((size_t)nrhs * fb > STATIC_SCRATCH_BYTES)
            return fail(LQCD_ERR_INVALID, "lqcd_dslash_schur_static: nrhs x (V/2 field) exceeds the 32 MiB static scratch");
        DeviceScope dev_scope;
        LQ_TRY(dev_scope.enter(c->device));
        void* scratch = nullptr;
        LQ_TRY(static_scratch(&scratch));
        const double saved = c->kappa;
        c->kappa = kappa;
        // the first sweep writes every even site of the intermediate before the
        // second reads any, so the scratch needs no clearing between calls
        lqcd_status st = op_schur(c, out, in, scratch, prec, dag != 0, nrhs, fb, fb, -1);
        c->kappa = saved;
        return st;
    } catch (...) {
        return fail(LQCD_ERR_INVALID, "unexpected exception");
    }
}
