// Instantiation of the hopping-term kernels for one storage combination
// (links/clover P32, spinors P16 with per-site norm; one unit per combination so
// that the translation units compile in parallel).
#include "dslash_impl.cuh"

namespace lqcd {
cudaError_t dslash_dispatch_f16spinors(const DslashArgs& A, int recon, bool dag, int epi, bool red, int nrhs,
                              int block, cudaStream_t s)
{
    return dispatch_dslash_p<P32, P16>(A, recon, dag, epi, red, nrhs, block, s);
}
}  // namespace lqcd
