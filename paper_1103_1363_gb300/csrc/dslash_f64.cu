// Instantiation of the hopping-term kernels for one storage precision
// (split per precision so the translation units compile in parallel).
#include "dslash_impl.cuh"

namespace lqcd {
cudaError_t dslash_dispatch_f64(const DslashArgs& A, int recon, bool dag, int epi, bool red, int nrhs,
                              int block, cudaStream_t s)
{
    return dispatch_dslash_p<P64>(A, recon, dag, epi, red, nrhs, block, s);
}
}  // namespace lqcd
