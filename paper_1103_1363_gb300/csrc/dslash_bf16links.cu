// Instantiation of the hopping-term kernels for one storage combination
// (links/clover PB16, spinors P32; one unit per combination so that the
// translation units compile in parallel).
#include "dslash_impl.cuh"

namespace lqcd {
cudaError_t dslash_dispatch_bf16links(const DslashArgs& A, int recon, bool dag, int epi, bool red, int nrhs,
                              int block, cudaStream_t s)
{
    return dispatch_dslash_p<PB16, P32>(A, recon, dag, epi, red, nrhs, block, s);
}
}  // namespace lqcd
