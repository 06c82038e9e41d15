// Instantiation of the hopping-term kernels with FP64 storage and
// double-float arithmetic (FP64-accurate residuals at FP32 instruction rate).
#include "dslash_impl.cuh"

namespace lqcd {
cudaError_t dslash_dispatch_df(const DslashArgs& A, int recon, bool dag, int epi, bool red, int nrhs, int block,
                               cudaStream_t s)
{
    return dispatch_dslash_p<PDF, PDF>(A, recon, dag, epi, red, nrhs, block, s);
}
}  // namespace lqcd
