// Persistent even-odd CG: one cooperative launch runs a whole block of
// inner CG iterations for every lattice (and every right-hand side) of a
// solve, with grid-wide barriers between the stages of an iteration.
//
// The CG on the normal equations of the Schur complement (Sec. 5) needs,
// per iteration, four hopping sweeps (Mhat p, then Mhat^dag of the result
// fused with the x and r updates), two global sums (|Mhat p|^2 and |r|^2)
// and the direction update p = r + beta p.  On small lattices each of these
// launches is a few microseconds of work behind a few microseconds of
// launch latency; here they are stages of one kernel:
//   S1  t_e = A_ee^{-1} H_eo p_o                       (all lattices, all rhs)
//   S2  q_o = A_oo p_o - kappa^2 H_oe t_e, |q_o|^2
//   S3  t_e = A_ee^{-1} H_eo^dag q_o
//   S4  x += alpha p, r -= alpha (A_oo q_o - kappa^2 H_oe^dag t_e), |r|^2
//   S5  p = r + beta p
// with a grid barrier after each (S5 is left out of the block's last
// iteration when a reliable update follows).  The stage arguments live in
// the kernel's parameter memory; within a block the |r|^2 slots form a ring
// of two, so even and odd iterations each have one fixed argument set.  Every (lattice, rhs) is spread
// over all blocks; its sums use the deterministic two-stage reduction of the
// other kernels (block partials, last block adds them in order), over this
// launch's grid: results are reproducible run to run and agree with the
// launch-per-stage path up to the summation order of the global sums.
//
// Grid barrier: a counter and a generation word in global memory.  The
// launch is cooperative, so every block is resident and a barrier is
// reached by all of them.  Each wait is bounded by %globaltimer: a block
// whose wait expires raises the abort word and the error word
// (ERRW_TIMEOUT) and returns; every other block sees the abort word at its
// next barrier (or in its own bounded wait) and returns too.  The host
// reads the abort word after the launch and reports LQCD_ERR_TIMEOUT.
#include "internal.h"

namespace lqcd {

namespace {

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// All blocks of the grid arrive before any leaves; false once the launch is
// aborting (a wait expired somewhere), and then the caller returns.
__device__ __forceinline__ bool grid_barrier(const PersistArgs& P)
{
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile int* ab = P.abort;
        volatile unsigned* gen = P.bar + 1;
        if (*ab) {
            ok = 0;
        } else {
            const unsigned g0 = *gen;  // read before arriving: the generation cannot move without us
            __threadfence();           // this block's writes before its arrival
            const unsigned arrived = atomicAdd(P.bar, 1u) + 1u;
            if (arrived == gridDim.x) {
                atomicExch(P.bar, 0u);
                __threadfence();
                atomicAdd(P.bar + 1, 1u);
            } else {
                const unsigned long long t0 = globaltimer_ns();
                while (*gen == g0) {
                    __nanosleep(32);  // fewer polls of the generation word competing with the arrivals
                    if (*ab) {
                        ok = 0;
                        break;
                    }
                    if (globaltimer_ns() - t0 > P.wait_ns) {
                        atomicExch(P.abort, 1);
                        atomicOr(P.errw, ERRW_TIMEOUT);
                        ok = 0;
                        break;
                    }
                }
            }
            __threadfence();  // the other blocks' writes after leaving
        }
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

// The (lattice, rhs) pair of tile t (pairs are few: a linear scan).
__device__ __forceinline__ int tile_pair(const PersistArgs& P, int t)
{
    int q = 0;
    while (q + 1 < P.npairs && P.tile0[q + 1] <= t) ++q;
    return q;
}

// One hopping stage: the tiles of every (lattice, rhs) still iterating,
// spread over the grid; a reducing stage sums each tile in its block and
// the pair's last tile (ticket) adds the pair's tile partials in order.
// The stage arguments of the tile's lattice are copied into shared memory
// (the parameter block of up to eight lattices is larger than the constant
// cache, and the site loop reads the arguments throughout).
template <int PG, int PS, int RECON, bool DAG, int EPI, bool RED>
__device__ __forceinline__ void hop_stage(const PersistArgs& P, int stage, int j)
{
    __shared__ __align__(16) DslashArgs As;
    __shared__ int cur_l;
    if (threadIdx.x == 0) cur_l = -1;
    const int ntile = P.tile0[P.npairs];
    for (int t = blockIdx.x; t < ntile; t += gridDim.x) {
        const int q = tile_pair(P, t);
        const int l = P.pair_lat[q], rhs = P.pair_rhs[q];
        const PersistLattice& L = P.lat[l];
        __syncthreads();  // the previous tile is done with As (and cur_l is set)
        if (cur_l != l) {
            const int* src = reinterpret_cast<const int*>(&L.d[j & 1][stage]);
            int* dst = reinterpret_cast<int*>(&As);
            for (int w = threadIdx.x; w < (int)(sizeof(DslashArgs) / sizeof(int)); w += blockDim.x) dst[w] = src[w];
            __syncthreads();
            if (threadIdx.x == 0) cur_l = l;
        }
        const DslashArgs& A = As;
        if (A.skip && A.skip[rhs]) continue;        // uniform over the block
        const int tl = t - P.tile0[q];
        double nrm = 0.0;
        for (int k = 0; k < L.spt; ++k) {
            const int i = (tl * L.spt + k) * PERSIST_THREADS + threadIdx.x;
            if (i < A.g.Vh) dslash_site<PG, PS, RECON, DAG, EPI, RED>(A, rhs, i, nrm);
        }
        if (RED) {
            double v[1] = {nrm};
            block_reduce_finalize<1>(v, A.partials + rhs * A.part_rs, A.tickets + rhs, A.red + rhs * A.red_rs, tl,
                                     L.ntiles);
            __syncthreads();  // the reduction's shared memory is reused by the next tile
        }
    }
}

// p_o = r_o + beta p_o, beta = |r_{j+1}|^2 / |r_j|^2 (even + odd slots of
// the two-slot ring), over the same tiles.
template <int PS>
__device__ __forceinline__ void p_stage(const PersistArgs& P, int j)
{
    typedef typename RealT<PS>::type RP;
    const int rr = SC_RR + 2 * (j & 1), rr1 = SC_RR + 2 * ((j + 1) & 1);
    const int ntile = P.tile0[P.npairs];
    for (int t = blockIdx.x; t < ntile; t += gridDim.x) {
        const int q = tile_pair(P, t);
        const int rhs = P.pair_rhs[q];
        const PersistLattice& L = P.lat[P.pair_lat[q]];
        if (L.skip && L.skip[rhs]) continue;
        const int tl = t - P.tile0[q];
        const double* sc = L.scal + rhs * SC_PER_RHS;
        const double den = sc[rr] + sc[rr + 1];  // 0 once the residual has vanished
        const float beta = den > 0.0 ? (float)((sc[rr1] + sc[rr1 + 1]) / den) : 0.f;
        char* p = L.p + rhs * L.p_rb;
        const char* r = L.r + rhs * L.r_rb;
        for (int k = 0; k < L.spt; ++k) {
            const int i = (tl * L.spt + k) * PERSIST_THREADS + threadIdx.x;
            if (i >= L.g.Vh) break;
            RP vp[24];
            float vr[24];
            SpinorIO<PS>::load(p, L.g.stride, i, vp);
            SpinorIO<P32>::load(r, L.g.stride, i, vr);
#pragma unroll
            for (int kk = 0; kk < 24; ++kk) vp[kk] = (RP)(vr[kk] + beta * (float)vp[kk]);
            SpinorIO<PS>::store(p, L.g.stride, i, vp);
        }
    }
}

template <int PG, int PS, int RECON>
__global__ void __launch_bounds__(PERSIST_THREADS, LQCD_DSLASH_MINB) cg_persist_kernel(const PersistArgs P)
{
    for (int j = 0; j < P.niter; ++j) {
        hop_stage<PG, PS, RECON, false, EPI_CLOVINV, false>(P, 0, j);
        if (!grid_barrier(P)) return;
        hop_stage<PG, PS, RECON, false, EPI_XPAY, true>(P, 1, j);
        if (!grid_barrier(P)) return;
        hop_stage<PG, PS, RECON, true, EPI_CLOVINV, false>(P, 2, j);
        if (!grid_barrier(P)) return;
        hop_stage<PG, PS, RECON, true, EPI_CG, true>(P, 3, j);
        if (!grid_barrier(P)) return;
        if (j == P.niter - 1 && !P.last_p) break;
        p_stage<PS>(P, j);
        if (!grid_barrier(P)) return;
    }
    // the next block starts from slot 0: |r|^2 of the block's last iterate
    if (P.copy_slots && blockIdx.x == 0 && (P.niter & 1)) {
        const int src = SC_RR + 2;
        for (int l = 0; l < P.nlat; ++l)
            for (int rhs = threadIdx.x; rhs < P.lat[l].R; rhs += blockDim.x) {
                double* sc = P.lat[l].scal + rhs * SC_PER_RHS;
                sc[SC_RR] = sc[src];
                sc[SC_RR + 1] = sc[src + 1];
            }
    }
}

template <int PG, int PS, int RECON>
cudaError_t grid_persist_t(int ntiles, int* grid)
{
    static int per_sm = 0, sms = 0;
    if (per_sm == 0) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cg_persist_kernel<PG, PS, RECON>,
                                                              PERSIST_THREADS, 0);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
    }
    // no more blocks than tiles, and all of them resident
    int g = per_sm * sms;
    if (g > ntiles) g = ntiles;
    if (g > PERSIST_MAX_GRID) g = PERSIST_MAX_GRID;
    *grid = g > 0 ? g : 1;
    return cudaSuccess;
}

template <int PG, int PS, int RECON>
cudaError_t launch_persist_t(const PersistArgs& P0, int grid, cudaStream_t s)
{
    PersistArgs P = P0;
    void* args[] = {&P};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(cg_persist_kernel<PG, PS, RECON>), dim3(grid),
                                       dim3(PERSIST_THREADS), args, 0, s);
}

}  // namespace

bool persist_supported(int mode) { return mode == P32 || mode == MODE_F16_SPINORS || mode == MODE_BF16_SPINORS; }

#define LQ_PERSIST_DISPATCH(FN, ...)                                                       \
    (mode == P32 ? (recon == 12 ? FN<P32, P32, 12>(__VA_ARGS__) : FN<P32, P32, 18>(__VA_ARGS__))  \
     : mode == MODE_F16_SPINORS ? (recon == 12 ? FN<P32, P16, 12>(__VA_ARGS__) : FN<P32, P16, 18>(__VA_ARGS__)) \
                                : (recon == 12 ? FN<P32, PB16, 12>(__VA_ARGS__) : FN<P32, PB16, 18>(__VA_ARGS__)))

lqcd_status persist_grid(int mode, int recon, int ntiles, int* grid)
{
    if (!persist_supported(mode))
        return fail(LQCD_ERR_INVALID, "persistent CG: the inner precision must be F32, F16_SPINORS or BF16_SPINORS");
    LQ_CUDA(LQ_PERSIST_DISPATCH(grid_persist_t, ntiles, grid));
    return LQCD_OK;
}

lqcd_status launch_persist(lqcd_ctx* c0, const PersistArgs& P, int mode, int recon, int grid)
{
    if (!persist_supported(mode))
        return fail(LQCD_ERR_INVALID, "persistent CG: the inner precision must be F32, F16_SPINORS or BF16_SPINORS");
    if (P.nlat < 1 || P.nlat > PERSIST_MAXL) return fail(LQCD_ERR_INVALID, "persistent CG: 1..8 lattices");
    LQ_CUDA(LQ_PERSIST_DISPATCH(launch_persist_t, P, grid, c0->stream));
    return LQCD_OK;
}
#undef LQ_PERSIST_DISPATCH

}  // namespace lqcd
