/*
 * lqcd.h - C ABI of the GB300 Wilson-clover Dirac operator and solver library.
 *
 * The library applies the Wilson(-clover) Dirac operator M and solves
 * M x = b through CG on the normal equations of the even-odd Schur
 * complement, the problem the paper states as M phi = b or
 * M^dag M phi = b (Sec. 3, Eq. (1)) and solves with CG in Sec. 5.
 *
 * Conventions (fixed; the paper uses the standard Wilson formulation
 * without writing it out):
 *   H psi(x) = sum_mu (1 - g_mu) U_mu(x) psi(x+mu) + (1 + g_mu) U_mu(x-mu)^dag psi(x-mu)
 *   A(x)     = 1 + i kappa csw sum_{mu<nu} sigma_{mu nu} Fhat_{mu nu}(x)   (clover)
 *   M        = A - kappa H
 *   Mhat     = A_oo - kappa^2 H_oe A_ee^{-1} H_eo       (odd-parity Schur complement)
 * DeGrand-Rossi (chiral) gamma matrices, sigma_{mu nu} = (i/2)[g_mu, g_nu],
 * Fhat = (Q - Q^dag)/8 made traceless with Q the sum of the four plaquette
 * leaves, periodic boundaries in x, y, z, and a factor -1 on every fermion
 * hop across the t boundary when t_antiperiodic is set.  Parity of a site is
 * (x + y + z + t) mod 2, even = 0, odd = 1.
 *
 * Canonical layouts (FP64, what users hand in and get back):
 *   gauge   U[t][z][y][x][mu][a][b][re,im]   mu = 0..3 for x, y, z, t
 *   spinor  psi[t][z][y][x][spin][colour][re,im]
 * Internal layouts (what lqcd_dslash / lqcd_clover_apply take; produced by
 * lqcd_pack): one field per parity, structure of arrays over the V/2 sites
 * of that parity in 16-byte vectors; lqcd_field_bytes gives the size.
 *   F64:      12 chunks of double2 (one complex each), [chunk][stride]
 *   F32:       6 chunks of float4 (two complex each),  [chunk][stride]
 *   F16/BF16:  3 chunks of 8 halves (four complex each), [chunk][stride],
 *              followed by one FP32 per-site norm [stride]; the stored
 *              value is q = v / n with n = max |v_i| over the 24 reals.
 * stride = V/2 rounded up to a multiple of 128.  A "full" internal field is
 * the even field followed by the odd field.  nrhs fields are stored back
 * to back.
 *
 * Memory: the library never allocates device memory.  All persistent
 * state (gauge copies, clover, solver vectors, reduction scratch) lives
 * in one caller-owned workspace (lqcd_workspace_size / lqcd_set_workspace),
 * typically a torch tensor.  Vectors handed to calls are caller-owned too.
 *
 * Devices: a call that touches the GPU makes the context's device current
 * while it runs and gives the calling thread its previous current device
 * back before returning.
 *
 * Errors: every call returns an lqcd_status and never throws.  A
 * human-readable message for the last failure on the calling thread is
 * available from lqcd_last_error().  Calls are asynchronous on the
 * context's stream; device-side problems (a singular clover block, a solver
 * breakdown, an expired bounded wait) are recorded in a device error word
 * and reported, then cleared, by lqcd_sync, or at the end of a solve.  A context is not thread-safe; separate
 * contexts may be used concurrently.
 */
#ifndef LQCD_H
#define LQCD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lqcd_ctx lqcd_ctx;

typedef enum {
    LQCD_OK = 0,
    LQCD_ERR_INVALID = 1,         /* bad argument (pointer, parity, size, flag) */
    LQCD_ERR_CUDA = 2,            /* a CUDA runtime call failed */
    LQCD_ERR_NOMEM = 3,           /* workspace missing or too small */
    LQCD_ERR_STATE = 4,           /* call out of order (no gauge, csw mismatch ...) */
    LQCD_ERR_NOT_CONVERGED = 5,   /* solver hit maxiter; x holds the partial solution */
    LQCD_ERR_BREAKDOWN = 6,       /* solver produced NaN/Inf or diverged */
    LQCD_ERR_TIMEOUT = 7,         /* a bounded device wait expired */
    LQCD_ERR_CLOVER_SINGULAR = 8  /* some 6x6 clover block has |pivot| < 1e-12 */
} lqcd_status;

/* Storage precision of links, clover and spinor fields.  Arithmetic is FP64
 * for LQCD_F64 and FP32 for every other value.  LQCD_F16_LINKS and
 * LQCD_BF16_LINKS keep the operator's coefficients (links and clover) in
 * FP16 / BF16 and every spinor field in the F32 layout; LQCD_F16_SPINORS and
 * LQCD_BF16_SPINORS the reverse: spinor fields in FP16 / BF16 with a per-site
 * norm, links and clover in FP32.  Rounding the coefficients perturbs M by a
 * fixed relative 2^-11 (2^-8), which CG on the normal equations feels through
 * cond(Mhat^dag Mhat); rounding the vectors perturbs each iteration by the
 * same relative amount without changing the operator. */
typedef enum {
    LQCD_F64 = 0,
    LQCD_F32 = 1,
    LQCD_F16 = 2,
    LQCD_BF16 = 3,
    LQCD_F16_LINKS = 4,
    LQCD_BF16_LINKS = 5,
    /* 6 is not used */
    LQCD_F16_SPINORS = 7,   /* FP16 spinors (per-site norm), FP32 links and clover */
    LQCD_BF16_SPINORS = 8,  /* BF16 spinors (per-site norm), FP32 links and clover */
    LQCD_NPREC = 9
} lqcd_prec;

/* operator selection for lqcd_dslash (op_flags) */
enum {
    LQCD_OP_HOP = 0,    /* out_p = H_{p,1-p} in_{1-p}; kappa, csw ignored */
    LQCD_OP_SCHUR = 1,  /* out_o = Mhat in_o; parity must be 1 (odd) */
    LQCD_OP_FULL = 2,   /* out = M in on full internal fields; parity ignored */
    LQCD_DAG = 1 << 8   /* apply the adjoint (H^dag = g5 H g5, Mhat^dag, M^dag) */
};

typedef struct {
    int dims[4];          /* Lx, Ly, Lz, Lt; each even and >= 2 */
    int t_antiperiodic;   /* 1: factor -1 on fermion hops across the t boundary */
    int recon;            /* 12 or 18: link storage for F32/F16/BF16 (F64 always 18) */
    int prec_mask;        /* bit (1 << lqcd_prec) for each precision to hold; F64 is always held */
    int max_nrhs;         /* largest nrhs used with the solver vectors (>= 1) */
    int gcr_nkrylov;      /* Krylov space of FGCR / FGMRES-DR, 0..256 (0: no vectors
                             reserved; 2 gcr_nkrylov + 3 FP32 full fields otherwise) */
    int part[4];          /* sub-domains of the global lattice along x, y, z, t (0 or 1:
                             not cut); dims are then this sub-domain's extents */
    int coord[4];         /* this sub-domain's position, 0 <= coord < part */
} lqcd_config;

/* Create a context for one lattice.  `cuda_stream` is a cudaStream_t (may
 * be NULL for the legacy default stream).  No device memory is touched
 * until lqcd_set_workspace.
 *
 * Sub-domains (the data-parallel split of one lattice over several GPUs, Sec.
 * 5's multi-node layout): with part[mu] > 1 the context holds the sub-domain
 * coord of a global lattice of dims[mu] x part[mu] sites along mu (every
 * local extent even, so that local and global parities agree).  Its links
 * are the sub-domain's own (canonical layout over the local sites); hops
 * across a cut boundary go through faces (lqcd_halo_*).  A cut context
 * supports gauge load, pack / unpack, clover_compute with csw = 0,
 * lqcd_halo_* and lqcd_norm2; every other call returns LQCD_ERR_STATE. */
lqcd_status lqcd_create(const lqcd_config* cfg, void* cuda_stream, lqcd_ctx** out);
lqcd_status lqcd_destroy(lqcd_ctx* ctx);
lqcd_status lqcd_set_stream(lqcd_ctx* ctx, void* cuda_stream);

/* Bytes of device workspace the context needs (256-byte aligned base). */
lqcd_status lqcd_workspace_size(const lqcd_ctx* ctx, size_t* bytes);
/* Hand the context its workspace (caller-owned, must outlive the context). */
lqcd_status lqcd_set_workspace(lqcd_ctx* ctx, void* dev_ptr, size_t bytes);

/* Bytes of one internal single-parity field of precision `prec`. */
lqcd_status lqcd_field_bytes(const lqcd_ctx* ctx, lqcd_prec prec, size_t* bytes);

/* Load the gauge field (canonical FP64, host or device pointer; detected)
 * and build every internal copy (F64 recon-18, the others with cfg.recon).
 * Invalidates the clover term. */
lqcd_status lqcd_gauge_load(lqcd_ctx* ctx, const double* links);

/* Build the clover term A and A^{-1} on both parities for (kappa, csw)
 * from the loaded links: four-leaf Fhat, two 6x6 Hermitian blocks per site,
 * computed and inverted in FP64 (Gauss-Jordan with partial pivoting), then
 * rounded into every held precision.  csw = 0 gives A = 1 (nothing stored
 * is read).  Returns LQCD_ERR_CLOVER_SINGULAR if some block is singular. */
lqcd_status lqcd_clover_compute(lqcd_ctx* ctx, double kappa, double csw);

/* Canonical FP64 spinor(s) (host or device) <-> internal field(s) of one
 * parity (parity 0/1) or of both (parity -1: full internal field).
 * nrhs canonical spinors are back to back; so are the internal fields. */
lqcd_status lqcd_pack(lqcd_ctx* ctx, void* internal, const double* canonical, int parity,
                      lqcd_prec prec, int nrhs);
lqcd_status lqcd_unpack(lqcd_ctx* ctx, double* canonical, const void* internal, int parity,
                        lqcd_prec prec, int nrhs);

/* Apply the operator selected by op_flags to nrhs internal fields (device
 * pointers, precision prec).  For LQCD_OP_HOP `in` has parity 1-parity
 * and `out` parity `parity`.  For LQCD_OP_SCHUR and LQCD_OP_FULL, kappa
 * and csw must be those of the last lqcd_clover_compute (csw = 0 without
 * one); otherwise LQCD_ERR_STATE.  `out` must not alias `in`. */
lqcd_status lqcd_dslash(lqcd_ctx* ctx, void* out, const void* in, int parity, double kappa,
                        double csw, int op_flags, lqcd_prec prec, int nrhs);

/* out_p = A_pp in_p (inverse = 0) or A_pp^{-1} in_p (inverse = 1) on
 * nrhs internal fields of parity `parity`.  Needs lqcd_clover_compute. */
lqcd_status lqcd_clover_apply(lqcd_ctx* ctx, void* out, const void* in, int parity, int inverse,
                              lqcd_prec prec, int nrhs);

typedef enum {
    LQCD_SOLVER_CG_EO = 0,   /* CG on Mhat^dag Mhat (even-odd), reconstruct x_e */
    LQCD_SOLVER_CG_FULL = 1, /* CG on M^dag M over the full lattice (CGNR) */
    LQCD_SOLVER_FGCR = 2,    /* flexible GCR(nkrylov) on M, right preconditioned */
    LQCD_SOLVER_FGMRES_DR = 3 /* flexible GMRES on M with a Krylov space of nkrylov
                                 vectors, ndefl of them kept at each restart
                                 (deflated restart, Sec. 7); right preconditioned */
} lqcd_solver_kind;

typedef struct {
    int solver;              /* lqcd_solver_kind */
    int inner_prec;          /* lqcd_prec of the inner iteration (F64 = plain FP64 CG) */
    int maxiter;             /* total inner iterations allowed */
    int reliable_interval;   /* FP64 residual replacement every this many iterations (0: off) */
    double reliable_delta;   /* ... or when |r| < delta * max |r| since the last one */
    int check_interval;      /* host reads the residual every this many iterations */
    int nkrylov;             /* FGCR restart length */
    int use_graph;           /* 1: replay the iteration block as a CUDA graph */
    int residual_prec;       /* LQCD_F64 (the only value): arithmetic of the
                                reliable-update, candidate-check and FGCR restart
                                residuals of a mixed solve */
    int ndefl;               /* FGMRES-DR: harmonic Ritz vectors kept at a restart
                                (0 <= ndefl <= 16, < nkrylov; 0: plain restarted FGMRES) */
    int persistent;          /* 1: even-odd CG runs each block of check_interval inner
                                iterations as one persistent cooperative launch over
                                every lattice and right-hand side of the call (grid
                                barriers between the four hopping stages, the two
                                reductions and the direction update); for small
                                lattices, whose launches are latency-bound.  Needs
                                LQCD_SOLVER_CG_EO, inner_prec LQCD_F32, LQCD_F16_SPINORS
                                or LQCD_BF16_SPINORS, at most 8 lattices and 64
                                right-hand sides in all; use_graph is then ignored.
                                The iterates agree with the launch-per-stage path up
                                to the summation order of the global sums. */
    int persistent_wait_us;  /* bound of each grid-barrier wait of the persistent launch
                                (0: 2 s); a wait that expires ends the launch and the
                                solve returns LQCD_ERR_TIMEOUT */
} lqcd_solver_params;

typedef struct {
    int iterations;          /* inner iterations (all right-hand sides: the maximum) */
    int reliable_updates;    /* FP64 residual replacements performed */
    int restarts;            /* FGCR restarts / CG true-residual re-checks */
    long dslash_count;       /* single-parity hopping applications (all precisions) */
    long kernel_launches;    /* kernels launched by the call (graph replays count their nodes) */
    double true_residual;    /* |b - M x| / |b| in FP64 on the device (max over rhs) */
    double seconds;          /* wall time of the call */
    int preconditioner_fallback; /* FGCR: 1 if the preconditioner stagnated (a restart
                                    cycle did not halve the residual) and the solve
                                    finished with the identity */
    int precision_fallback;  /* CG with a 16-bit inner precision: 1 if three reliable
                                updates in a row failed to halve |r|^2 and the solve
                                finished with FP32 inner storage */
} lqcd_solver_stats;

/* Defaults: CG_EO, F32 inner, maxiter 100000, reliable every 50, delta 0.1,
 * check every 10, nkrylov 20, no graph, ndefl 0, not persistent.
 *
 * LQCD_SOLVER_FGCR and LQCD_SOLVER_FGMRES_DR run their recursion on FP32
 * full fields (inner_prec F32, F16_LINKS or BF16_LINKS for the operator) and
 * recompute the residual b - M x in FP64 at every restart; they need
 * cfg.gcr_nkrylov >= nkrylov.  FGCR allows nkrylov <= 24, FGMRES-DR
 * nkrylov <= cfg.gcr_nkrylov. */
lqcd_status lqcd_solver_params_default(lqcd_solver_params* p);

/* Solve M x = b for nrhs canonical FP64 right-hand sides (host or device
 * pointers, back to back) to |b - M x| / |b| <= tol, using the clover
 * term of the last lqcd_clover_compute (kappa from there; csw = 0 without
 * one).  x is overwritten (initial guess 0).  The true residual is
 * recomputed in FP64 at the end.  LQCD_ERR_NOT_CONVERGED leaves the
 * partial solution in x. */
lqcd_status lqcd_solve(lqcd_ctx* ctx, double* x, const double* b, double tol, int nrhs,
                       const lqcd_solver_params* params, lqcd_solver_stats* stats);

/* Same result as lqcd_dslash(ctx, out, in, 1, kappa, csw, LQCD_OP_SCHUR |
 * (dag ? LQCD_DAG : 0), prec, nrhs), but the even-parity intermediate between
 * the two hopping sweeps lives in a 32 MiB array that the library's CUDA
 * module carries on every GPU that loads it (held until the process exits),
 * not in the context's workspace.  For callers that cannot allocate device
 * memory where they apply the operator: a fixed memory budget, an allocator
 * that must not grow, or code running where cudaMalloc is not allowed.  The
 * paper has no counterpart.
 *   - The call allocates nothing, calls no allocating routine and writes
 *     nothing in the context's workspace (its solver vectors stay intact).
 *   - Limit: nrhs x lqcd_field_bytes(prec) <= 32 MiB, else LQCD_ERR_INVALID.
 *   - Every call looks up the array's address on the context's device
 *     (cudaGetSymbolAddress); the first call on a device can load the
 *     library's module there, so make that first call before any stream
 *     capture.
 *   - Every call on a device shares the one array: calls that overlap on the
 *     GPU (other streams, other contexts, other threads) race.  Nothing in it
 *     needs clearing: each call overwrites the part it reads.
 * Inputs and outputs are internal odd-parity fields as for lqcd_dslash. */
lqcd_status lqcd_dslash_schur_static(lqcd_ctx* ctx, void* out, const void* in, double kappa, double csw,
                                     int dag, lqcd_prec prec, int nrhs);

/* ---------------------------------------------------------------------
 * Learned preconditioner: a gauge-equivariant network of parallel-transport
 * convolutions, used as the right preconditioner of flexible GCR.  (The
 * paper preconditions FGCR with SAP and notes that the flexible outer
 * iteration tolerates a preconditioner that is not a fixed operator, Sec. 5;
 * the network takes SAP's slot.)  A layer maps C_in to C_out channels of
 * spinor fields:
 *   out(x)[co][s] = sum_{h=0..8} sum_{ci,r} W_h[co*4+s][ci*4+r] (T_h in)(x)[ci][r]
 * T_0 = 1, T_{2mu+1} in(x) = U_mu(x) in(x+mu), T_{2mu+2} in(x) = U_mu(x-mu)^dag in(x-mu),
 * with the fermion t sign; the links are the context's F32 copy.  The
 * network is linear (no activation, no bias).
 * Activations: FP32 complex, [batch][site][channel][spin][colour], canonical
 * site order; the network's input and output are canonical FP32 spinors.
 * Weights: FP32 complex, layer after layer, each [9][4 C_out][4 C_in].
 * Gradients are dL/dRe W + i dL/dIm W.  bf16 = 1 runs the channel
 * contractions on the tensor cores (tcgen05, BF16 operands, FP32
 * accumulators in tensor memory); bf16 = 0 runs them in FP32.  Inside the
 * network activations are kept planar (per channel, six float4 planes over
 * the sites); the calls below convert at the boundary, so callers always see
 * the canonical layout.  A bounded device wait that expires inside a layer
 * sets the error word (lqcd_sync returns LQCD_ERR_TIMEOUT). */
typedef struct lqcd_net lqcd_net;
/* channels[0..nlayers], channels[0] = channels[nlayers] = 1, each <= 12;
 * max_batch: largest batch of forward / training calls.  Needs F32 links. */
lqcd_status lqcd_net_create(lqcd_ctx* ctx, int nlayers, const int* channels, int bf16, int max_batch,
                            lqcd_net** out);
/* Frees the handle; the caller frees the workspace it provided. */
lqcd_status lqcd_net_destroy(lqcd_net* net);
/* Device bytes the network needs: weights, gradients, Adam moments, the
 * real-ified forward and adjoint weights, activations of every layer
 * boundary and two gradient buffers for max_batch items, reduction scratch. */
lqcd_status lqcd_net_workspace_size(const lqcd_net* net, size_t* bytes);
/* Caller-owned device workspace, 256-byte aligned; weights start at zero. */
lqcd_status lqcd_net_set_workspace(lqcd_net* net, void* dev_ptr, size_t bytes);
/* Bind the network to another context of the same lattice (extents, t
 * boundary, recon, device) that holds loaded F32 links: later layers
 * transport with that context's links and run on its stream; the network's
 * workspace, weights and Adam state stay.  Training over several gauge fields
 * keeps one context per field resident and binds instead of reloading links.
 * LQCD_ERR_INVALID if the lattices differ, LQCD_ERR_STATE without links. */
lqcd_status lqcd_net_bind(lqcd_net* net, lqcd_ctx* ctx);
/* Cap the CTAs of the BF16 network's persistent launches: at most max_ctas
 * CTAs for a layer (forward or adjoint; by default one per SM, each striding
 * over the batch x 128-site tiles) and for a weight gradient (one input or
 * output channel: all hops per CTA, default one CTA per SM; otherwise at
 * most max_ctas per group of hops, default SMs / 2); the FP32 weight
 * gradient takes the same cap per hop.  0 restores the defaults.  Results do not depend on the cap
 * beyond the FP32 summation order of the weight gradient's atomics; a small
 * cap makes every CTA run many tiles (tests use it to check the multi-tile
 * path on small lattices).  LQCD_ERR_INVALID for max_ctas < 0. */
lqcd_status lqcd_net_set_max_ctas(lqcd_net* net, int max_ctas);
/* Bound of the BF16 network kernels' waits on their own tensor-core MMAs and
 * copies (mbarriers): limit_ns > 0 sets it, 0 restores the default of 2 s.
 * A wait that runs out sets the device error word (lqcd_sync then returns
 * LQCD_ERR_TIMEOUT); the CTA waits, with the default bound, for its own
 * operations in flight, frees its tensor memory and exits, and the network
 * stays usable.  expire_test = 1 is a test of that path: each CTA's last
 * wait of a launch is then for an mbarrier phase that nothing completes, so
 * it runs out after limit_ns.  LQCD_ERR_INVALID for a null network. */
lqcd_status lqcd_net_set_wait(lqcd_net* net, unsigned long long limit_ns, int expire_test);
/* Complex weights in all: the sum over layers of 9 x 4 C_out x 4 C_in. */
lqcd_status lqcd_net_num_weights(const lqcd_net* net, size_t* complex_count);
/* w: host or device FP32 complex weights (resets the Adam moments). */
lqcd_status lqcd_net_set_weights(lqcd_net* net, const float* w);
/* Copy the weights and / or the last gradient out (either may be NULL). */
lqcd_status lqcd_net_get_weights(const lqcd_net* net, float* w, float* grad);
/* One layer (adjoint = 0) or its adjoint (adjoint = 1, the input gradient:
 * sum_h T_h^dag W_h^dag applied to `in`) on device activations. */
lqcd_status lqcd_net_layer_apply(lqcd_net* net, int layer, int adjoint, float* out, const float* in, int batch);
/* Weight gradient of one layer from its input activations and output
 * gradient, added into the net's gradient buffer (zeroed first if zero).
 * Both layer calls take batch <= max_batch (LQCD_ERR_INVALID otherwise). */
lqcd_status lqcd_net_layer_wgrad(lqcd_net* net, int layer, const float* in, const float* gout, int batch, int zero);
/* out = N(in) for batch canonical FP32 spinors (device). */
lqcd_status lqcd_net_forward(lqcd_net* net, float* out, const float* in, int batch);
/* One Adam step on L = mean_b |N(r_b) - e_b|^2 / |e_b|^2 over batch pairs of
 * canonical FP32 spinors (device); *loss (may be NULL) receives L before the
 * step (reading it synchronises the stream). */
lqcd_status lqcd_net_train_step(lqcd_net* net, const float* r, const float* e, int batch, double lr, double beta1,
                                double beta2, double eps, double* loss);

/* Training pair of the learned preconditioner: for nrhs canonical FP64
 * spinors x* (xstar) and x (device pointers, back to back; x = NULL means
 * x = 0), e = x* - x and r = M e, with M the operator of the last
 * lqcd_clover_compute.  r and e are written as canonical FP32 complex
 * spinors (device, nrhs back to back), the network's input and target
 * layout.  With x the iterate of a solver started from 0 on b = M x*, r is
 * that solver's residual b - M x and e its error.  M e is applied in FP64
 * and rounded to FP32 once.  Uses the workspace's solver vectors as scratch
 * (in chunks of cfg.max_nrhs); asynchronous on the stream.  LQCD_ERR_STATE
 * without a gauge field and clover term, LQCD_ERR_INVALID for host
 * pointers. */
lqcd_status lqcd_training_pair(lqcd_ctx* ctx, float* r, float* e, const double* xstar, const double* x, int nrhs);

/* Right preconditioner of LQCD_SOLVER_FGCR and LQCD_SOLVER_FGMRES_DR (NULL:
 * identity).  The network must belong to this context and outlive its use. */
lqcd_status lqcd_set_preconditioner(lqcd_ctx* ctx, lqcd_net* net);

/* Schwarz alternating procedure (Sec. 5, the SAP preconditioner of the
 * SAP-FGCR solver): the lattice is cut into non-overlapping blocks of
 * block[0] x block[1] x block[2] x block[3] sites, coloured by the parity of
 * the sum of the block coordinates.  Starting from z = 0, each of `ncycle`
 * cycles takes the blocks of colour 0 and then those of colour 1; for one
 * colour the residual rho = r - M z is formed, every block of that colour
 * runs `nmr` minimal-residual iterations on M_B delta = rho_B (M restricted
 * to the block: hops leaving it are dropped, i.e. Dirichlet boundaries) and
 * z += delta on the block.  M = A - kappa H with the kappa and clover of the
 * last lqcd_clover_compute (A = 1 when csw = 0).
 *
 * lqcd_set_preconditioner_sap makes SAP the right preconditioner of
 * LQCD_SOLVER_FGCR (it replaces a network set by lqcd_set_preconditioner,
 * and setting a network replaces SAP); block = NULL switches it off.
 * lqcd_sap_apply computes z = SAP(r) once.  z and r: device pointers to
 * FP32 full fields in the internal layout (lqcd_field_bytes(ctx, LQCD_F32)
 * bytes per parity, even then odd; pack with parity -1), z != r.  Uses the
 * solver vectors of the workspace as scratch; asynchronous on the stream.
 * Requirements (LQCD_ERR_INVALID otherwise): every block extent divides the
 * lattice extent with an even number (>= 2) of blocks per direction, at most
 * 1024 sites per block, ncycle >= 1, nmr >= 1; the context must hold FP32
 * links (LQCD_ERR_STATE). */
lqcd_status lqcd_set_preconditioner_sap(lqcd_ctx* ctx, const int block[4], int ncycle, int nmr);
lqcd_status lqcd_sap_apply(lqcd_ctx* ctx, void* z, const void* r, const int block[4], int ncycle, int nmr);

/* Solve the systems of n contexts (lattices of any sizes, one right-hand
 * side each, canonical FP64 x[i], b[i] on host or device) together with a
 * CG solver: set-up per lattice, then iteration blocks in lockstep on the
 * stream of ctxs[0] (every context uses it during the call); with
 * params->use_graph one CUDA graph holds the block of every lattice still
 * iterating, each lattice on a parallel branch of its own when the contexts
 * are distinct (their kernels then run side by side), and is replayed.  Each lattice stops on its own true residual
 * tol[i] (stats[i]).  Returns the first non-OK status of the lattices. */
lqcd_status lqcd_solve_batch(lqcd_ctx* const* ctxs, int n, double* const* x, const double* const* b,
                             const double* tol, const lqcd_solver_params* params, lqcd_solver_stats* stats);

/* The deflation step of FGMRES-DR (Sec. 7, deflated restart), host only:
 * for M Z = V Hbar with Hbar of nz + 1 rows and nz columns (complex,
 * column-major, leading dimension ldh >= nz + 1, interleaved re/im
 * doubles), the k harmonic Ritz pairs of smallest |theta|, i.e. solutions
 * of Hbar^H Hbar g = theta Hsq^H g with Hsq the leading nz x nz block.
 * theta: k complex (2k doubles); g: nz x k complex, column-major, unit
 * columns.  1 <= k <= nz <= 256.  LQCD_ERR_BREAKDOWN if Hsq is singular or
 * the eigenvalue iteration does not converge.  Needs no GPU. */
lqcd_status lqcd_harmonic_ritz(int nz, const double* hbar, int ldh, int k, double* theta, double* g);

/* ---------------------------------------------------------------------
 * Halo exchange of a sub-domain context (part[mu] > 1 in some direction).
 * The hopping term of a cut lattice needs, for every output site next to a
 * cut boundary, the spin-projected neighbour across it: 12 reals (two colour
 * vectors) per face site and direction, half of a spinor.
 *
 * Face buffers: for each cut mu in increasing order, two segments, side 0
 * then side 1, each at a 256-byte aligned offset (lqcd_halo_layout), of
 * F/2 face sites x 12 reals (FP64 for LQCD_F64, FP32 for LQCD_F32), F =
 * local volume / dims[mu]; structure of arrays over the face sites (F64: 6
 * chunks of double2, F32: 3 chunks of float4).  A face site is indexed by
 * its three coordinates other than mu, lexicographic with the lowest
 * direction fastest, halved (the sites of one parity).  nrhs buffer sets
 * are stored back to back, lqcd_halo_layout's total apart.
 *
 * Exchange: the send segment (mu, 0) goes to the backward neighbour along
 * mu (coord - 1, periodic) and lands in its receive segment (mu, 0); the
 * send segment (mu, 1) goes to the forward neighbour (coord + 1) and lands
 * in its receive segment (mu, 1).  Receive side 0 thus holds the forward
 * hops of the local last slice, side 1 the backward hops of the first.
 * The fermion sign of hops across the global t boundary is applied by the
 * receiver.  Only LQCD_F64 and LQCD_F32 storage. */

/* Byte offsets and lengths of the segments [2 mu + side] of one buffer set
 * (0 for uncut directions) and the set's total size per right-hand side. */
lqcd_status lqcd_halo_layout(const lqcd_ctx* ctx, lqcd_prec prec, size_t off[8], size_t len[8], size_t* total);

/* Send faces of nrhs internal fields `in` of parity `parity` (the parity
 * the hopping term reads) for lqcd_halo_dslash with the same dag: segment
 * (mu, 0) = P psi on the local first slice along mu (the projector of the
 * forward hop), segment (mu, 1) = U_mu^dag P psi on the last slice (the
 * backward hop's projector and this sub-domain's own link).  send: device,
 * nrhs x total bytes.  Asynchronous on the stream. */
lqcd_status lqcd_halo_pack(lqcd_ctx* ctx, void* send, const void* in, int parity, int dag, lqcd_prec prec,
                           int nrhs);

/* The hopping term of a sub-domain with an epilogue, out_p = epi(H_{p,1-p} in):
 *   epi 0: out = a H in;  epi 1: out = a A_pp^{-1} H in;  epi 2: out = A_pp y + a H in
 * (A = 1: a cut context has no clover term), dag: H^dag.  stage 1 runs the
 * interior pass (every hop inside the sub-domain; output sites next to a cut
 * boundary keep a partial sum in out), stage 2 the face pass (adds the faces
 * of recv to those sites and applies the epilogue), stage 0 both.  Between
 * the passes the exchange of the faces can run (recv is read only by the
 * face pass and must hold the neighbours' faces by then).  out, in, y: nrhs
 * internal fields; recv: nrhs face buffer sets.  out must not alias in or y. */
lqcd_status lqcd_halo_dslash(lqcd_ctx* ctx, void* out, const void* in, const void* recv, int parity, int dag,
                             int epi, const void* y, double a, int stage, lqcd_prec prec, int nrhs);

/* FP64 |field|^2 of nrhs internal fields of one parity (parity 0, 1) or
 * full fields (parity -1) of precision prec, per right-hand side, into
 * out[nrhs] (host).  On a sub-domain it is the local part of the global sum
 * (the caller adds the parts, e.g. with an allreduce).  nrhs <= max_nrhs.
 * Synchronises the stream. */
lqcd_status lqcd_norm2(lqcd_ctx* ctx, const void* field, int parity, lqcd_prec prec, int nrhs, double* out);

/* Measured arithmetic peak of GPU `device` in TFLOP/s (2 flops per
 * multiply-add and lane), the roofline denominator of the kernels bound by
 * arithmetic rather than by memory: kind 0 = FP32 multiply-add, 1 = FP32
 * packed two-lane multiply-add, 2 = FP64 multiply-add.  Runs one short and
 * one ~20 ms launch of independent multiply-add chains on a stream of its own
 * (no device memory is allocated; synchronises that stream).  The paper
 * has no counterpart.  LQCD_ERR_INVALID for another kind or a null result. */
lqcd_status lqcd_fma_peak(int device, int kind, double* tflops);

/* Wait for the context's stream and report device-side errors. */
lqcd_status lqcd_sync(lqcd_ctx* ctx);

/* Autotuner: time the hopping kernels of precision `prec` (plain and dagger,
 * x-pay epilogue as in the solvers, with and without the fused norm
 * reduction) at 128, 96, 64 and 32 threads per block on this context's
 * lattice and keep, for each of the four classes, the fastest (a smaller
 * block must win by 2 %) for every later launch of that class.  For the
 * plain classes of the modes with FP32 links (LQCD_F32, LQCD_F16_SPINORS,
 * LQCD_BF16_SPINORS) with recon-12 the candidates also include the
 * shared-memory staged kernel (LQCD_BLOCK_STAGED below), which must win by
 * 2 % as well.  Reducing
 * launches (fused norms, fused CG updates) write one partial sum per block:
 * they are tuned apart from the plain ones, and for them also the sites each
 * thread handles (one wave of resident blocks, the default, or 1, 4 or 16
 * sites per thread; another choice must win by 2 %).  Needs a loaded gauge
 * field; overwrites the solver vectors of the workspace.  best_block (may be
 * NULL) receives the block sizes [2 * dag + reducing], best_sites (may be
 * NULL) the sites per thread of the reducing launches [dag] (0: one wave).
 * Synchronises the stream. */
lqcd_status lqcd_tune(lqcd_ctx* ctx, lqcd_prec prec, int best_block[4], int best_sites[2]);

/* The "block size" that selects the shared-memory staged hopping kernel for
 * a plain class: each block copies the input spinors of a tile of 4 x 2 x 2
 * (y, z, t) rows of all Lx/2 checkerboard sites, and of the tile's six faces,
 * into shared memory with asynchronous copies, then reads every neighbour
 * from there (the neighbour faces of Sec. 5's kernel, staged on chip).  It
 * applies to plain launches with FP32 recon-12 links on an uncut lattice with
 * Lx <= 32, Ly % 4 = Lz % 2 = Lt % 2 = 0; other launches of the class use the
 * gathering kernel at 128 threads.  Its arithmetic is that of the gathering
 * kernel, in the same order (the results are identical). */
#define LQCD_BLOCK_STAGED 1

/* Set the tuner's choices for precision `prec` directly (e.g. ones saved
 * from an earlier lqcd_tune): block[2 * dag + reducing] in {32, 64, 96, 128}
 * or, for the plain classes (indices 0 and 2), LQCD_BLOCK_STAGED; sites[dag]
 * (may be NULL: unchanged) the sites per thread of the reducing launches, 0
 * (one wave of resident blocks) or 1 to 64.  Anything else is
 * LQCD_ERR_INVALID and changes nothing.  No GPU work. */
lqcd_status lqcd_tune_set(lqcd_ctx* ctx, lqcd_prec prec, const int block[4], const int sites[2]);

/* Kernel timing.  While enabled, every hopping-term launch the context
 * issues is bracketed by CUDA events on its stream (graph replays are not
 * recorded).  lqcd_profile_read waits for the stream and returns, for each
 * storage precision (index lqcd_prec), the launches since the last read,
 * their summed device time, and their algorithmic bytes and flops: bytes
 * count every right-hand side's input and epilogue fields and output once
 * per output site, and the links and clover entry once per output site and
 * launch (the compulsory traffic), flops count 1320 per output site and
 * right-hand side (the hopping term alone). */
typedef struct {
    long launches;
    double ms;
    double bytes;
    double flops;
} lqcd_profile_entry;
lqcd_status lqcd_profile_enable(lqcd_ctx* ctx, int enable);
lqcd_status lqcd_profile_read(lqcd_ctx* ctx, lqcd_profile_entry out[LQCD_NPREC]);

/* Kernel timing of a network: while enabled, every layer launch (forward,
 * adjoint) and weight-gradient launch is bracketed by CUDA events on the
 * context's stream (not the layout conversions at the ABI calls; graph
 * replays are not recorded).  lqcd_net_profile_read waits for the stream and
 * fills out[3 * layer + kind] (kind 0 forward, 1 adjoint, 2 weight gradient;
 * nentries >= 3 nlayers) with the launches since the last read, their device
 * time, their compulsory bytes (FP32 input and output activations and each
 * FP32 link once per item) and the flops of the channel contraction (8 per
 * complex multiply-add, 4 C_out x 4 C_in x 3 colours x 9 hops per site and
 * item). */
lqcd_status lqcd_net_profile_enable(lqcd_net* net, int enable);
lqcd_status lqcd_net_profile_read(lqcd_net* net, lqcd_profile_entry* out, int nentries);

/* Message describing the last failure on the calling thread ("" if none). */
const char* lqcd_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LQCD_H */
