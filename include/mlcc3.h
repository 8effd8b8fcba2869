/*
 * mlcc3.h -- C ABI of the MLCC3 triples library (GB300, sm_103a).
 *
 * The library computes the triples (T3, R3, L3) contributions of multilevel
 * CC3 (arXiv 2202.08612, Sec. 3 "Implementation" and the SI equations):
 * the ground-state residual, the right and transpose Jacobian
 * transformations, the transition densities and the oscillator strength.
 * The triples amplitudes are built on the fly per batch of active occupied
 * indices i >= j >= k.  One n_v^3 block per unique batch of the current chunk
 * is held on the device: when every block fits (mlcc3_set_param
 * "chunk_blocks", sized from the free memory by default) that is all of the
 * unique blocks; larger systems are swept in chunks.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Orbitals: occupied first, then virtual (n_mo = N_O + N_V).  Active occupied
 *   orbitals are occupied indices [0, n_o), active virtual orbitals are
 *   virtual indices [0, n_v).
 * Arrays: C row-major, IEEE double, dense.  Every array argument may be a
 *   device pointer or a host pointer (detected per call with
 *   cudaPointerGetAttributes); host arrays are staged through buffers the
 *   context owns, except the Cholesky vectors of mlcc3_build_integrals, which
 *   are copied straight into the context's own transformed copy from device,
 *   pinned or pageable memory (no staging buffer of the largest input).  The
 *   caller keeps ownership of all arrays.
 * Singles: X[A][I] = X^A_I, shape [N_V][N_O].
 * Doubles: the active-pair block X[i][a][L][D] = X^{aD}_{iL}, shape
 *   [n_o][n_v][N_O][N_V] (the paper's N_V N_O n_v n_o sub-block, Sec. 3).
 *   Elements whose two pairs are both active appear twice and must be equal.
 *   Vectors (R, L, rho, sigma, Omega) hold one number per unique excitation,
 *   the bra <mu| being biorthonormal to E_ai E_bj |HF>; the trial vector's
 *   doubles operator is 1/2 sum Rbar E E with Rbar = (1 + delta_ij delta_ab) R.
 * Densities: [n_mo][n_mo], D_pq pairs with the operator element A_pq of the
 *   T1-transformed one-electron operator, sum_pq D_pq A_pq.
 * Outputs are overwritten with the triples contribution only; the caller adds
 *   it to its CCSD-level quantity.
 * Errors: every function returns MLCC3_OK (0) or a negative MLCC3_ERR_* code;
 *   mlcc3_last_error() returns a message for the calling thread.  Nothing is
 *   thrown or aborted across the ABI.  Calls on one context are serialised on
 *   the context's stream and are not thread safe.
 */
#ifndef MLCC3_H
#define MLCC3_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MLCC3_OK 0
#define MLCC3_ERR_ARG (-1)            /* bad dimension, null pointer, bad mode */
#define MLCC3_ERR_CUDA (-2)           /* a CUDA call failed */
#define MLCC3_ERR_OOM (-3)            /* device allocation failed */
#define MLCC3_ERR_SINGULAR_DENOM (-4) /* |eps^{abc}_{ijk} - omega| < 1e-3 */
#define MLCC3_ERR_TIMEOUT (-5)        /* a device wait gave up */
#define MLCC3_ERR_STATE (-6)          /* call order: integrals not built */

/* Arithmetic of the contractions.  MLCC3_FP64: every product and sum in
 * IEEE double.  MLCC3_SPLIT_BF16X3: integral-amplitude products on the
 * tensor cores from hi/lo bfloat16 splits with FP32 accumulation;
 * denominators and final reductions stay in FP64.
 * An FP16 hi/lo split is not offered: FP16's five exponent bits put the low
 * half of an operand of magnitude below about 2^-3 (most amplitudes and
 * integrals here) into the subnormal range, where it loses the bits the
 * split exists to keep, unless every operand is rescaled per block; the
 * bfloat16 split has FP32's exponent range and needs no scaling.  The value 2
 * is rejected with MLCC3_ERR_ARG. */
#define MLCC3_FP64 0
#define MLCC3_SPLIT_BF16X3 1

typedef struct mlcc3_ctx mlcc3_ctx;

typedef struct {
  int64_t n_occ;     /* N_O */
  int64_t n_vir;     /* N_V */
  int64_t n_act_occ; /* n_o, 0 <= n_o <= min(N_O, 32) */
  int64_t n_act_vir; /* n_v, 0 <= n_v <= min(N_V, 1024) */
  int64_t n_chol;    /* N_J, number of Cholesky vectors */
  /* [N_O] host array, 1 = core orbital; NULL = no core-valence separation.
   * With a mask, the Jacobian transformations and the densities skip every
   * batch i,j,k without a core index (Sec. 3, CVS). Copied at create. */
  const uint8_t *core_mask;
} mlcc3_dims;

/* Create a context on the current device.  `cuda_stream` is a cudaStream_t
 * (NULL = legacy default stream) on which every later call runs. */
int mlcc3_create(mlcc3_ctx **out, const mlcc3_dims *dims, int precision, void *cuda_stream);
void mlcc3_destroy(mlcc3_ctx *ctx);
const char *mlcc3_last_error(void);

/* Set the ground-state amplitudes and build the T1-transformed integral
 * blocks (Sec. 2: H = exp(-T1) H exp(T1); SI: g_PQRS = sum_J L^J_PQ L^J_RS).
 *   chol [N_J][n_mo][n_mo]  Cholesky vectors of (pq|rs), symmetric in p,q
 *   t1   [N_V][N_O]         singles amplitudes t^A_I
 *   eps  [n_mo]             orbital energies (canonical, Sec. 2 eps^{abc}_{ijk})
 *   t2c  [n_o][n_v][N_O][N_V]  t^{aD}_{iL}
 *   t2x  [n_o][n_v][N_O][N_V]  t^{aD}_{Li} (only the transition density reads it)
 * Must precede every other compute call; may be repeated. */
int mlcc3_build_integrals(mlcc3_ctx *ctx, const double *chol, const double *t1,
                          const double *eps, const double *t2c, const double *t2x);

/* Triples contributions to the ground-state residual (Sec. 3, Eq. tau3, SI):
 *   omega1 [N_V][N_O], omega2 [n_o][n_v][N_O][N_V]. */
int mlcc3_triples_omega(mlcc3_ctx *ctx, double *omega1, double *omega2);

/* Right Jacobian transformation rho = A R, triples part (Sec. 3, Eq. R3,
 * Eqs. ups_v/ups_o, SI), for n_vec trial vectors at frequencies omega[n_vec]
 * (host array).  R1 [n_vec][N_V][N_O], R2 [n_vec][n_o][n_v][N_O][N_V];
 * rho1, rho2 the same shapes. */
int mlcc3_jacobian_right(mlcc3_ctx *ctx, int n_vec, const double *omega, const double *R1,
                         const double *R2, double *rho1, double *rho2);

/* Transpose Jacobian transformation sigma = L^T A, triples part (Sec. 3, SI
 * L3 and sigma equations); the exact adjoint of mlcc3_jacobian_right under
 * the unique-element inner product. Shapes as for mlcc3_jacobian_right. */
int mlcc3_jacobian_left(mlcc3_ctx *ctx, int n_vec, const double *omega, const double *L1,
                        const double *L2, double *sigma1, double *sigma2);

/* Triples parts of the ground-state density D^{0-0} and of the left and
 * right transition densities D^{m-0}, D^{0-m} of one state (Sec. 3,
 * Eq. DL_oo, SI densities).  lam1/lam2 are the ground-state multipliers
 * (lambda3 is built from them with omega = 0); D00_in [n_mo][n_mo] is the
 * caller's CCSD-level ground-state density including the reference
 * (2 delta_IJ), used by the normalisation term of D^{0-m}.
 * Outputs D00_T, Dm0_T, D0m_T [n_mo][n_mo]. */
int mlcc3_transition_density(mlcc3_ctx *ctx, double omega, const double *lam1,
                             const double *lam2, const double *R1, const double *R2,
                             const double *L1, const double *L2, const double *D00_in,
                             double *D00_T, double *Dm0_T, double *D0m_T);

/* Ground-state multipliers (Sec. 2: the lambda equations lambda^T A(0) = -eta,
 * eta without a triples part): the triples part of lambda^T A at omega = 0,
 * i.e. mlcc3_jacobian_left of the one vector (lam1, lam2) at omega = 0, the
 * skip rule of a core mask off (the ground state is not core-valence
 * separated).  lam1 [N_V][N_O], lam2 [n_o][n_v][N_O][N_V]; eta1, eta2 the same
 * shapes, overwritten. */
int mlcc3_multiplier_transformation(mlcc3_ctx *ctx, const double *lam1, const double *lam2,
                                    double *eta1, double *eta2);

/* Triples part of the ground-state density D^{0-0} alone (SI: the D^{m-0}
 * blocks kl, ld, LD, cd with lambda3, the L3 formula at omega = 0 on the
 * multipliers, in place of L3), without the transition densities of a state.
 * lam1, lam2 as above; D00_T [n_mo][n_mo], overwritten. */
int mlcc3_ground_density(mlcc3_ctx *ctx, const double *lam1, const double *lam2, double *D00_T);

/* The densities of n_states states in one call (same definitions as
 * mlcc3_transition_density): tau, lambda3 and D^{0-0}, which do not depend on
 * the state, are built once per block of batches and shared; L3, R3, D^{m-0}
 * and D^{0-m} are per state.  omega [n_states] (host); R1, L1
 * [n_states][N_V][N_O]; R2, L2 [n_states][n_o][n_v][N_O][N_V]; D00_T
 * [n_mo][n_mo]; Dm0_T, D0m_T [n_states][n_mo][n_mo].  Every state follows
 * the context's skip rule ("cvs"): pass valence and core states in separate
 * calls. */
int mlcc3_transition_densities(mlcc3_ctx *ctx, int n_states, const double *omega,
                               const double *lam1, const double *lam2, const double *R1,
                               const double *R2, const double *L1, const double *L2,
                               const double *D00_in, double *D00_T, double *Dm0_T, double *D0m_T);

/* Excitation-energy Rayleigh quotient of one state (Sec. 2: the CC3
 * excitation energies are eigenvalues of the omega-dependent Jacobian A(omega);
 * the Davidson iterations estimate them from trial vectors):
 *   omega_rq = (sd_part + <L, rho_T(omega)>) / <L, R>
 * rho_T = the triples part of A(omega) R (as mlcc3_jacobian_right), sd_part =
 * the caller's <L, A_SD R> (its singles-doubles Jacobian, which the library
 * does not hold), <,> the unique-element inner product (weight 1/2 on the
 * doubles elements the active-pair block stores twice).  R1, R2, L1, L2 as one
 * vector of mlcc3_jacobian_right / _left; the dot products are FP64 on the
 * device; *omega_rq is a host scalar.  MLCC3_ERR_ARG when <L, R> = 0. */
int mlcc3_rayleigh_quotient(mlcc3_ctx *ctx, double omega, const double *R1, const double *R2,
                            const double *L1, const double *L2, double sd_part, double *omega_rq);

/* Length-gauge oscillator strength of one state from its full (CCSD-level +
 * triples) transition densities (Sec. 2 transition moments):
 *   f = 2/3 omega sum_x (sum_pq D0m_pq mu~^x_pq)(sum_pq Dm0_pq mu~^x_pq),
 *   mu~ = (1 - t1) mu (1 + t1).  mu [3][n_mo][n_mo]; f is a host scalar. */
int mlcc3_oscillator_strength(mlcc3_ctx *ctx, double omega, const double *D0m,
                              const double *Dm0, const double *mu, double *f);

/* Batched sweep (Sec. 3: the triples right transformation is the part of a
 * Davidson iteration that scales as N_V n_v^3 n_o^3; the paper applies it per
 * trial vector): the right Jacobian transformations of several systems, each
 * with its own context and possibly different (n_o, n_v, N_V), and of all
 * their trial vectors, run as one CUDA graph launch.  Each system runs on its
 * own stream, forked from and joined back into `cuda_stream` inside the graph,
 * so that small systems fill the GPU together.
 *   mlcc3_sweep_create   contexts (built, same device, each once); with tune,
 *                        the first run times, per system, the candidates 0, 2,
 *                        4, 8 of "bstc_fill" on one trial vector and keeps the
 *                        fastest, then keeps the faster of the concurrent and
 *                        the serial graph.  Contexts whose "chunk_blocks" is 0
 *                        get a share of half the free device memory.
 *   mlcc3_sweep_set_system  n_vec trial vectors of system `sys`: R1, R2, rho1,
 *                        rho2 are DEVICE arrays with the shapes of
 *                        mlcc3_jacobian_right; the graph reads and writes these
 *                        addresses, so they must stay valid.
 *   mlcc3_sweep_run      omega[sum of n_vec] (host, system-major).  The first
 *                        run (and the first after mlcc3_sweep_set_system,
 *                        mlcc3_build_integrals or a change of "chunk_blocks" on
 *                        any of the contexts) runs eagerly once, tunes, and
 *                        captures the graph; later runs copy omega to the
 *                        device and replay it.  Results as mlcc3_jacobian_right.
 *                        Blocks the host until the graph has finished.
 *   mlcc3_sweep_info     a JSON summary (graph nodes, tuning choices and times).
 * Calls on the contexts themselves may be mixed with sweeps; a sweep does not
 * rely on their state (it rebuilds tau in every replay).  Not thread safe. */
typedef struct mlcc3_sweep mlcc3_sweep;
int mlcc3_sweep_create(mlcc3_sweep **out, mlcc3_ctx *const *ctxs, int n_sys, int tune,
                       void *cuda_stream);
int mlcc3_sweep_set_system(mlcc3_sweep *sweep, int sys, int n_vec, const double *R1,
                           const double *R2, double *rho1, double *rho2);
int mlcc3_sweep_run(mlcc3_sweep *sweep, const double *omega);
int mlcc3_sweep_info(mlcc3_sweep *sweep, char *buf, size_t len);
void mlcc3_sweep_destroy(mlcc3_sweep *sweep);

/* Tuning parameters of a context (no counterpart in the paper; results stay
 * within the precision mode's error bounds for every accepted value):
 *   "tc_kcap"  longest FP32 accumulation chain of the split-precision tensor
 *              core kernel, in 64-wide K blocks, for the contractions whose
 *              partial results are summed in FP64 (back-contractions,
 *              densities, Cholesky-index builds); 0 = unlimited.  The tensor
 *              cores accumulate with truncation, so the error of a chain
 *              grows with its length.  Default 16 (K = 1024).  Range 0..4096.
 *   "tc_group"  most unique batches stacked along N in one tile of the
 *              split-precision triples build: batches that share the two
 *              occupied indices outside the tile's single virtual position
 *              share every integral-side operand, so up to tc_group of their
 *              amplitude operands (one n_v-wide box each) fill one wider MMA.
 *              Default 4.  Range 1..4 (capped at 256 columns).
 *   "tc_wide_bn"  tile width (columns) of the split-precision pair
 *              contractions whose output has more than 256 columns (the sigma
 *              singles intermediates, N = N_V): 256 (two pipeline stages fit in
 *              shared memory), 160 or 128 (three stages).  Default 256.  Set it
 *              before mlcc3_build_integrals: the operands converted there carry
 *              the width, and a later change makes the transformations fail with
 *              MLCC3_ERR_ARG.
 *   "tc_persist_from"  tensor-core launches with more output tiles than this
 *              run the persistent kernel (one CTA per SM looping over tiles,
 *              accumulator double-buffered in TMEM); smaller ones run one CTA
 *              per tile.  Default 304; 0 always persistent.
 *   "release_scratch"  0 (default): the scratch of a call (triples blocks of
 *              a chunk, their split copies, intermediates; sized for the
 *              largest call so far) stays allocated for the next call and
 *              keeps tau and the layouts cached.  1: every call ends by freeing
 *              all scratch that mlcc3_build_integrals did not create, so that
 *              the device holds only the integral blocks between calls and the
 *              peak is the largest single call's, not the sum over the kinds of
 *              call (the transition densities need more than the Jacobian
 *              transformations); each call then allocates its scratch again.
 *              A sweep needs contexts with 0 (MLCC3_ERR_STATE otherwise).
 *   "bstc_big_from"  split-precision contractions with one reduction index
 *              and at least this many multiply-adds per launch (M N K summed
 *              over the launch's items) run on 128 x 128 CUDA-core tiles with
 *              FP32 accumulation over K ranges of at most 1024 (summed in
 *              FP64); the others on 64 x 64 tiles.  Default 10^9; 0: never.
 *   "finish_fused"  1 (default): in the split-precision mode the finish of a
 *              triples build (rank-1 terms, denominators) and the contravariant
 *              transform of its blocks run as one pass over tile orbits; 0: as
 *              a streaming finish followed by the transform.  Same results up
 *              to rounding order.
 *   "cvs"      1 (default): a context created with a core mask applies the CVS
 *              skip rule (mlcc3_dims.core_mask) in the Jacobian transformations
 *              and the densities; 0: the same context treats its vectors as
 *              valence states (every batch kept), so that the valence and the
 *              core states of one system share one integral build.  1 needs a
 *              core mask.
 *   "shard_count", "shard_index"  batch sharding across GPUs (default 1, 0):
 *              mlcc3_triples_omega, the Jacobian transformations, the multiplier
 *              transformation and the sweep run over the unique batches of shard
 *              shard_index only (mlcc3_shard_batches gives the list), so that
 *              one context per GPU, each with its own shard_index, computes
 *              partial outputs whose sum over the shards (one all-reduce) is the
 *              unsharded result: every one of these outputs is linear in the
 *              per-batch terms.  The densities are not sharded (their
 *              normalisation multiplies two sums over batches); they always run
 *              over every batch.  A compute call with shard_index >= shard_count
 *              returns MLCC3_ERR_ARG.
 *   "tc_wait_clocks"  clock limit of the split-precision tensor-core kernel's
 *              pipeline waits (a stage to fill or free, an accumulator to finish
 *              or to be read); 0 (default) is about one second.  On expiry the
 *              kernel stops issuing work, waits for the copies and MMAs it has
 *              issued, frees its tensor memory and returns; the call then
 *              returns MLCC3_ERR_TIMEOUT and drops the context's cached tau, and
 *              the context stays usable.  A small value (a few clocks) makes the
 *              waits run out: failure-path testing only.  Range 0..2^40.
 *   "bstc_fill"  split-K target of the FP64 strided contractions: a launch
 *              with few output tiles and a long reduction splits K until about
 *              bstc_fill x 152 CTAs run; 0 never splits.  Default 4.  Range 0..64.
 *   "chunk_blocks"  most unique batches whose triples blocks (n_v^3 each) the
 *              context holds on the device at once; larger systems are swept
 *              in chunks (the densities by ranges of occupied indices, which
 *              rebuilds the blocks a range shares with others).  0 (default)
 *              sizes the chunks from the free device memory at create.
 * Returns MLCC3_ERR_ARG for an unknown name or a value out of range. */
int mlcc3_set_param(mlcc3_ctx *ctx, const char *name, long long value);

/* CNTO matrices of one excited state (Sec. 2, Eqs. M and N; the active space
 * of MLCC3 is spanned by the leading eigenvectors of their state averages):
 *   M_ij = sum_a R^a_i R^a_j + 1/2 sum_{abk} (1 + delta_{ai,bk} delta_ij) R^{ab}_{ik} R^{ab}_{jk}
 *   N_ab = sum_i R^a_i R^b_i + 1/2 sum_{cij} (1 + delta_{ai,cj} delta_ab) R^{ac}_{ij} R^{bc}_{ij}
 * R1 [N_V][N_O]; R2 [N_V][N_O][N_V][N_O] = R^{AB}_{IJ} in full storage (a CCSD
 * excitation vector, symmetric under (A,I) <-> (B,J)); M [N_O][N_O] and
 * N [N_V][N_V] are overwritten.  Device pointers only (MLCC3_ERR_ARG
 * otherwise); FP64; runs on `cuda_stream` and returns when it has finished.
 * No context is needed. */
int mlcc3_cnto_matrices(int64_t n_occ, int64_t n_vir, const double *R1, const double *R2,
                        double *M, double *N, void *cuda_stream);

/* C = A B^T in FP64 accuracy on the BF16 tensor cores (the contractions of
 * Sec. 3 at FP64 accuracy, by error-free splitting after Ozaki, Ogita, Oishi
 * and Rump): every row of A and of B is scaled by a power of two and written
 * as `slices` balanced base-256 digits (integers in [-128, 128], exact in
 * bfloat16); the digit slices are multiplied on tcgen05 with FP32 sums that
 * are exact over K chains of up to 1024, the chains added in FP64; the digit
 * pairs (t, u) with t + u < slices are kept, so the normwise relative error is
 * about 2^-(8 slices) (slices = 5: about 1e-12).  A [M][K] with rows lda
 * apart, B [N][K] rows ldb apart, C [M][N] rows ldc apart, all FP64 device
 * arrays (MLCC3_ERR_ARG otherwise, and for slices outside 2..6 or a leading
 * dimension below the row length).  Allocates its temporaries (about
 * 2 slices (M + N) K bytes), runs on `cuda_stream` and returns when C holds
 * the product; MLCC3_ERR_OOM when an allocation fails, MLCC3_ERR_TIMEOUT when
 * a tensor-core pipeline wait ran out (C is then not valid). */
int mlcc3_fp64emu_gemm(const double *A, long long lda, const double *B, long long ldb, double *C,
                       long long ldc, int M, int N, int K, int slices, void *cuda_stream);

/* Triples residual without allocating (no counterpart in the paper).
 * Some callers cannot allocate device memory at the moment they call: a
 * solver loop whose host application gives all device memory to its own pool
 * at start-up and forbids a cudaMalloc afterwards, or one that cannot afford
 * the implicit device synchronisation that cudaMalloc/cudaFree can bring.
 * This entry point returns the same omega1 and
 * omega2 as mlcc3_triples_omega but takes all of its scratch (the unique-batch
 * tau blocks, their contravariant copies, the doubles accumulator and the
 * index tables) from one fixed 32 MiB device array compiled into the
 * library, which every device that loads the library holds until exit.  It
 * calls no cudaMalloc, cudaFree or other allocating routine.
 * It computes in FP64 (the FP64 kernels of the MLCC3_FP64 mode) and takes
 * MLCC3_FP64 contexts only: a split-precision context gets MLCC3_ERR_STATE.
 * Requirements: mlcc3_build_integrals has run on `ctx` (that call allocates,
 * so make it during set-up); omega1/omega2 are device pointers (host arrays
 * would need staging buffers); the current device is the context's; and
 * 2 n_batch n_v^3 + n_o n_v N_O N_V doubles plus the index tables fit in
 * 32 MiB (n_batch = unique i >= j >= k, i = j = k excluded) -- larger systems
 * get MLCC3_ERR_ARG with the required size in mlcc3_last_error().
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * The address is kept until exit: cudaDeviceReset while the library is
 * loaded is not supported.
 * Every call shares the array and finds the previous call's contents in it
 * (the accumulators are cleared on entry); calls that overlap on the GPU
 * (other streams, other contexts on the same device) race on it and must be
 * serialised by the caller. */
int mlcc3_triples_omega_static(mlcc3_ctx *ctx, double *omega1, double *omega2);

/* The unique batches i >= j >= k (i = j = k excluded; with cvs != 0 and a
 * core_mask [n_act_occ] only those with a core index) that shard shard_index
 * of shard_count processes under the "shard_count"/"shard_index" parameters:
 * longest-processing-time assignment by the number of distinct orderings of a
 * batch (6, or 3 with two equal indices), in list order.  Writes up to
 * max_batches (i, j, k) triples to ijk[3 * max_batches] and returns the
 * shard's batch count, or MLCC3_ERR_ARG.  Host only: no GPU is needed. */
int mlcc3_shard_batches(int n_act_occ, const uint8_t *core_mask, int cvs, int shard_count,
                        int shard_index, int *ijk, int max_batches);

/* Diagnostics (used by the test-suite).  mlcc3_debug_fetch copies the first
 * n doubles of a named device buffer of the context into `host` (integral
 * blocks "Lt", "Gv", "Gb", "Go", "Gx", "Govov", "F", or a named scratch
 * buffer such as "tau"); MLCC3_ERR_ARG for an unknown name or n too large.
 * mlcc3_debug_nbatches returns the number of unique batches i >= j >= k
 * (i = j = k excluded), or -1 for a null context. */
int mlcc3_debug_fetch(mlcc3_ctx *ctx, const char *name, double *host, size_t n);
long long mlcc3_debug_nbatches(mlcc3_ctx *ctx);

/* Launch accounting.  The context counts every kernel it launches, per
 * kernel name, with the floating-point operations of the launch.
 * mlcc3_debug_profile(ctx, 1) clears the counters and additionally brackets
 * each launch with CUDA events on the context's stream (timings are summed
 * when a call finishes); mlcc3_debug_profile(ctx, 0) clears and stops timing.
 * mlcc3_debug_kernel_stats reports entry `index` (0-based, in name order):
 * its name (NUL-terminated, truncated to name_len), launches, summed event
 * milliseconds (0 without profiling) and flops; MLCC3_ERR_ARG past the end. */
int mlcc3_debug_profile(mlcc3_ctx *ctx, int enable);

/* C = A B^T on the split-precision tensor-core path (the contraction kernel
 * of MLCC3_SPLIT_BF16X3, persistent form): A [M][K], B [N][K], C [M][N],
 * row-major FP64 device arrays.  A and B are split into hi/lo bfloat16 pairs;
 * the three products A_hi B_hi + A_hi B_lo + A_lo B_hi accumulate in FP32.
 * Diagnostic: it allocates temporaries and synchronises the default stream. */
int mlcc3_debug_tc_gemm(const double *A, const double *B, double *C, int M, int N, int K);
int mlcc3_debug_kernel_stats(mlcc3_ctx *ctx, int index, char *name, size_t name_len,
                             long long *launches, double *ms, double *flops);

#ifdef __cplusplus
}
#endif
#endif /* MLCC3_H */
