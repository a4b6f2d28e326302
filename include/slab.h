/*
 * slab.h -- C ABI of the GB300 slab factor+solve library (libslab.so).
 *
 * The library factors and solves the finite-difference system A u = f of a
 * second-order elliptic PDE on the unit square/cube with homogeneous Dirichlet
 * data, by the two-level slab method of Yesypenko & Martinsson (SlabLU):
 *   Stage 1 (Sec. 3, Algorithm 3): eliminate the interior of every slab of
 *     width b, giving the block-tridiagonal reduced matrix T on the slab
 *     interfaces (eqs. T11-T35), formed here exactly and densely;
 *   Stage 2 (Sec. 4, Algorithm 1): block (Cholesky) LU sweep over T;
 *   Solve (Algorithm 4): reduced load f~ (eqs. f1-f5), sweeping solve
 *     (Algorithm 2), interior back-solve (eq. usol_even),
 * with an FP64 stencil residual and iterative refinement on top of a factor
 * kept in FP32 or FP64.
 *
 * Operator (Sec. 2.1 eq. "discretiation" with the sign of eq. "var_helm"):
 *   (A u)_P = n^2 sum_{faces P~Q} k_PQ (u_P - u_Q) + q_P u_P,   u = 0 on the boundary,
 *   k_PQ = (kappa_P + kappa_Q)/2 (DIFFUSION, CONVECTION) or 1 (POISSON, HELMHOLTZ),
 *   q_P = 0, or -(omega / c_P)^2 for HELMHOLTZ.
 * CONVECTION (2-D) adds a first-order term, -div(kappa grad u) + beta . grad u (a second-order
 * elliptic operator of the class of Sec. 1.1, eq. "bvp"), by central differences at P:
 *   (A u)_P += sum_a beta_a(P) (u_{P+e_a} - u_{P-e_a}) n / 2,
 * so A is not symmetric: T_{q+1,q} != T_{q,q+1}^T, and the adjoint solves with A^T.
 *
 * Conventions shared by every entry point
 *   - Node fields (kappa, c) have (n+1)^d FP64 entries, C order [z][y][x]
 *     (x fastest), boundary nodes included.
 *   - Vectors (f, u, r, lambda) have k blocks of (n-1)^d FP64 entries over the
 *     interior nodes, layout [k][z][y][x], contiguous.
 *   - Interface vectors (f~, u~) have k blocks of N_I*(n-1)^(d-1) FP64 entries,
 *     layout [k][q][j]: interface q = 0..N_I-1 is the grid plane x = (q+1) b,
 *     its nodes j ordered by y (then z), y fastest.
 *   - Unless a parameter says "host", every pointer is a DEVICE pointer owned
 *     by the caller.  With k == 0 right-hand sides a call does nothing and
 *     its vector pointers may be NULL.  Calls are asynchronous on opts.stream except where a
 *     host output is requested; those synchronise that stream before return.
 *   - The handle owns all factor memory; release it with slab_destroy().
 *   - No C++ exception crosses the ABI.  Errors are returned as slab_status;
 *     the first CUDA error is also latched in the handle (slab_last_error).
 *   - A handle may be used by one host thread at a time.
 */
#ifndef SLAB_H
#define SLAB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SLAB_OK = 0,
    SLAB_EINVAL = 1,        /* bad argument: b does not divide n, b < 2, k < 0, NULL pointer ... */
    SLAB_ENOMEM = 2,        /* device allocation failed */
    SLAB_ESINGULAR = 3,     /* non-positive / zero pivot in a factorisation */
    SLAB_ENOCONV = 4,       /* refinement did not reach opts.rtol within opts.max_refine steps */
    SLAB_ETIMEOUT = 5,      /* a bounded device-side wait gave up */
    SLAB_ECUDA = 6,         /* a CUDA runtime call failed */
    SLAB_EUNSUPPORTED = 7   /* valid request this build does not implement */
} slab_status;

typedef enum { SLAB_POISSON = 0, SLAB_DIFFUSION = 1, SLAB_HELMHOLTZ = 2, SLAB_CONVECTION = 3 } slab_kind;

typedef enum {
    SLAB_PREC_FP64 = 0,     /* factor and solves in FP64 (the plain FP64 GPU path) */
    SLAB_PREC_FP32 = 1,     /* factor and solves in FP32; FP64 residual + refinement */
    SLAB_PREC_TF32 = 2,     /* as FP32, but the factor's tensor-core products run in one TF32 pass
                               (10-bit mantissa) instead of the 3xTF32 split; the solves keep the
                               split.  Trades refinement steps for factor time. */
    SLAB_PREC_FP64_TC = 3   /* interface_prec only: FP64 data, the interface elimination's products
                               FP64-accurate on the tensor cores (slab_fp64_tc_gemm) */
} slab_precision;

/*
 * Elimination order of the block-tridiagonal reduced matrix T in Stage 2.
 * SWEEP: the sequential block elimination of Algorithm 1 (one block after another).
 * ODDEVEN: the odd-even order the paper names as the more parallel alternative
 * (Sec. 4 remark on the elimination order; conclusion): log2(N_I) levels, each
 * eliminating every other remaining block in one batch; Cholesky based, so POISSON
 * and DIFFUSION only (SLAB_EUNSUPPORTED for HELMHOLTZ and CONVECTION).  It holds about 9 s_pad^2
 * numbers per interface in the factor versus about 5 for SWEEP.
 * ODDEVEN does about 4x the dense flops of SWEEP but in log2(N_I) batched levels, which pays
 * on the tensor-core (FP32) path; on the SIMT FP64 path SWEEP is faster.
 * AUTO: for POISSON / DIFFUSION with N_I >= 4 and an FP32 interface system, whichever order a cost
 * model (latency of the s_pad / 64 panel steps on the critical path plus the dense flops) predicts
 * faster -- ODDEVEN for many small interface blocks (e.g. 2-D n = 2048, b = 32), SWEEP for few
 * large ones (e.g. 3-D n = 96, b = 8); SWEEP otherwise.
 */
typedef enum {
    SLAB_STAGE2_AUTO = 0,
    SLAB_STAGE2_SWEEP = 1,
    SLAB_STAGE2_ODDEVEN = 2
} slab_stage2;

typedef struct {
    int dim;                /* 2 or 3 */
    int n;                  /* grid intervals per side, h = 1/n, (n-1)^d unknowns */
} slab_grid;

typedef struct {
    int kind;               /* slab_kind */
    const double* kappa;    /* device, (n+1)^d nodes; DIFFUSION and CONVECTION (NULL otherwise) */
    const double* c;        /* device, (n+1)^d nodes; HELMHOLTZ only (NULL otherwise) */
    double omega;           /* HELMHOLTZ angular frequency */
    const double* beta;     /* device, 2 x (n+1)^2 nodes: the velocity components beta_x then
                               beta_y, each C order [y][x]; CONVECTION only (never read for the
                               other kinds, so callers built before this field may omit it) */
} slab_coeffs;

typedef struct {
    int factor_prec;        /* slab_precision */
    int pivot;              /* row choice of the interface elimination of HELMHOLTZ and CONVECTION
                               (the Gauss-Jordan sweep): 0 = tournament pivoting over all remaining
                               rows (default); 1 = pivot rows restricted to each 64-row diagonal
                               block (partial pivoting inside it only), which skips the tournament and
                               suits diagonally dominant interface systems (diffusion-dominated
                               convection, cell Peclet number below 1).  Other values: SLAB_EINVAL;
                               ignored by the Cholesky-based kinds */
    double rtol;            /* refinement target for max_k ||f - A u||_2 / ||f||_2 */
    int max_refine;         /* refinement steps after the first solve (0: a single pass) */
    int krylov;             /* 0: plain refinement u += A_f^{-1} (f - A u); m > 0: restarted GMRES(m)
                               in FP64 with the factor as right preconditioner (for operators
                               where the FP32 factor's error times the conditioning is not small,
                               e.g. Helmholtz); max_refine then bounds the preconditioner
                               applications after the first.  0..200, else SLAB_EINVAL */
    void* stream;           /* cudaStream_t all work is ordered on (NULL: legacy default) */
    int profile;            /* 1: time every kernel launch from the start (see slab_profile) */
    int stage2;             /* slab_stage2 */
    int interface_prec;     /* slab_precision of Stage 2 (the interface elimination and sweep),
                               or -1: FP64 for HELMHOLTZ with an FP32 factor, else factor_prec;
                               SLAB_PREC_FP64_TC: FP64 with tensor-core products (see above).
                               FP32 slab trees with an FP64 interface system is the mixed mode;
                               an FP64 factor with an FP32 interface is SLAB_EINVAL */
} slab_opts;

typedef struct slab_handle slab_handle;

/* Fill every field of opts with the defaults: FP32 factor, pivot 0, rtol 1e-10, max_refine 30,
 * krylov 0, default stream (NULL), profile 0, SLAB_STAGE2_AUTO, interface_prec -1.
 * slab_factor with opts == NULL uses exactly these. */
void slab_default_opts(slab_opts* opts);

/*
 * Factor A (Algorithm 3): Stage 1 for every slab in parallel, assembly of the
 * reduced matrix T, Stage 2 (Algorithm 1's sweep or the odd-even order, opts.stage2).  b is the interface spacing:
 * interfaces at x = q b, q = 1..n/b-1, slab interiors b-1 nodes wide.
 * Requires dim 2 or 3, b >= 2, n % b == 0 and n/b >= 2 (SLAB_EINVAL otherwise).  In 2-D the slab
 * interior width b - 1 is at most 32 (SLAB_EUNSUPPORTED otherwise); HELMHOLTZ or CONVECTION in 3-D,
 * and SLAB_STAGE2_ODDEVEN with HELMHOLTZ or CONVECTION, are SLAB_EUNSUPPORTED.  POISSON and DIFFUSION are factored by
 * Cholesky (slab separators and Stage 2); HELMHOLTZ (indefinite) and CONVECTION (nonsymmetric) by
 * Gauss-Jordan with partial pivoting in the slab separators, and in Stage 2 (Algorithm 1 as printed)
 * by a blocked Gauss-Jordan elimination of [S_j | T_{j,j+1} | I] over [T_{j+1,j} | T_{j+1,j+1}] with
 * tournament pivoting (64-column panels; each panel's pivot rows are the winners of pairwise
 * partial-pivoting eliminations over groups of 128 candidate rows; opts.pivot = 1 takes them from the
 * diagonal block instead), in opts.factor_prec.  CONVECTION keeps both orientations of every slab
 * coupling so that the same factors also solve with A^T (slab_adjoint).  A zero / non-positive pivot
 * returns SLAB_ESINGULAR.  kappa/c/beta are read during the call only.  On success
 * *out is a new handle.  Synchronises opts->stream (returns after the factor).
 */
slab_status slab_factor(const slab_grid* grid, const slab_coeffs* coeffs, int b,
                        const slab_opts* opts, slab_handle** out);

/*
 * Solve A u = f for k right-hand sides (Algorithm 4 + iterative refinement).
 * f, u: device, [k][(n-1)^d]; u is overwritten.  relres_out: HOST, k entries
 * (may be NULL) receiving ||f - A u||_2/||f||_2; iters_out: HOST (may be NULL)
 * receiving the number of refinement steps taken.  Returns SLAB_ENOCONV when
 * max_refine steps did not reach rtol, when the residual stagnated (two steps without halving
 * the worst relative residual), or when it is not finite (relres_out then holds NaN); u holds
 * the last iterate.
 */
slab_status slab_solve(slab_handle* h, const double* f, double* u, int k,
                       double* relres_out, int* iters_out);

/*
 * Batches of independent problems (uneven sizes allowed; the batched adjoint workload).
 * slab_factor_batched factors count problems: problem i has grids[i], coeffs[i], b[i] and
 * opts (opts->stream is ignored: every handle gets a stream of its own, created here and
 * destroyed by slab_destroy).  Up to `workers` host threads (0: 8) drive the problems
 * concurrently, so small problems overlap on the GPU.  out[i] receives the handle, or NULL
 * if problem i failed; the first failure's status is returned (the other handles stay valid
 * and must still be destroyed).  Synchronises before returning.
 */
slab_status slab_factor_batched(int count, const slab_grid* grids, const slab_coeffs* coeffs, const int* b,
                                const slab_opts* opts, int workers, slab_handle** out);

/*
 * slab_solve on every handle of a batch: f[i], u[i] device pointers ([k[i]][N_i]),
 * relres_out[i] host arrays of k[i] entries (or NULL), iters_out host, count entries (or NULL).
 * Returns the first non-OK status (SLAB_ENOCONV included); all problems are attempted.
 */
slab_status slab_solve_batched(int count, slab_handle* const* h, const double* const* f, double* const* u,
                               const int* k, double* const* relres_out, int* iters_out, int workers);

/* slab_adjoint on every handle of a batch (dLdkappa[i] may be NULL).  Status as slab_solve_batched;
 * synchronises every handle's stream before returning. */
slab_status slab_adjoint_batched(int count, slab_handle* const* h, const double* const* dLdu,
                                 const double* const* u, double* const* lambda, double* const* dLdkappa,
                                 const int* k, int workers);

/* r = f - A u in FP64 for k vectors (stencil kernel; the eq. "discretiation" operator). */
slab_status slab_apply_residual(slab_handle* h, const double* u, const double* f, double* r, int k);

/* y = A x in FP64 for k vectors. */
slab_status slab_apply(slab_handle* h, const double* x, double* y, int k);

/* y = A^T x in FP64 for k vectors (the same stencil with its couplings transposed; equal to
 * slab_apply for the symmetric kinds). */
slab_status slab_apply_transpose(slab_handle* h, const double* x, double* y, int k);

/*
 * Non-zero Dirichlet data (Sec. 1.1 with u = g on the boundary instead of 0).  Eliminating the
 * boundary unknowns from the interior rows gives A u = f + lift(g) with
 *   lift(g)_P = h^-2 sum over the boundary neighbours Q of P of k_PQ g_Q,
 * k_PQ the operator's face coefficients; this writes f_out = f + lift(g), so that
 * slab_solve(h, f_out, u, k) returns the interior values of the solution.
 * g: device, k x (n+1)^d FP64 over all nodes (C order [z][y][x], only boundary entries are
 * read); f: device, k x (n-1)^d interior load, or NULL for zero; f_out: device, same layout as f,
 * may be f itself.  Caller owns all buffers.  SLAB_EINVAL for a null handle, g or f_out, or
 * k < 0; SLAB_EUNSUPPORTED for CONVECTION.  Asynchronous on the handle's stream.
 */
slab_status slab_boundary_lift(slab_handle* h, const double* g, const double* f, double* f_out, int k);

/*
 * Adjoint solve and coefficient gradient (DIFFUSION, CONVECTION).  Given dL/du (device,
 * [k][(n-1)^d]) and the state u, solves A^T lambda = dL/du with the stored factors, refined
 * like slab_solve against the FP64 residual of A^T, and, if dLdkappa != NULL, accumulates into
 * it (device, (n+1)^d, k gradients summed) dL/dkappa_p = -lambda^T (dA/dkappa_p) u (the
 * first-order term of CONVECTION does not depend on kappa).  For the symmetric kinds the solve
 * is slab_solve's; for CONVECTION every phase runs transposed on the same factors: the slab
 * trees with S^-T and the other orientation of their couplings, Algorithm 2 on T^T = U^T L^T
 * (forward with W_j^T, backward with S_j^-T and T_{j+1,j}^T).  Status as slab_solve.
 */
slab_status slab_adjoint(slab_handle* h, const double* dLdu, const double* u, double* lambda,
                         double* dLdkappa, int k);

/* --- phase-level entry points (one step of Algorithm 4 each, no refinement) --- */

/* Reduced load on the interfaces, eqs. f1-f5: ftilde = f_I - A_IJ A_JJ^-1 f_J. */
slab_status slab_reduced_rhs(slab_handle* h, const double* f, double* ftilde, int k);

/* Algorithm 2 with the Stage-2 factors: utilde = T^-1 ftilde. */
slab_status slab_interface_solve(slab_handle* h, const double* ftilde, double* utilde, int k);

/* Eq. usol_even: u_J = A_JJ^-1 (f_J - A_JI utilde) per slab; u_I = utilde.  Writes all of u. */
slab_status slab_interior_solve(slab_handle* h, const double* f, const double* utilde, double* u,
                                int k);

/*
 * Y = T X without forming T, the operation the randomized recovery of T in Sec. 3.3 is built on
 * (T is only ever applied to a sketch matrix there).  With the interface values u_I = X, the slab
 * interiors u_J = -A_JJ^-1 A_JI X come from one interior solve with zero load (eq. usol_even, the
 * stored Stage-1 factors), and T X = A_II X + A_IJ u_J = (A u)_I is read off the stencil rows of the
 * interface nodes.  X, Y: device, k interface vectors ([k][N_I (n-1)^(d-1)], the interface layout
 * above); work: device scratch of 2 k (n-1)^d doubles owned by the caller.  Accuracy: that of the
 * Stage-1 factor (FP32 or FP64).  SLAB_EINVAL for a null handle or pointer, k < 0.  Asynchronous on
 * the handle's stream.
 */
slab_status slab_apply_T(slab_handle* h, const double* X, double* Y, int k, double* work);

/*
 * Copy one (n-1)^(d-1) square block of the reduced matrix T (as assembled,
 * before Stage 2) to out (HOST, row-major, FP64): which = 0 gives T_qq, which
 * = 1 gives T_{q,q+1} and which = 2 gives T_{q+1,q} (q = 0..N_I-2; assembled separately
 * for CONVECTION, the transpose of T_{q,q+1} otherwise).  Synchronises the stream.
 */
slab_status slab_get_T_block(slab_handle* h, int which, int q, double* out);

/*
 * Dense building block of the Stage-2 kernels, exposed for direct use and testing:
 * C = alpha A B^T + beta C on the tensor cores (tcgen05, TMA-fed, FP32 accumulation in
 * tensor memory).  A: M x K, B: N x K, C: M x N, all FP32 row-major on the device with
 * leading dimensions lda, ldb, ldc (elements); trans_c = 1 writes C^T instead (C is then
 * N x M with leading dimension ldc).  split = 1 multiplies with three TF32 products
 * (hi*hi + hi*lo + lo*hi), which keeps FP32 accuracy; split = 0 uses one TF32 product;
 * split = 2 scales every row of A and B by a power of two into (-1, 1), splits it into FP16
 * hi + lo and multiplies with three FP16 products (FP32 accuracy at twice the TF32 rate; needs
 * K % 64 == 0; scratch of about 4 (M + N) K bytes comes from the stream-ordered allocator,
 * SLAB_ENOMEM if it cannot).  The factorization uses split 2 for its Schur and trailing
 * products.  Requires K % 32 == 0, lda, ldb multiples of 4 and 16-byte aligned A and B
 * (SLAB_EINVAL otherwise).  dev_err: device word, bit 2 is set if a bounded device wait gave
 * up.  Asynchronous on stream.  Used in the paper's sense by Algorithm 1 (Sec. 4) products.
 */
slab_status slab_tc_gemm(int M, int N, int K, float alpha, const float* A, int64_t lda, const float* B,
                         int64_t ldb, float beta, float* C, int64_t ldc, int trans_c, int split,
                         unsigned* dev_err, void* stream);

/*
 * Measurement support.  Kernel classes of the library, for per-class timing:
 *   0 coefficient setup (A0), 1 slab tree factor (A1/A2), 2 T assembly (A3),
 *   3 panel factor of Stage 2 (A4), 4 Stage-2 trailing update (A4, tensor cores in FP32),
 *   5 Stage-2 Schur update S_{j+1} = T - Y^T Y (A4), 6 interface sweep products (A6),
 *   7 tree up pass + reduced load (A5), 8 tree down pass (A7), 9 FP64 stencil residual (A8),
 *   10 other (transposes, reductions, scatter/gather, gradient),
 *   11-13 the panel, trailing-update and Schur-update products of the 3-D slab elimination
 *   (Stage 1 in 3-D runs the same dense kernels as Stage 2; these classes keep them apart).
 * slab_profile(h, 1) starts recording a CUDA event pair around every launch on the handle's
 * stream; slab_profile_read fills ms[c] (summed device time) and launches[c] (HOST arrays
 * of n <= SLAB_KERNEL_CLASSES entries) for the launches since the previous read, then
 * clears the record; it synchronises the stream.  Launch counts are kept even when timing
 * is off.  Timing adds an event record per launch; keep it off for timed runs.
 */
/*
 * FP64-accurate product on the tensor cores: C (FP64, M x N, row-major, ldc) += alpha A B^T with
 * A (M x K, lda) and B (N x K, ldb) FP64 row-major, K <= 64 and K % 32 == 0 (SLAB_EINVAL
 * otherwise).  Every row of A and of B is scaled by a power of two and cut into 8 exact 7-bit
 * integer slices; the slice products run on the TF32 tensor cores without rounding and are
 * recombined in FP64 (error ~2^-48 |A| |B| per element, like an FP64 product).  work: device
 * scratch of slab_fp64_tc_gemm_work_bytes(M, N, K) bytes; dev_err as in slab_tc_gemm.
 * Asynchronous on `stream`.  Used for the interface elimination with interface_prec
 * SLAB_PREC_FP64_TC; the paper has no counterpart (its arithmetic is native FP64).
 */
slab_status slab_fp64_tc_gemm(int M, int N, int K, double alpha, const double* A, int64_t lda,
                              const double* B, int64_t ldb, double* C, int64_t ldc, void* work,
                              unsigned* dev_err, void* stream);
size_t slab_fp64_tc_gemm_work_bytes(int M, int N, int K);

/*
 * Batches of independent problems as CUDA graphs (the batched adjoint workload).  count 2-D
 * DIFFUSION problems, problem i on the n[i] x n[i] grid with interface spacing b[i] (uneven sizes
 * allowed), each with one load f_i and one target t_i and the least-squares objective
 *   L_i = ||u_i - t_i||^2,  u_i = A_i^-1 f_i.
 * One run computes, for every problem: the factor (Algorithm 3), u_i with one solve pass and
 * `steps` refinement passes (Algorithm 4), L_i, lambda_i = A_i^-T dL_i/du_i with the same factors
 * (A_i is symmetric) and steps refinement passes, and grad_i = dL_i/dkappa_i at the (n[i]+1)^2 nodes.
 * slab_batch_create allocates every device buffer once (one region: the inputs and outputs of all
 * problems plus the factor memory of the largest wave) and records all launches of each wave of
 * `wave` problems (0: all) into one CUDA graph, the wave's problems spread over `branches` parallel
 * graph branches (0: 16); waves run one after another and reuse the factor memory.  A run is then
 * one graph launch per wave with no allocation, no host synchronisation and no host decision.
 * opts: as for slab_factor (factor_prec, interface_prec, stage2, rtol; krylov must be 0; stream
 * and profile are ignored); steps in 0..100.  SLAB_EINVAL for bad sizes, SLAB_ENOMEM when the region
 * does not fit, SLAB_EUNSUPPORTED for krylov > 0.  Synchronises before returning.
 */
typedef struct slab_batch slab_batch;
slab_status slab_batch_create(int count, const int* n, const int* b, const slab_opts* opts, int steps, int wave,
                              int branches, slab_batch** out);
/* Device buffers of problem i, owned by the batch (valid until slab_batch_destroy): inputs kappa
 * ((n+1)^2 nodes), f and target ((n-1)^2 interior nodes); outputs u, lambda ((n-1)^2) and grad
 * ((n+1)^2).  Write the inputs before slab_batch_run (any stream ordered before it); any pointer
 * argument may be NULL. */
slab_status slab_batch_buffers(slab_batch* B, int i, double** kappa, double** f, double** target, double** u,
                               double** lambda, double** grad);
/* Enqueue one run of every wave's graph on `stream` (a cudaStream_t, NULL = legacy default).
 * Runs of one batch must not overlap (they share the factor memory). */
slab_status slab_batch_run(slab_batch* B, void* stream);
/* Wait for the last run and read per problem (HOST arrays of count entries, each may be NULL) the
 * loss L_i and the relative residuals ||f - A u|| / ||f|| and ||g - A lambda|| / ||g|| it reached.
 * Returns SLAB_ESINGULAR / SLAB_ETIMEOUT if a factor reported one, else SLAB_ENOCONV if a residual
 * is above opts->rtol (raise `steps`), else SLAB_OK. */
slab_status slab_batch_results(slab_batch* B, double* loss, double* relres_u, double* relres_lambda);
/* Bytes of the batch's device region. */
int64_t slab_batch_device_bytes(const slab_batch* B);
void slab_batch_destroy(slab_batch* B);

/*
 * Online tuning of the factor's tensor-core products (process-wide, all devices).  The FP32-accurate
 * factor products have three implementations: three FP16 products of row-scaled hi/lo splits on
 * 128 x 128 or 128 x 256 tiles (a pre-pass makes the splits), or 3xTF32 with the split inside the
 * kernel (no pre-pass, half the MMA rate).  mode 1: the first calls of each shape class (log2
 * buckets of M, N, K and the batch) run every candidate twice, timed by CUDA events on the
 * launching stream, and the class then keeps the fastest per flop; mode 0: a fixed size heuristic
 * (the default; also set by the environment variable SLAB_AUTOTUNE=1 / 0 before the first call);
 * mode 2: forget every decision (mode unchanged).  Returns the previous mode.  Results of the
 * candidates agree to FP32 rounding, so tuning changes only the last bits and the time.  Launches
 * on a stream under CUDA graph capture are never timed: they use the decided candidate, or the
 * heuristic one while the class is undecided.
 */
int slab_autotune(int mode);
/* Shape classes seen, decided, decided for 3xTF32, decided for the other tile width (each may be NULL). */
slab_status slab_autotune_stats(int* classes, int* decided, int* tf32x3, int* alt_width);

#define SLAB_KERNEL_CLASSES 14
slab_status slab_profile(slab_handle* h, int enable);
slab_status slab_profile_read(slab_handle* h, double* ms, int64_t* launches, int n);

/* Sizes: unknowns (n-1)^d, interface size (n-1)^(d-1), number of interfaces N_I. */
slab_status slab_sizes(const slab_handle* h, int64_t* unknowns, int64_t* iface_size, int* n_ifaces);

/* Elimination order Stage 2 used for this handle: SLAB_STAGE2_SWEEP or SLAB_STAGE2_ODDEVEN (what
 * SLAB_STAGE2_AUTO resolved to); 0 for a NULL handle. */
int slab_stage2_order(const slab_handle* h);

/* Bytes of device memory the handle holds. */
int64_t slab_device_bytes(const slab_handle* h);

/* Latched first error of the handle (SLAB_OK if none). */
slab_status slab_last_error(const slab_handle* h);

void slab_destroy(slab_handle* h);
const char* slab_strerror(slab_status s);

/*
 * Residual and norms for callers that cannot allocate device memory.  The
 * paper has no counterpart: this is a library convenience.  Some callers may
 * not call cudaMalloc at all -- code running inside a stream capture that must
 * stay free of allocation nodes, a process whose device memory pool belongs to
 * another framework, a real-time loop that bans allocator calls.  This entry
 * point allocates nothing and needs no handle: for the 2-D grid n (h = 1/n)
 * and the operator given by kind/kappa/c/omega (as in slab_coeffs; POISSON, DIFFUSION or HELMHOLTZ,
 * SLAB_EINVAL for CONVECTION), it writes
 * r = f - A u (device, [k][(n-1)^2]) and the squared 2-norms nrm_r[q] =
 * ||r_q||^2, nrm_f[q] = ||f_q||^2 (device, k entries each), on the given
 * stream (a cudaStream_t, NULL = legacy default).  All buffers are the
 * caller's.  The norm reduction uses a fixed 4 MiB scratch array built into
 * the library (held by every GPU that loads it until exit); requests with
 * k * ceil((n-1)/256) * ceil((n-1)/32) * 2 > 2^19 or k > 8192 are rejected
 * with SLAB_EINVAL.  All calls share that scratch: calls that overlap on the
 * GPU race and must be serialised by the caller.  The first call on a device
 * looks up the scratch address for that device; make it before any stream
 * capture starts.
 */
slab_status slab_residual_norms_noalloc(int n, int kind, const double* kappa, const double* c,
                                        double omega, const double* u, const double* f, double* r,
                                        int k, double* nrm_r, double* nrm_f, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SLAB_H */
