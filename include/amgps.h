/*
 * amgps.h -- C ABI of libamgps: polynomial-accelerated l1-Jacobi smoothers
 * inside a symmetric AMG V-cycle preconditioning CG, on one GB300 (sm_103a).
 *
 * The operations follow arXiv 2407.09848 ("Optimal Polynomial Smoothers for
 * Parallel AMG"):
 *   - the SPD system A x = b                                  (Sec. 1, Eq. sys1)
 *   - Galerkin hierarchy A_{l+1} = P_l^T A_l P_l              (Sec. 2)
 *   - symmetric multiplicative V-cycle                        (Sec. 2, Eq. amg)
 *   - l1-Jacobi M_i = a_ii + sum_{j != i} |a_ij|              (Sec. 2, Eq. l1smooth)
 *   - 4th-kind Chebyshev smoother                             (Sec. 2.1, Eq. polsmoother)
 *   - optimised 4th-kind weights                              (Sec. 2.1, Eq. polsmootheropt)
 *   - 1st-kind Chebyshev acceleration on [a_k*, 1]            (Sec. 2.2, Algorithm 1;
 *                                                              a_k* from Eq. optimalparameter)
 *   - preconditioned CG as the outer solver                   (Sec. 4)
 *
 * Conventions (every entry point):
 *   - No exception crosses this ABI.  Each call returns an amgps_status; the
 *     text of the last failure is available from amgps_last_error(ctx).
 *   - Host arrays passed in are borrowed for the duration of the call and
 *     copied; the library owns every device copy and workspace it makes.
 *   - Vector arguments named *_dev are device pointers owned by the caller,
 *     FP64, length n_l of the level they refer to, in the caller's row order
 *     (the order of the CSR rows given to amgps_hierarchy_load).
 *   - Work is ordered after prior work on the caller's stream given to
 *     amgps_create and the caller's stream is ordered after it on return, so
 *     the calls are stream-asynchronous unless documented otherwise.
 *   - A context is not thread-safe; use one context per host thread.
 *   - Device faults are never used for error reporting: invalid input is
 *     rejected on the host before any launch.
 */
#ifndef AMGPS_H
#define AMGPS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  AMGPS_OK = 0,
  AMGPS_E_ARG = 1,      /* bad argument: null pointer, malformed CSR, size mismatch,
                           bad kind/degree */
  AMGPS_E_NOT_SPD = 2,  /* non-positive diagonal, Cholesky pivot <= 0, or p^T A p <= 0 in PCG */
  AMGPS_E_NOCONV = 3,   /* PCG reached maxit without meeting rtol (x holds the last iterate) */
  AMGPS_E_NAN = 4,      /* a NaN/Inf appeared in a PCG scalar */
  AMGPS_E_CUDA = 5,     /* a CUDA runtime call failed (message has cudaGetErrorString) */
  AMGPS_E_TIMEOUT = 6,  /* a bounded wait inside a pipelined kernel gave up */
  AMGPS_E_STATE = 7,    /* call out of order (e.g. smooth before hierarchy_load) */
  AMGPS_E_NOMEM = 8     /* device or pinned host allocation failed */
} amgps_status;

/* Smoother kinds (the rows of Table 1, Sec. 4, plus two configurations). */
typedef enum {
  AMGPS_L1JACOBI = 0,   /* k sweeps x += M^{-1}(b - A x)                                */
  AMGPS_CHEB4 = 1,      /* Eq. polsmoother, rho(M^{-1}A) := 1 (or the level's rho)        */
  AMGPS_CHEB4_OPT = 2,  /* Eq. polsmootheropt with the tabulated optimal beta_{j,k}       */
  AMGPS_CHEB1 = 3,      /* Algorithm 1 on [a_k*,1] with rho = the level's rho (e.g. 1.1 x
                           a power-iteration estimate, amgps_estimate_lambda)             */
  AMGPS_CHEB1_OPT = 4,  /* Algorithm 1 on [a_k*,1] with rho(M^{-1}A) := 1 (Sec. 3)        */
  AMGPS_WEIGHTS = 5     /* Eq. polsmootheropt with caller-supplied weights (learned)      */
} amgps_kind;

/* Storage of matrix values on the smoother and transfer path.  F64: all FP64.
 * F32 / BF16: values rounded to nearest-even at load, V-cycle vectors and
 * accumulation in FP32; the outer PCG (its SpMV, vectors and dot products) and
 * the coarsest dense solve stay FP64. */
typedef enum { AMGPS_F64 = 0, AMGPS_F32 = 1, AMGPS_BF16 = 2 } amgps_prec;

/* Host CSR, borrowed.  rowptr[n_rows+1], col[nnz], val[nnz]; 0-based; columns
 * need not be sorted; duplicates are not allowed. */
typedef struct {
  int64_t n_rows, n_cols, nnz;
  const int32_t* rowptr;
  const int32_t* col;
  const double* val;
} amgps_csr;

typedef struct amgps_ctx amgps_ctx;

/* Library ABI version (monotone integer). */
int amgps_version(void);

/* Create a context on CUDA device `device`.  `user_stream` (cudaStream_t,
 * may be NULL for the legacy default stream) is the stream the caller's work
 * lives on; the library runs on a stream of its own, ordered against it with
 * events.  *out is NULL on failure. */
amgps_status amgps_create(amgps_ctx** out, int device, void* user_stream);

/* Release every device and host resource of the context.  NULL is allowed. */
amgps_status amgps_destroy(amgps_ctx* ctx);

/* Message of the last failing call on this context ("" if none).  Valid until
 * the next call on the context.  With ctx == NULL: the last creation error. */
const char* amgps_last_error(const amgps_ctx* ctx);

/* Load the level hierarchy (Sec. 2): A[0..n_levels-1] square SPD CSR with
 * n_rows(A[l+1]) == n_cols(P[l]); P[0..n_levels-2] the prolongators (any
 * sparsity; A[l+1] should be P[l]^T A[l] P[l]).  A P[l] whose every row holds
 * one entry equal to 1 (unsmoothed aggregation) restricts by summing each
 * aggregate's children and prolongs by a gather; any other P (e.g. smoothed
 * aggregation, amgps_sa_level) is stored with its transpose in explicit
 * SELL-32 form and both transfers are sparse products.
 * The coarsest level (n <= 1024) is solved by a dense FP64 Cholesky
 * factorisation computed here on the device (AMGPS_E_NOT_SPD if a pivot is
 * not positive).  Replaces any earlier hierarchy; every level's smoother is
 * reset to CHEB4_OPT of degree 4.  Synchronous. */
amgps_status amgps_hierarchy_load(amgps_ctx* ctx, int n_levels, const amgps_csr* A,
                                  const amgps_csr* P, amgps_prec prec);

/* Host CSR allocated by the library (results of amgps_galerkin and
 * amgps_sa_level).  Rows are sorted by column.  Release with
 * amgps_csr_buf_free, which frees the three arrays and zeroes the struct
 * (NULL allowed). */
typedef struct {
  int64_t n_rows, n_cols, nnz;
  int32_t* rowptr; /* n_rows + 1 */
  int32_t* col;    /* nnz */
  double* val;     /* nnz */
} amgps_csr_buf;
void amgps_csr_buf_free(amgps_csr_buf* m);

/* Galerkin coarse operator A_c = P^T A P (Sec. 2), computed on the context's
 * device by two sparse products (A P, then P^T (A P)) with P^T formed on the
 * device.  A: square CSR; P: n_rows(A) x n_c CSR whose rows have strictly
 * ascending columns.  Every entry of the product is summed in a fixed order,
 * so repeated calls give identical bits.  AMGPS_E_ARG for malformed input or
 * when a row of an intermediate product (or of P^T) exceeds 6144 distinct
 * columns;
 * AMGPS_E_NOMEM when device scratch cannot be allocated.  Synchronous; needs
 * no loaded hierarchy.  *Ac receives library-allocated host CSR. */
amgps_status amgps_galerkin(amgps_ctx* ctx, const amgps_csr* A, const amgps_csr* P,
                            amgps_csr_buf* Ac);

/* One level of smoothed aggregation (Sec. 4): from the aggregates agg
 * (n_rows(A) entries in [0, n_coarse), every coarse index used) the
 * tentative prolongator P_hat (P_hat[i, agg[i]] = 1) is smoothed by one damped
 * Jacobi step,
 *     P = (I - omega D^{-1} A) P_hat,  D = diag(A),  omega = 4 / (3 lambda),
 * with lambda = max_i sum_j |a_ij| / a_ii, the row-sum bound on the spectrum
 * of D^{-1} A, and A_c = P^T A P as in amgps_galerkin.  All of it runs on the
 * device.  Returns omega, P (n x n_coarse) and A_c as library-allocated host
 * CSR.  AMGPS_E_NOT_SPD for a missing or non-positive diagonal entry;
 * otherwise errors as amgps_galerkin.  Synchronous. */
amgps_status amgps_sa_level(amgps_ctx* ctx, const amgps_csr* A, const int32_t* agg,
                            int64_t n_coarse, double* omega, amgps_csr_buf* P,
                            amgps_csr_buf* Ac);

/* Rows, nonzeros and stored matrix entries (after padding) of a level. */
amgps_status amgps_level_info(amgps_ctx* ctx, int level, int64_t* n, int64_t* nnz,
                              int64_t* stored);

/* Smoother used by amgps_vcycle / amgps_pcg on `level` (-1: every non-coarsest
 * level).  degree in 1..16.  `weights` (host, `degree` doubles) is read only for
 * AMGPS_WEIGHTS and copied.  `rho` scales the spectral interval: the smoother
 * uses rho in place of rho(M^{-1}A) (CHEB1, CHEB4, WEIGHTS, CHEB4_OPT);
 * rho <= 0 means 1.  Synchronous host bookkeeping only. */
amgps_status amgps_set_smoother(amgps_ctx* ctx, int level, amgps_kind kind, int degree,
                                const double* weights, double rho);

/* Power-iteration estimate of the largest eigenvalue of M^{-1}A_l on the
 * device: v_0 = v0/||v0||, w = M^{-1}A v_{i-1}, lambda_i = ||w||,
 * v_i = w/lambda_i, i = 1..iters; returns lambda_iters.  v0_dev: n_l FP64.
 * Synchronous. */
amgps_status amgps_estimate_lambda(amgps_ctx* ctx, int level, const double* v0_dev,
                                   int iters, double* lambda_out);

/* One smoother application on `level` (Sec. 2.1-2.2): x <- S(b, x).  `kind`
 * and `degree` select the recurrence; CHEB4_OPT takes the tabulated weights,
 * WEIGHTS the weights and rho stored by amgps_set_smoother for this level,
 * CHEB1 the level's rho.  x_is_zero != 0 means the start vector is zero and
 * x_dev is write-only.  b_dev, x_dev: n_l FP64 device vectors, must not alias. */
amgps_status amgps_smooth(amgps_ctx* ctx, int level, amgps_kind kind, int degree,
                          const double* b_dev, double* x_dev, int x_is_zero);

/* Reverse mode of one smoother application x = S(b, x0) on `level` (FP64
 * hierarchies).  No passage of the paper defines it; it serves the learned
 * weights.  Given gx = dL/dx returns gb = dL/db and gx0 = dL/dx0 (device,
 * nullable) and, for the 4th-kind family (CHEB4, CHEB4_OPT, WEIGHTS),
 * gweights[j] = dL/dbeta_{j+1} (host, `degree` doubles, nullable; zeros for
 * other kinds).  x0_dev NULL means a zero start.  The smoother operator
 * Q = q(M^{-1}A) M^{-1} is symmetric, so gb is one more smoother application
 * (to gx, from zero) and gx0 = gx - A gb; the weight gradients are
 * <gx, z_j> with the z recurrence recomputed from (b, x0), so no recurrence
 * vector is stored.  The first backward call allocates the reverse-mode
 * buffers of every level.  Synchronous when gweights is requested. */
amgps_status amgps_smooth_backward(amgps_ctx* ctx, int level, amgps_kind kind, int degree,
                                   const double* b_dev, const double* x0_dev,
                                   const double* gx_dev, double* gb_dev, double* gx0_dev,
                                   double* gweights);

/* Reverse mode of one V-cycle z = B(beta) r with the smoothers set by
 * amgps_set_smoother (FP64 hierarchies): recomputes the forward V-cycle from
 * r (recording each level's post-smoother input), then returns gr = dL/dr
 * (device, nullable) and, in gweights (host, nullable), dL/dbeta for every
 * non-coarsest level l at gweights[16 l + j], j < that level's degree (zeros
 * for kinds without weights).  Synchronous when gweights is requested. */
amgps_status amgps_vcycle_backward(amgps_ctx* ctx, const double* r_dev, const double* gz_dev,
                                   double* gr_dev, double* gweights);

/* Mean A-norm error reduction of one V-cycle over m error vectors and its
 * gradient in every level's weights (the training loss of the learned
 * weights; no passage of the paper defines it):
 *   loss = (1/m) sum_i ||(I - B A) e_i||_A^2 / ||e_i||_A^2,
 * E0_dev holds e_0..e_{m-1} (m x n_0 doubles, vector i at E0_dev + i n_0),
 * m <= 4096, FP64 hierarchies.  *loss (host) and gweights (host, nullable,
 * 16 per non-coarsest level as in amgps_vcycle_backward).  Every product,
 * V-cycle, reverse pass and dot runs in the library's kernels.  Synchronous. */
amgps_status amgps_vcycle_loss_grad(amgps_ctx* ctx, const double* E0_dev, int m, double* loss,
                                    double* gweights);

/* Apply the V-cycle error propagation E = I - B A `cycles` times, in place,
 * to each of the m vectors of E_dev (m x n_0 doubles, vector i at
 * E_dev + i n_0), with the current smoothers.  Repeated application
 * concentrates the vectors on the slowest modes of E, so the loss of
 * amgps_vcycle_loss_grad on them estimates the squared convergence factor
 * rho(E)^2 (E is self-adjoint in the A inner product) and its gradient.  No
 * passage of the paper defines it.  Asynchronous. */
amgps_status amgps_error_cycles(amgps_ctx* ctx, double* E_dev, int m, int cycles);

/* The weight-predicting MLP of the learned smoother (not in the paper):
 * 8 level features -> 64 -> 64 -> 4, ReLU, beta = beta_ref exp(2 tanh(o / 2)).
 * Stateless FP32 kernels on caller-owned device buffers, enqueued on `stream`
 * (cudaStream_t, may be NULL); errors through amgps_last_error(NULL).
 * params: 4996 floats [W1 (64x8 row-major), b1 (64), W2 (64x64), b2, W3 (4x64),
 * b3 (4)]; feats: batch x 8; beta_ref: 4; beta: batch x 4; acts: batch x 132
 * (saved by forward for backward); work: batch x 132 scratch; grads: 4996
 * (overwritten with dL/dparams for the given gbeta = dL/dbeta, batch x 4);
 * Adam: step counts from 1, m and v are 4996-float moment buffers. */
amgps_status amgps_mlp_forward(const float* params_dev, const float* feats_dev, int batch,
                               const float* beta_ref_dev, float* beta_dev, float* acts_dev,
                               void* stream);
amgps_status amgps_mlp_backward(const float* params_dev, const float* feats_dev,
                                const float* acts_dev, const float* beta_dev, int batch,
                                const float* gbeta_dev, float* work_dev, float* grads_dev,
                                void* stream);
amgps_status amgps_mlp_adam(float* params_dev, const float* grads_dev, float* m_dev, float* v_dev,
                            int step, float lr, float beta1, float beta2, float eps, void* stream);

/* amgps_smooth without any device allocation, for callers that may not
 * allocate device memory at the point of the call (for example code running
 * under an allocator that owns all device memory, or a phase of a real-time
 * loop where allocation is forbidden).  No counterpart in the paper: same
 * kernels and result as amgps_smooth, but the work vectors live in one static
 * device array of 3 MiB, so levels with more than 65536 rows are rejected with
 * AMGPS_E_ARG.  amgps_create claims that array on its device (it looks up the
 * array's device address with cudaGetSymbolAddress, which under lazy module
 * loading also brings the array onto the device) and keeps the address in the
 * context; the array stays on that device until the process exits.  Kernels
 * are loaded by the CUDA runtime on their first launch: before the phase where
 * allocation is forbidden, run the same smoother once through amgps_smooth (or
 * load modules eagerly, CUDA_MODULE_LOADING=EAGER).  Every call shares the
 * array: calls that overlap on the GPU (other streams, other contexts, other
 * host threads) race and corrupt each other's results.  Nothing needs
 * clearing between calls: each call writes every scratch entry it reads before
 * reading it.  Arguments as for amgps_smooth. */
amgps_status amgps_smooth_noalloc(amgps_ctx* ctx, int level, amgps_kind kind, int degree,
                                  const double* b_dev, double* x_dev, int x_is_zero);

/* One V-cycle z = B r (Eq. amg) from level 0, with the smoothers set by
 * amgps_set_smoother.  r_dev, z_dev: n_0 FP64 device vectors, must not alias. */
amgps_status amgps_vcycle(amgps_ctx* ctx, const double* r_dev, double* z_dev);

/* Preconditioned CG on A_0 x = b with one V-cycle as preconditioner, x_0 = 0,
 * stopping when ||r_k||_2 <= rtol ||b||_2 (recurrence residual) or after maxit
 * iterations.  *iters = products with A_0 performed, *relres = final
 * ||r_k||/||b||.  b_dev, x_dev: n_0 FP64 device vectors.  Synchronous (one
 * host read of ||r||^2 per iteration).  Returns AMGPS_E_NOCONV at maxit. */
amgps_status amgps_pcg(amgps_ctx* ctx, const double* b_dev, double* x_dev, double rtol,
                       int maxit, int* iters, double* relres);

/* PCG on A_0 x = b preconditioned by ONE smoother application on level 0
 * from zero, z = S(r, 0) = q(M^{-1}A) M^{-1} r (SPD because |p| < 1 on (0,1]),
 * without coarse levels: the smoother-only experiment of the remark in
 * Sec. 2.3 (PCG iteration counts for the 1st- and 4th-kind polynomials on
 * A = Q D Q^T).  Needs a hierarchy of two or more levels (level 0 must own a
 * smoother).  Otherwise as amgps_pcg (honours AMGPS_OPT_FLEXIBLE). */
amgps_status amgps_pcg_smoother(amgps_ctx* ctx, amgps_kind kind, int degree, const double* b_dev,
                                double* x_dev, double rtol, int maxit, int* iters,
                                double* relres);

/* amgps_pcg with host vectors: copies b (pinned staging) to the device,
 * solves, copies x back.  b_host, x_host: n_0 doubles. Synchronous. */
amgps_status amgps_pcg_host(amgps_ctx* ctx, const double* b_host, double* x_host,
                            double rtol, int maxit, int* iters, double* relres);

/* Wait for all work of the context.  */
amgps_status amgps_synchronize(amgps_ctx* ctx);

/* Context options.  AMGPS_OPT_TMA selects the kernel of the fused smoother
 * step: 0 the direct-load kernel everywhere; 1 (default) the TMA-fed
 * pipelined kernel on levels whose layout allows it and that hold at least
 * 4 tiles per SM, the direct one elsewhere; 2 the
 * TMA-fed kernel wherever the layout allows it.  Results are identical
 * across the three.  Other values: AMGPS_E_ARG.
 * AMGPS_OPT_FLEXIBLE (default 0) selects the outer CG form of amgps_pcg and
 * amgps_pcg_smoother, all three equal in exact arithmetic for a fixed SPD
 * preconditioner:
 *   0  standard PCG, beta = r_{k+1}.z_{k+1} / (r_k.z_k);
 *   1  flexible, Polak-Ribiere beta = r_{k+1}.(z_{k+1} - z_k) / (r_k.z_k),
 *      robust when the preconditioner is not exactly a fixed symmetric
 *      operator (FP32/BF16 smoothers);
 *   2  flexible CG with one global reduction per iteration, the outer solver
 *      of Sec. 4: w = A z, then rho = z.r, gamma = z.q, delta = z.w in one
 *      reduction; beta = gamma / eta_old, p = z - beta p, q = w - beta q
 *      (q = A p kept by recurrence), eta = delta - beta gamma, alpha = rho/eta.
 *      Other values: AMGPS_E_ARG.
 * AMGPS_OPT_COARSE_SWEEPS (default 0): the coarsest level of the V-cycle is
 * solved with the dense FP64 inverse (0), or by m = 1..1000 l1-Jacobi sweeps
 * from zero, x <- x + M^{-1}(b - A_c x), the coarse solver of the paper's
 * experiments (Sec. 4 uses 30); the V-cycle stays symmetric either way.
 * AMGPS_OPT_COARSE_KERNEL (default 0): 1 runs the levels below the last one
 * that runs the TMA-fed step, down to the coarsest, as one persistent kernel
 * (one co-resident grid with a bounded grid-wide barrier between dependent
 * kernels' work) when they use aggregation transfers and one warp per slice;
 * 0 launches their kernels one by one (inside the CUDA graph of the coarse
 * levels).  Results are identical either way.  A barrier wait that gives up
 * is reported by the next amgps_pcg as AMGPS_E_TIMEOUT.
 * AMGPS_OPT_ALLOC_LIMIT (default 0 = none): the most bytes of device memory
 * the context may allocate for a hierarchy and its work vectors (the
 * buffers of amgps_hierarchy_load and of the reverse-mode calls).  A request
 * that would pass it fails with AMGPS_E_NOMEM before reaching the CUDA
 * allocator, so a caller can reject a problem that would not fit its memory
 * share.  Any failed amgps_hierarchy_load leaves no hierarchy loaded and
 * keeps none of its buffers.
 * AMGPS_OPT_STEP_FORM (default 1): how the smoothers of degree >= 2 (every
 * kind) run on FP64 levels of at least 131,072 rows that the step kernel
 * evaluates one warp per 32-row slice (every level whose rows average fewer
 * than 24 stored entries, and wider ones with enough slices).  0: the
 * recurrences of Eq. polsmoother / polsmootheropt, Algorithm 1 and
 * Eq. l1smooth step by step.  1: the same polynomial
 * evaluated backwards (Clenshaw's scheme on its three-term recurrence) with
 * each step's operator tau_j I - sigma_j M^{-1} A stored in A's layout --
 * degree - 1 extra arrays of A's stored entries per such level, built by
 * amgps_hierarchy_load, amgps_set_smoother and this option, and counted
 * against AMGPS_OPT_ALLOC_LIMIT; a level whose arrays do not fit keeps form
 * 0.  The two forms agree to rounding (not bit for bit); amgps_smooth uses
 * form 1 on a level only for the kind, degree, weights and rho set for it by
 * amgps_set_smoother.  Other values: AMGPS_E_ARG. */
enum { AMGPS_OPT_TMA = 1, AMGPS_OPT_FLEXIBLE = 2, AMGPS_OPT_COARSE_SWEEPS = 3,
       AMGPS_OPT_COARSE_KERNEL = 4, AMGPS_OPT_ALLOC_LIMIT = 5, AMGPS_OPT_STEP_FORM = 6 };
amgps_status amgps_set_option(amgps_ctx* ctx, int option, int64_t value);

/* Host-only planning query (no device needed): how the TMA-fed step would
 * cover matrix A at precision `prec` -- tiles it takes (480 rows for FP64
 * vectors, 1024 for FP32 ones), 32-row slices left to the direct kernel, bytes
 * per shared-memory stage and stages per CTA.  Every bulk copy of the plan is
 * checked on the host for bounds and 16-byte alignment; a violation returns
 * AMGPS_E_ARG. */
amgps_status amgps_tma_plan_stats(const amgps_csr* A, amgps_prec prec, int64_t* tiles,
                                  int64_t* generic_slices, int* stage_bytes, int* nstages);

/* Host-only (no device needed): the BF16 bit patterns that
 * amgps_hierarchy_load stores for AMGPS_BF16 levels -- each finite FP64 value
 * rounded directly to the nearest BF16 value, ties to even (no intermediate
 * FP32 rounding).  AMGPS_E_ARG for a non-finite value. */
amgps_status amgps_round_bf16(const double* x, int64_t n, uint16_t* out);

/* Host-only (no device needed): the step scalars the kernels use for one
 * application of `kind` at `degree` (weights and rho as in
 * amgps_set_smoother), arrays of degree+1 doubles indexed by step j.
 * 4th kind (CHEB4, CHEB4_OPT, WEIGHTS): step j computes
 * z_j = c1[j] z_{j-1} + c2[j] M^{-1} r_{j-1}, x += beta[j] z_j (Sec. 2.1).
 * 1st kind (CHEB1, CHEB1_OPT; Algorithm 1): d_0 = c2[0] r_0 and, for j >= 1,
 * d_j = c1[j] d_{j-1} + c2[j] r_j, with residuals scaled by *rhoinv.
 * l1-Jacobi uses none of them.  AMGPS_E_ARG for a bad kind, degree or weight. */
amgps_status amgps_step_coefs(amgps_kind kind, int degree, const double* weights, double rho,
                              double* c1, double* c2, double* beta, double* rhoinv);

/* Host-only inspection (no device needed): the TMA plan behind
 * amgps_tma_plan_stats.  info[32] receives, in order: rows per tile, stencil
 * width w, window groups G, d0 (stage-window index of the tile's own rows),
 * value bytes, vector bytes, window bytes, stage bytes, stages, then
 * g_start[4], g_elems[4], g_smem[4] (window g copies u[r0 + g_start .. +
 * g_elems) to stage-window index g_smem) and d[8] (entry k of tile row i
 * reads stage-window index d[k] + i); unused slots are 0.  Call once with null
 * tiles/gen for *ntiles and *ngen, then with tiles[2 * ntiles] (first row,
 * value index of each tile) and gen[ngen] (slices left to the direct kernel).
 * AMGPS_E_ARG for a malformed A. */
amgps_status amgps_tma_plan(const amgps_csr* A, amgps_prec prec, int32_t* info, int64_t* ntiles,
                            int64_t* tiles, int64_t* ngen, int32_t* gen);

/* Host-only inspection (no device needed): the SELL-32 layout that
 * amgps_hierarchy_load uploads for the square matrix A.  Slice s holds rows
 * 32s .. 32s+31; entry k of its lane l (row 32s+l) sits at index
 * vbase[s] + 32k + l of val (and of col), k < width[s].  A uniform slice
 * (cref[s] >= 0) stores no columns: its entry k is column row + off[cref[s]+k],
 * clamped to [0, n-1], and an entry absent from a row holds 0.  An explicit
 * slice (cref[s] < 0) stores the columns in col (row-sorted; padding holds 0
 * and an in-range column).  Call once with null arrays for the sizes
 * (*nslices, *stored, *noff), then with arrays of those lengths (col entries of
 * uniform slices are written as -1).  AMGPS_E_ARG for a malformed A. */
amgps_status amgps_sell_layout(const amgps_csr* A, int64_t* nslices, int64_t* stored,
                               int64_t* noff, int64_t* vbase, int32_t* width, int32_t* cref,
                               double* val, int32_t* col, int32_t* off);

/* Host-only query: the steps of one smoother application in the
 * stored-operator form (AMGPS_OPT_STEP_FORM 1) for any kind (AMGPS_WEIGHTS:
 * weights as in amgps_set_smoother) and degree k in 2..16.
 * With B = M^{-1} A and s0 = M^{-1} (b - A x0), step q = 0 .. k-2 forms
 *   v_q = h[q] s0 + g[q] v_{q-2} + (tau[q] I - sigma[q] B) w_q,
 *   w_0 = s0, w_q = v_{q-1} (v_{-1} = v_{-2} = 0),
 * and the application returns x = x0 + v_{k-2}.  Each array receives k - 1
 * entries (host).  Other kinds or degrees: AMGPS_E_ARG. */
amgps_status amgps_op_coefs(amgps_kind kind, int degree, const double* weights, double rho,
                            double* tau, double* sigma, double* h, double* g);

/* The library's tabulated optimal 4th-kind weights beta_{1..degree} for
 * Eq. polsmootheropt (degree 1..16), written to beta_out (host). */
amgps_status amgps_opt4_weights(int degree, double* beta_out);

/* The library's tabulated a_k* of Eq. optimalparameter (degree 1..16). */
amgps_status amgps_cheb1_astar(int degree, double* a_out);

/* Kernel timing with CUDA events on the library stream.  When enabled, every
 * launch of the listed kernel classes is bracketed by an event pair; pairs are
 * harvested at synchronisation points.  Classes: 0 = fused smoother step on
 * level 0, 1 = residual+restriction on level 0, 2 = PCG SpMV+dot; for these,
 * *launches, *total_ms (sum of event-timed durations) and *bytes (algorithmic
 * bytes of the launches: matrix nonzeros and stored indices once, each vector
 * stream once) are returned.  Class 3 counts every kernel of this library
 * executed since the last reset (whether or not timing is enabled; a graph
 * replay counts its kernel nodes); its *total_ms and *bytes are 0.  Class 4
 * times the coarse part of each V-cycle (every level below the finest, one
 * interval per cycle); its *bytes is 0.
 * reset != 0 clears the counters of the class.  Reading is synchronous. */
amgps_status amgps_profile_enable(amgps_ctx* ctx, int on);
amgps_status amgps_profile_read(amgps_ctx* ctx, int kernel_class, int reset,
                                int64_t* launches, double* total_ms, double* bytes);

/* The algorithmic FP64 flops of the launches counted in class 0, 1 or 2
 * since its last reset (a multiply-add counts 2, a lone multiply or add 1;
 * the products of a step count 2 per nonzero of A): class 0 has them for
 * both step forms of AMGPS_OPT_STEP_FORM, classes 1 and 2 report 0.  Read it
 * before the amgps_profile_read call that resets the class.  Synchronous. */
amgps_status amgps_profile_flops(amgps_ctx* ctx, int kernel_class, double* flops);

/* The FP64 thread instructions the same launches issue (class 0; others 0):
 * one multiply-add per stored matrix entry, zeros of the SELL padding
 * included, plus one per vector term of a row.  Against the FP64 issue rate
 * (2 per clock per SM on GB300) it gives the pipe's utilisation, which the
 * flop count understates where a lone multiply takes a whole issue slot.
 * Read it before the resetting amgps_profile_read.  Synchronous. */
amgps_status amgps_profile_fp64_inst(amgps_ctx* ctx, int kernel_class, double* inst);

#ifdef __cplusplus
}
#endif

#endif /* AMGPS_H */
