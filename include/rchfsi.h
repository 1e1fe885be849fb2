/*
 * rchfsi.h -- C ABI of the GB300 (sm_103a) R-ChFSI eigensolver.
 *
 * The library finds the nev smallest eigenpairs of a Hermitian-definite pencil
 *     A u = lambda B u        (A Hermitian, B Hermitian positive definite; Section 2, Eq. (1))
 * with subspace iteration accelerated by a Chebyshev filter (Algorithm 1).  The filter is
 * either the classical three-term recurrence on the eigenvector block (Algorithm 2, "ChFSI")
 * or its residual-based reformulation (Algorithm 3, "R-ChFSI", Proposition 3.3 and the
 * inexact recurrence that follows it), whose operator products may use an approximate inverse
 * D^-1 of B and reduced precision (FP32 / TF32 / BF16 with FP32 accumulation).  Residuals,
 * Gram matrices, the Cholesky factorisation and the projected eigenproblem stay in FP64.
 *
 * Conventions
 *   - Every function returns an int status: RCHFSI_OK (0) on success, a negative RCHFSI_ERR_*
 *     code on failure.  No C++ exception crosses the ABI.  rchfsi_last_error() gives the text.
 *   - Blocks (X, W, Y_p) are m x N arrays of double, ROW-major ("dof-major": row i holds the N
 *     entries of dof i, N contiguous), N = rchfsi_params.block.  Eigenvalue arrays hold N doubles.
 *   - Every array argument may be a host pointer or a CUDA device pointer of the handle's device;
 *     the library detects which (cudaPointerGetAttributes) and stages host data through its own
 *     device buffers.  The caller owns all argument buffers; the library copies what it keeps.
 *   - Calls on one handle are serialised on the handle's CUDA stream and return after the result
 *     is complete (the stream is synchronised before returning).  Device inputs are read on that
 *     stream: work that writes them on another stream (including the legacy default stream,
 *     which a library-owned non-blocking stream does not wait for) must be complete before the
 *     call.  A handle must not be used by two host threads at once.  Different handles are
 *     independent.
 *   - Complex Hermitian problems (field = RCHFSI_COMPLEX, e.g. the Bloch k-point operators of
 *     Section 4.2) take complex blocks X, W, Y_p, the dense A and the cell matrices A_cells as
 *     interleaved (re, im) pairs of doubles, i.e. C99 `double complex` / NumPy complex128 arrays of
 *     the same shape, row-major.  B, B_cells, Dinv and every eigenvalue / residual array stay
 *     real.  Internally the library solves the real symmetric embedding
 *     [[Ar, -Ai], [Ai, Ar]] of order 2m with the block [[Xr, -Xi], [Xi, Xr]] of 2N columns; each
 *     complex eigenpair appears twice there, and one representative per pair is returned.  The
 *     filter runs on N embedded columns only (the other N are their products with i).  block is
 *     limited to 3072 for complex problems.  A_filter and Dinv_dense are real-only.
 */
#ifndef RCHFSI_H
#define RCHFSI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status codes */
#define RCHFSI_OK 0
#define RCHFSI_PENDING 1               /* rchfsi_poll: request not finished yet */
#define RCHFSI_ERR_INVALID_ARG (-1)    /* a size, pointer or parameter is out of range */
#define RCHFSI_ERR_OOM (-2)            /* device allocation failed or the HBM budget is exceeded */
#define RCHFSI_ERR_NOT_CONVERGED (-3)  /* max_iter reached above the tolerance */
#define RCHFSI_ERR_STAGNATED (-4)      /* residual stopped decreasing (see rchfsi_params.stall_iters) */
#define RCHFSI_ERR_ILL_CONDITIONED (-5) /* Gram matrix not positive definite (Cholesky failed) */
#define RCHFSI_ERR_NUMERIC (-6)        /* NaN or Inf met */
#define RCHFSI_ERR_TIMEOUT (-7)        /* a bounded device wait ran out */
#define RCHFSI_ERR_CUDA (-8)           /* a CUDA runtime / library call failed */
#define RCHFSI_ERR_NO_OPERATOR (-9)    /* rchfsi_set_operator has not been called */
#define RCHFSI_ERR_UNSUPPORTED (-10)   /* valid request that this build does not implement */

/* ---------------------------------------------------------------- enums */
typedef enum {
  RCHFSI_FP64 = 0, /* products in FP64 (parity mode and the FP64 baseline) */
  RCHFSI_FP32 = 1, /* FP32 storage of R_X, R_Y and FP32 (FFMA) products */
  RCHFSI_TF32 = 2, /* FP32 storage, tcgen05 kind::tf32 products, FP32 accumulation */
  RCHFSI_BF16 = 3  /* BF16 storage of the product operands, tcgen05 kind::f16, FP32 accumulation */
} rchfsi_precision;

typedef enum {
  RCHFSI_METHOD_RCHFSI = 0, /* Algorithm 3 */
  RCHFSI_METHOD_CHFSI = 1   /* Algorithm 2 with H = D^-1 A */
} rchfsi_method;

typedef enum { RCHFSI_REAL = 0, RCHFSI_COMPLEX = 1 } rchfsi_field;

typedef enum {
  RCHFSI_OP_DENSE = 0,  /* dense A (and B) */
  RCHFSI_OP_FE_CELL = 1 /* finite-element cell matrices + connectivity (element-level operator) */
} rchfsi_op_kind;

/* ---------------------------------------------------------------- parameters */
typedef struct rchfsi_params {
  int64_t m;             /* order of A and B (> 0) */
  int32_t nev;           /* wanted eigenpairs (1 <= nev <= block) */
  int32_t block;         /* N: subspace dimension (nev <= N <= m) */
  int32_t degree;        /* Chebyshev degree p used by rchfsi_solve (>= 1) */
  int32_t precision;     /* rchfsi_precision of the filter's operator products */
  int32_t method;        /* rchfsi_method */
  int32_t field;         /* rchfsi_field */
  int32_t max_iter;      /* outer iterations allowed in rchfsi_solve */
  int32_t min_iter;      /* outer iterations run before the tolerance may stop the loop */
  int32_t lanczos_steps; /* k of the Lanczos upper-bound estimate (>= 2) */
  int32_t stall_iters;   /* report RCHFSI_ERR_STAGNATED when the residual has not improved by 2x in
                            this many iterations (0 = never) */
  int32_t fixed_bounds;  /* 1: use lmin/lT/lmax below for every filter; 0: Ritz values + Lanczos */
  double tol;            /* relative residual tolerance ||Ax - eps Bx|| / (||A|| ||x||) */
  double lmin, lT, lmax; /* bounds when fixed_bounds = 1 */
  uint64_t hbm_budget_bytes; /* device memory the handle may hold (0 = unlimited) */
  int32_t rr_mode;       /* FP64 products of the residual / Rayleigh-Ritz steps: RCHFSI_RR_FP64 (FP64
                            arithmetic units) or RCHFSI_RR_FP64_EMULATED (FP64-accurate products from
                            exact BF16 slices on the tensor cores) */
  int32_t eig_mode;      /* N x N projected eigenproblem: RCHFSI_EIG_SYEVD (cuSOLVER dsyevd, a library
                            call), RCHFSI_EIG_JACOBI or RCHFSI_EIG_TRIDIAG (this library's kernels) */
} rchfsi_params;

typedef enum {
  RCHFSI_EIG_SYEVD = 0,  /* divide and conquer (cuSOLVER) */
  RCHFSI_EIG_JACOBI = 1, /* parallel cyclic Jacobi, one cooperative kernel, tolerance 1e-14 */
  RCHFSI_EIG_TRIDIAG = 2 /* this library's Householder tridiagonalisation (one thread-block cluster or
                            cooperative grid), Sturm bisection and inverse iteration with Gram-Schmidt in
                            clusters of numerically equal eigenvalues; falls back to RCHFSI_EIG_SYEVD for an
                            order above 3072 or a cluster of more than 256 equal eigenvalues */
} rchfsi_eig_mode;

typedef enum {
  RCHFSI_RR_FP64 = 0,          /* FP64 FMA (DFMA) GEMMs */
  RCHFSI_RR_FP64_EMULATED = 1  /* error-free BF16 splitting, 7 slices, exact per-chunk FP32 sums; the
                                  FE cell contributions summed in 64-bit fixed point (order-free) */
} rchfsi_rr_mode;

/* Operator description for rchfsi_set_operator.  Unused fields must be 0 / NULL.
 * Dense:  A (m*m, row-major, symmetric), optional B (m*m; NULL = identity), optional A_filter
 *         (m*m; the matrix used inside the filter instead of A, e.g. a perturbed or rounded copy,
 *         Section 4.1.2), and the approximate inverse of B: Dinv (diagonal, m entries), or
 *         Dinv_dense (m*m row-major), or neither (= identity).
 * FE cell: n_cells cells of n_c dofs, cell_dofs[n_cells*n_c] (int32 global dof of each local
 *         node), A_cells[n_cells*n_c*n_c] (row-major cell matrices), B_cells (same layout, or one
 *         n_c*n_c matrix shared by all cells when B_cells_shared = 1), Dinv (m entries).  The
 *         global operator is A = sum_c P_c^T A_c P_c (element-level products, Section 4.2).
 */
typedef struct rchfsi_operator {
  int32_t kind;  /* rchfsi_op_kind */
  int32_t field; /* rchfsi_field */
  int64_t m;
  const double* A;
  const double* B;
  const double* A_filter;
  const double* Dinv;
  const double* Dinv_dense;
  int64_t n_cells;
  int32_t n_c;
  int32_t B_cells_shared;
  const int32_t* cell_dofs;
  const double* A_cells;
  const double* B_cells;
} rchfsi_operator;

/* Statistics of one rchfsi_solve. */
typedef struct rchfsi_stats {
  int32_t iterations;      /* filter + Rayleigh-Ritz passes done */
  int32_t status;          /* same as the return value */
  double max_rel_residual; /* max_{j<nev} ||Ax_j - eps_j Bx_j|| / (||A|| ||x_j||) at exit */
  double max_abs_residual; /* max_{j<nev} ||Ax_j - eps_j Bx_j|| at exit (the paper's measure) */
  double lmax;             /* Lanczos upper bound used */
  double normA;            /* ||A||_2 estimate used in the relative residual */
  double t_total_ms;       /* wall time of the solve on the device stream */
  double t_filter_ms;      /* time in the Chebyshev filters */
  double t_rr_ms;          /* time in Rayleigh-Ritz + residuals */
  double filter_flops;     /* algorithmic flops of all filter operator products */
  int64_t operator_applies;/* block operator products done by the filters */
  double* history;         /* optional caller array of max_iter+1 doubles: max relative residual
                              before each filter (may be NULL) */
  int32_t cholqr_retries;  /* Rayleigh-Ritz steps whose Gram matrix G_B had no Cholesky factor and
                              that went through the shifted Cholesky QR step (real problems) */
} rchfsi_stats;

/* ---------------------------------------------------------------- lifecycle */

/* Fill *p with defaults: nev = 1, block = 1, degree = 20, FP64, R-ChFSI, real, max_iter = 100,
 * min_iter = 0, lanczos_steps = 10, stall_iters = 0, fixed_bounds = 0, tol = 1e-8,
 * rr_mode = RCHFSI_RR_FP64_EMULATED, eig_mode = RCHFSI_EIG_TRIDIAG. */
int rchfsi_params_default(rchfsi_params* p);

/* Create a handle on the current CUDA device.  cuda_stream: a cudaStream_t to run on, or NULL
 * for a library-owned stream.  The params are copied.  Errors: INVALID_ARG for bad sizes. */
int rchfsi_create(struct rchfsi_ctx** out, const rchfsi_params* p, void* cuda_stream);

/* Release every device buffer of the handle.  Safe on NULL. */
int rchfsi_destroy(struct rchfsi_ctx* h);

/* Update degree / precision / method / bounds / tolerances of an existing handle (m, block
 * and field must not change).  Cached low-precision operator copies are kept. */
int rchfsi_set_params(struct rchfsi_ctx* h, const rchfsi_params* p);

/* Upload the operator (copied to device memory) and precompute what the filter needs:
 * A D^-1 for Algorithm 3 and D^-1 A for Algorithm 2 (dense), and the reduced-precision copies.
 * Errors: INVALID_ARG (sizes/pointers, field differing from the handle's), UNSUPPORTED
 * (A_filter or Dinv_dense with a complex operator), OOM. */
int rchfsi_set_operator(struct rchfsi_ctx* h, const rchfsi_operator* op);

/* ---------------------------------------------------------------- the filter (Algorithm 3) */

/* R-ChFSI filter, Algorithm 3, on caller data:
 *   X      m x N current Ritz vectors X^(i)                       (row-major)
 *   Lambda N   current Ritz values (diagonal of Lambda^(i))
 *   W      m x N residual A X - B X Lambda (the algorithm's input "Y")   (row-major)
 *   lmin, lT, lmax  bounds (lmin < lT < lmax)
 *   degree p >= 1
 *   Yp     m x N output: D^-1 R_Y + X Lambda_Y                     (row-major)
 * The degree loop runs the fused step R_X <- a_k A D^-1 R_Y + b_k R_Y + c_k R_X + a_k W Lambda_Y
 * in the handle's precision.  Errors: NO_OPERATOR, INVALID_ARG. */
int rchfsi_filter(struct rchfsi_ctx* h, const double* X, const double* Lambda, const double* W, double lmin,
                  double lT, double lmax, int degree, double* Yp);

/* Classical ChFSI filter, Algorithm 2: Yp = C_p(D^-1 A) X (row-major m x N). */
int rchfsi_chfsi_filter(struct rchfsi_ctx* h, const double* X, double lmin, double lT, double lmax, int degree,
                        double* Yp);

/* ---------------------------------------------------------------- FP64 building blocks */

/* W = A X - B X diag(Lambda) in FP64 (Algorithm 3 input; Section 2.1 residual) and its column
 * 2-norms rnorm[N] (rnorm may be NULL). */
int rchfsi_residual(struct rchfsi_ctx* h, const double* X, const double* Lambda, double* W, double* rnorm);

/* Rayleigh-Ritz for a non-orthogonal basis (Section 2.1, Algorithm 1 steps 2-3), FP64:
 * columns of Y scaled to unit norm, G_A = Y^T A Y, G_B = Y^T B Y, Cholesky G_B = L L^T, eigen-
 * decomposition of L^-1 G_A L^-T, X = Y L^-T V (B-orthonormal), evals ascending.
 * When G_B has no Cholesky factor (a numerically rank-deficient basis), a real problem's basis is
 * first preconditioned by one shifted Cholesky QR step in the B inner product (Y <- Y L_s^-T,
 * L_s L_s^T = G_B + s I, s = 11 (m N + N (N + 1)) 2^-53 tr(G_B)) and the Gram matrices are formed
 * again.  Errors: ILL_CONDITIONED when G_B (after that step) is not numerically positive definite,
 * e.g. an indefinite B. */
int rchfsi_rayleigh_ritz(struct rchfsi_ctx* h, const double* Y, double* X, double* evals);

/* k-step Lanczos (no re-orthogonalisation) on D^-1/2 A D^-1/2 from start vector v0 (m doubles):
 * *lmax = theta_max + beta_k (upper-bound estimate of the filter operator's spectrum, the paper
 * only requires an estimate, Section 2.1), and on A: *normA = max |theta| (||A||_2 estimate). */
int rchfsi_lanczos_bounds(struct rchfsi_ctx* h, const double* v0, int steps, double* lmax, double* normA);

/* ---------------------------------------------------------------- the solver (Algorithm 1) */

/* Subspace iteration, Algorithm 1 with the handle's filter (Algorithm 3 or 2):
 *   X_inout  m x N: initial guess on entry (any full-rank block, e.g. Gaussian), B-orthonormal Ritz
 *            vectors on exit (row-major)
 *   evals    N Ritz values, ascending (first nev are the wanted ones)
 *   resid    N relative residuals ||Ax_j - eps_j Bx_j|| / (||A|| ||x_j||) (may be NULL)
 *   st       statistics (may be NULL)
 * Bounds: lmax from Lanczos on D^-1/2 A D^-1/2 started from the first column of X_inout;
 * lmin / lT = smallest / largest current Ritz value (unless fixed_bounds).  Stops when the
 * max relative residual over the first nev columns is <= tol.  Returns OK, NOT_CONVERGED,
 * STAGNATED, ILL_CONDITIONED or NUMERIC (X_inout/evals hold the last iterate in every case). */
int rchfsi_solve(struct rchfsi_ctx* h, double* X_inout, double* evals, double* resid, rchfsi_stats* st);

/* Several independent problems solved together (e.g. the k-points of a Bloch problem): count
 * distinct handles, each with its operator set; X_inout[i], evals[i], resid[i] (evals / resid may be
 * NULL, or hold NULL entries), stats[i] (stats may be NULL) are as for rchfsi_solve.  Every problem
 * runs Algorithm 1 with its own bounds and convergence test, in lockstep outer iterations: the
 * filters of all unconverged problems with FE operators, R-ChFSI, one TF32/BF16 precision and one
 * degree run together - per degree step the recurrence terms of each problem and ONE persistent
 * tensor-core launch over the cells of every problem (up to 64 real products: 16 complex
 * problems), the degree loop replayed from a CUDA graph, the cell-GEMM column tile chosen by timing
 * candidates once per shape - and the residual / Rayleigh-Ritz steps of the problems run
 * concurrently, each on its own handle's stream from its own host thread.  Other problems are
 * filtered one after the other.  The handles must not be used elsewhere during the call.  Returns
 * OK when every problem converged, else the status of the first one that did not (each
 * stats[i].status holds its own). */
int rchfsi_solve_batch(struct rchfsi_ctx** handles, int count, double** X_inout, double** evals, double** resid,
                       rchfsi_stats* stats);

/* ---------------------------------------------------------------- serving (request loop) */

/* One eigensolve request for the server: an operator (copied at submit), the solver params, and
 * an optional warm-start key.  Requests with the same nonzero warm_key and the same (m, block)
 * start from the previous result of that key kept on the device (Ritz vectors and values), as
 * an outer self-consistent loop would; X0 (m x N, may be NULL when a warm start exists) is the
 * initial guess otherwise. */
typedef struct rchfsi_request {
  rchfsi_operator op;
  rchfsi_params params;
  const double* X0;
  uint64_t warm_key;
} rchfsi_request;

typedef struct rchfsi_result {
  int32_t status;     /* RCHFSI_OK or an error of rchfsi_solve */
  int32_t iterations;
  double max_rel_residual;
  double latency_ms;  /* submit -> completion */
  double queue_ms;    /* submit -> admission */
  double* evals;      /* caller buffer of block doubles to receive the Ritz values (may be NULL) */
  double* X;          /* caller buffer of m x block doubles for the Ritz vectors (may be NULL) */
  char error[160];    /* text of the error when status != RCHFSI_OK (empty otherwise) */
} rchfsi_result;

/* Create / destroy a server: up to `slots` requests run concurrently, each on its own stream,
 * admitted in arrival order while their estimated device footprint fits in hbm_budget_bytes. */
int rchfsi_server_create(struct rchfsi_ctx** out, int slots, uint64_t hbm_budget_bytes);
int rchfsi_server_destroy(struct rchfsi_ctx* server);
/* Enqueue a request; *ticket identifies it.  The operator arrays are copied before returning. */
int rchfsi_submit(struct rchfsi_ctx* server, const rchfsi_request* rq, uint64_t* ticket);
/* RCHFSI_PENDING while running; otherwise fills *out (copying evals / X into the caller's
 * buffers when given) and returns RCHFSI_OK; the ticket is then retired. */
int rchfsi_poll(struct rchfsi_ctx* server, uint64_t ticket, rchfsi_result* out);

/* ---------------------------------------------------------------- kernel timers */

/* Kernel classes timed by the opt-in device timers. */
typedef enum {
  RCHFSI_KERNEL_FILTER_TC = 0,     /* tcgen05 dense filter product (TF32 / BF16) */
  RCHFSI_KERNEL_SPLITK_REDUCE = 1, /* split-K reduction fused with the recurrence update */
  RCHFSI_KERNEL_FILTER_SIMT = 2,   /* SIMT dense filter product (FP32 / FP64) */
  RCHFSI_KERNEL_GEMM_F64 = 3,      /* FP64 GEMMs of the residual and Rayleigh-Ritz steps */
  RCHFSI_KERNEL_FE_CELL = 4,       /* FE cell-matrix product inside the filter */
  RCHFSI_KERNEL_FE_CELL_F64 = 5,   /* FE cell-matrix product of the residual / Rayleigh-Ritz (FP64) */
  RCHFSI_KERNEL_GEMM_F64_EMU = 6,  /* FP64-accurate GEMM from BF16 slices on the tensor cores; flops are
                                      the tensor-core flops (28 slice products) */
  RCHFSI_KERNEL_SMALL_DENSE = 7,   /* N x N steps of Rayleigh-Ritz: Cholesky and L^-1, the N x N
                                      FP64 GEMMs of rr_mode fp64, symmetrisation */
  RCHFSI_KERNEL_EIG = 8,           /* projected N x N eigensolver (this library's tridiagonal or Jacobi
                                      kernels, or the cuSOLVER dsyevd call of RCHFSI_EIG_SYEVD) */
  RCHFSI_KERNEL_RR_AUX = 9,        /* m x N passes of Rayleigh-Ritz: column norms and scaling, BF16
                                      slicing of the emulated GEMM and FE product operands, and the
                                      FE products' fixed-point to FP64 conversion */
  RCHFSI_KERNEL_CLASSES = 10
} rchfsi_kernel_class;

/* enable = 1: start timing every instrumented launch of this handle with CUDA events on the
 * launching stream (previous records are cleared); enable = 0: stop and clear.  Either value
 * restarts the launch count read with kernel_class = RCHFSI_KERNEL_CLASSES, so enable = 0 counts
 * launches without adding any event to the stream. */
int rchfsi_profile(struct rchfsi_ctx* h, int enable);

/* Totals for one kernel class since rchfsi_profile(h, 1): device time (ms), number of launches,
 * and the algorithmic flops and bytes of those launches (each may be NULL).  Synchronises the
 * handle's stream.  kernel_class = RCHFSI_KERNEL_CLASSES returns in *launches the number of all
 * kernel launches of this library (any handle, any thread) since the last rchfsi_profile(h, .). */
int rchfsi_profile_read(struct rchfsi_ctx* h, int kernel_class, double* total_ms, int64_t* launches,
                        double* flops, double* bytes);

/* ---------------------------------------------------------------- allocation-free filter step */

/* Size of the fixed scratch array behind rchfsi_filter_step_tf32_static: 4 Mi floats (16 MiB). */
#define RCHFSI_STATIC_SCRATCH_FLOATS (4u * 1024u * 1024u)

/* One TF32 step of the filter recurrence that allocates no device memory.  The paper has no
 * counterpart; it is for callers that cannot let a library call cudaMalloc -- for example a
 * serving loop that must not allocate after start-up (cudaMalloc can synchronise the device and
 * its latency is unbounded), or an application whose device memory is all owned by its own pool
 * allocator.  The caller allocates and passes every input and output:
 *   out = a * (A Ry) + b * Ry + c * Rx + a * W diag(lambda_y)
 *   A        m x m FP32, row-major, row pitch lda (the operator A D^-1, values read as TF32)
 *   Ry, Rx, W, out   m x n FP32, column-major, leading dimension ldr; Rx and W may be NULL (their
 *            terms are dropped); out may be the same array as Rx, but must not overlap Ry, W or
 *            only part of Rx (checked on the byte ranges; INVALID_ARG otherwise)
 *   lambda_y n doubles
 * lda and ldr must be >= m and multiples of 4; all arrays are device memory of the current device
 * (or managed memory; device memory of another GPU is refused with INVALID_ARG);
 * cuda_stream is the stream to run on (NULL = legacy default stream).  Returns after the step has
 * completed (the stream is synchronised).
 * Scratch: the split-K partial sums live in one file-scope __device__ array of
 * RCHFSI_STATIC_SCRATCH_FLOATS floats, which every GPU that loads the library holds until the
 * process exits.  Shapes whose partials need more return RCHFSI_ERR_INVALID_ARG with a message
 * giving both sizes (rchfsi_last_error(NULL, ...)).  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Every call shares the one array and its timeout flag: calls that
 * overlap on the GPU (other streams, other host threads) race and must be serialised by the caller.
 * Errors: INVALID_ARG (sizes, pitches, host pointers, scratch too small), TIMEOUT, CUDA. */
int rchfsi_filter_step_tf32_static(const float* A, int64_t lda, const float* Ry, const float* Rx, const float* W,
                                   const double* lambda_y, float a, float b, float c, int64_t m, int64_t n,
                                   int64_t ldr, float* out, void* cuda_stream);

/* ---------------------------------------------------------------- errors */
const char* rchfsi_strerror(int code);
/* Copy the last error message of the handle (NUL-terminated, truncated to len). */
int rchfsi_last_error(struct rchfsi_ctx* h, char* buf, size_t len);

typedef struct rchfsi_ctx* rchfsi_t;

#ifdef __cplusplus
}
#endif
#endif /* RCHFSI_H */
