/*
 * jmg.h -- C ABI of the single-GPU dense SPD solver (sm_103a, GB300).
 *
 * The operations are those of the paper's `potrs` workflow ("Software design"
 * section): solve A X = B for a symmetric positive-definite A through the
 * Cholesky factorisation A = L L^T (potrf) followed by the two triangular
 * solves (potrs); `posv` is both in one call.  The paper runs them through
 * cuSOLVERMp on a 2D process grid; this library is a one-GPU implementation
 * whose every step runs in its own CUDA kernels.
 *
 * Conventions (all entry points):
 *  - Matrices are column-major: element (i, j) of A lives at A[i + j*lda].
 *  - Only the LOWER triangle of A is read.  The strict upper triangle and the
 *    padding rows n..lda-1 are never read or written.
 *  - Every pointer to matrix data is a DEVICE pointer owned by the caller
 *    (jmg_posv_host alone takes host matrices and stages them in `work`); the
 *    library allocates no device memory.  Scratch space is the caller's `work`
 *    buffer, sized by jmg_workspace_size() (alignment: 256 bytes).
 *  - `stream` is a cudaStream_t passed as void*; work is queued on it in
 *    order.  NULL means the legacy default stream.
 *  - Return value: JMG_OK (0), -i when argument i (1-based) is illegal (LAPACK
 *    style; nothing is queued), or a positive JMG_ERR_* code.
 *  - `info` words are device pointers written asynchronously: 0, or k > 0 when
 *    the leading minor of order k is not positive definite (its pivot is
 *    <= 0 or NaN).  After a failure the factor is left partly computed, as in
 *    LAPACK, and later kernels of the same call do nothing.  info = -1 reports
 *    an internal error: a device-side wait of the solve ran out (the kernels
 *    never spin without a time limit), and B is then not a solution.
 */
#ifndef JMG_H
#define JMG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* storage type of A and B */
typedef enum { JMG_F64 = 0, JMG_F32 = 1 } jmg_dtype;

/* arithmetic of the trailing-matrix updates of the factorisation */
typedef enum {
  JMG_PREC_NATIVE = 0, /* FP64 throughout (potrf / potrs in place)              */
  JMG_PREC_BF16 = 1,   /* BF16 tensor-core updates, FP32 accumulate, FP64 refine */
  JMG_PREC_FP16 = 2,   /* FP16 tensor-core updates, FP32 accumulate, FP64 refine */
  JMG_PREC_FP8 = 3,    /* FP8 e4m3, power-of-two scale per 128x128 tile          */
  JMG_PREC_FP32 = 4    /* posv only, n <= 2048, nrhs <= 64: FP32 factor on CUDA
                          cores and FP64 refinement in ONE persistent kernel
                          (the stopping rule runs on the device; classic IR,
                          no PCG switch); larger problems: JMG_ERR_UNSUPPORTED */
} jmg_prec;

typedef enum { JMG_REFINE_IR = 0, JMG_REFINE_PCG = 1, JMG_REFINE_AUTO = 2 } jmg_refine;

typedef enum { JMG_OP_POTRF = 0, JMG_OP_POTRS = 1, JMG_OP_POSV = 2, JMG_OP_POSV_HOST = 3 } jmg_op;

enum {
  JMG_OK = 0,
  JMG_ERR_CUDA = 1,          /* a CUDA call or launch failed                       */
  JMG_ERR_WORKSPACE = 2,     /* lwork smaller than jmg_workspace_size()            */
  JMG_ERR_NOT_SPD = 3,       /* posv: the matrix is not positive definite          */
  JMG_ERR_NOT_CONVERGED = 4, /* posv: refinement stopped above the tolerance       */
  JMG_ERR_TIMEOUT = 5,       /* a device-side wait ran out; the kernel gave up     */
  JMG_ERR_UNSUPPORTED = 6,   /* option combination not built                       */
  JMG_ERR_ALIGN = 7          /* a pointer or leading dimension breaks alignment    */
};

/* Options; pass NULL for the defaults of jmg_default_options(). */
typedef struct {
  int nb;           /* diagonal-block / panel width (64 or 128)                     */
  int NB;           /* mixed modes: width of the outer blocks of the two-level      */
                    /* factorisation, i.e. the depth (in columns of L) of one       */
                    /* update of the trailing matrix (rounded down to a multiple of */
                    /* nb, at least nb; 0 = nb)                                     */
  int prec;         /* jmg_prec                                                     */
  int words;        /* split words per tensor-core operand, 1..3 (BF16 / FP16)      */
  double tol;       /* target normwise backward error of posv (mixed modes)         */
  int maxit;        /* maximum refinement iterations (IR steps + PCG steps)         */
  int refine;       /* jmg_refine                                                   */
  int shift_retry;  /* low-precision breakdown: retry with a diagonal shift (0/1): */
                    /* u_f max|a_ii| / 4, then x4 per retry (u_f: the factor's unit */
                    /* roundoff).  The FP8 factor always starts at that first shift */
  int timing;       /* 1: time the FP64 residual kernel with CUDA events (stats)    */
  int reuse_factor; /* mixed posv only: 1 = skip the factorisation and refine with  */
                    /* the factor that an earlier jmg_posv call with the same A, n  */
                    /* and options left in `work` (the adjoint solve of autograd)   */
  int resid;        /* mixed posv: how the FP64-accurate products A X of the        */
                    /* refinement are formed: 0 auto (= 2), 1 FP64 CUDA cores,      */
                    /* 2 BF16 tensor cores with error-free splitting (16 n^2 bytes  */
                    /* of extra workspace)                                          */
} jmg_options;

/* Host-side report of one posv call (filled when the call returns). */
typedef struct {
  int status;       /* JMG_OK or JMG_ERR_*                                          */
  int info;         /* potrf info of the (last) factorisation                       */
  int iters;        /* refinement iterations performed                              */
  int refine_used;  /* jmg_refine actually used (IR, or PCG after a switch)          */
  int words_used;   /* split words of the factor                                    */
  int factor_tries; /* 1 + number of shifted refactorisations                       */
  double bwd_err;   /* final max_j ||b_j - A x_j||_inf / (||A||_inf ||x_j|| + ||b_j||) */
  double shift;     /* diagonal shift of the factor (0 if none)                     */
  double anorm;     /* ||A||_inf                                                     */
  double t_factor_ms, t_solve_ms, t_refine_ms; /* host-timed phases (0 if not synced) */
  double t_resid_gpu_ms; /* with opt->timing: summed CUDA-event time of the FP64 A*X GEMM  */
  int n_resid;           /* number of FP64 A*X evaluations (residuals and PCG products)  */
  int n_hist;            /* entries of eta_hist written (may exceed 32: first 32 kept)   */
  double eta_hist[32];   /* max_j backward error after each residual / PCG step          */
  double t_solve_gpu_ms; /* with opt->timing: summed CUDA-event time of the triangular   */
  int n_solve;           /*   solve pairs (L Y = R, L^T Z = Y) and their number          */
  double t_factor_gpu_ms; /* with opt->timing: CUDA-event time of the factorisations    */
  long long h2d_bytes;    /* jmg_posv_host: bytes copied host -> device (0 otherwise)    */
  long long d2h_bytes;    /* jmg_posv_host: bytes copied device -> host (0 otherwise)    */
} jmg_stats;

/* Fill *opt with the defaults: nb 128, NB 1024, prec NATIVE, words 1, tol 1e-13,
 * maxit 300, refine AUTO, shift_retry 1, timing 0, reuse_factor 0, resid 0. */
void jmg_default_options(jmg_options* opt);

/* Bytes of `work` that the call (op, n, nrhs, dtype, opt) needs; 0 is valid. */
size_t jmg_workspace_size(int op, int n, int nrhs, int dtype, const jmg_options* opt);

/*
 * potrf -- Cholesky factorisation A = L L^T in place (paper: "Software design",
 * the factorisation step of potrs).
 *   n       order of A (n >= 0; n == 0 is a no-op)
 *   A       device, lower(A) in, lower(L) out; lda >= max(1, n)
 *   dtype   JMG_F64, or JMG_F32 (FP32 storage: FP32 panel solves and trailing
 *           updates on the CUDA cores; the diagonal blocks are factored in FP64
 *           arithmetic and rounded to FP32)
 *   info    device int, written asynchronously (see above); may not be NULL
 *   opt     NULL or options (prec must be NATIVE)
 *   work    may be NULL when jmg_workspace_size(JMG_OP_POTRF, ...) is 0
 * Asynchronous: returns once the kernels are queued on `stream`.
 */
int jmg_potrf(int n, void* A, int lda, int dtype, int* info, const jmg_options* opt,
              void* work, size_t lwork, void* stream);

/*
 * potrs -- solve (L L^T) X = B given the factor from jmg_potrf (paper:
 * "Software design", the solve step of potrs): forward substitution
 * L Y = B, then back substitution L^T X = Y.
 *   L       device, lower(L) read; lda >= max(1, n)
 *   B       device, n x nrhs, overwritten with X; ldb >= max(1, n)
 *   dtype   JMG_F64 or JMG_F32 (L and B of that type; the solve runs in it)
 * Asynchronous.
 */
int jmg_potrs(int n, int nrhs, const void* L, int lda, void* B, int ldb, int dtype,
              void* work, size_t lwork, void* stream);
/* Outcome word of jmg_potrs: once the call's kernels have completed (after a
 * synchronisation of `stream`), the first int of `work` holds 0, or
 * JMG_ERR_TIMEOUT if a device-side wait of the solve ran out (B is then not a
 * solution).  The word is written on the device; read it with a copy. */

/*
 * potrs_static -- jmg_potrs without a `work` buffer.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate device
 * memory when they solve -- code running under a fixed device-memory budget
 * handed out at start-up, a host framework that owns every device byte through
 * its own pool, or plain C callers without a device allocator -- and so cannot
 * pass the scratch that jmg_potrs wants.  It allocates nothing (no cudaMalloc,
 * no cudaFree, no allocating library routine); its scratch is a fixed 256 KiB
 * array in device memory that every GPU loading the library keeps until the
 * process exits.
 *   Arguments and results as jmg_potrs (FP64 only).
 *   Limit: ceil(nrhs/16) * (2 + ceil(n/32)) + 1 <= 65536 ints of
 *     scratch (e.g. nrhs <= 496 at n = 65536); larger problems return JMG_ERR_WORKSPACE
 *     with nothing queued.
 *   The first call on a device, with that device current, looks up the device
 *     address of the array (cudaGetSymbolAddress); make that first call before
 *     any stream capture.
 *   Every call shares the one array, which keeps the last call's contents (the
 *     call clears what must start at zero): calls that overlap on the GPU (for
 *     example on two streams) race and must not be issued.
 */
int jmg_potrs_static(int n, int nrhs, const void* L, int lda, void* B, int ldb, int dtype,
                     void* stream);

/*
 * potrs_static_status -- the outcome of the last jmg_potrs_static call on the
 * current device: waits for `stream`, then sets *status (a HOST int) to 0, or
 * to JMG_ERR_TIMEOUT if a device-side wait of that solve ran out (its B is then
 * not a solution).  Allocates nothing.  Returns JMG_OK, -1 for a NULL status,
 * or JMG_ERR_CUDA.
 */
int jmg_potrs_static_status(int* status, void* stream);

/*
 * posv -- solve A X = B (paper: "Software design", potrs as one call).
 *   prec == NATIVE: potrf then potrs, in place (A becomes L), asynchronous;
 *     dtype JMG_F64 or JMG_F32.
 *   prec != NATIVE: A is PRESERVED (it is needed for the FP64 residual).  The
 *     factor is built in `work` with tensor-core trailing updates and used as
 *     the preconditioner of an FP64 refinement loop that stops when the
 *     backward error (see jmg_stats.bwd_err) is <= opt->tol.  This mode
 *     synchronises `stream` once per refinement iteration and returns only when
 *     X is final.  B is overwritten with X.  FP64 data only (JMG_F32 returns
 *     JMG_ERR_UNSUPPORTED).
 *   prec == FP32 (n <= 2048, nrhs <= 64): the same solve as ONE persistent
 *     cooperative kernel: FP32 tile Cholesky (shifted and refactored on the
 *     device after a breakdown when opt->shift_retry), FP64 residuals and the
 *     stopping rule on the device; the call synchronises `stream` once, after
 *     the kernel, to read the status.  opt->nb, NB, words, refine and resid
 *     are ignored.  Larger problems return JMG_ERR_UNSUPPORTED.
 *   info    device int (potrf convention); may not be NULL
 *   stats   host pointer or NULL
 */
int jmg_posv(int n, int nrhs, void* A, int lda, void* B, int ldb, int dtype, int* info,
             const jmg_options* opt, jmg_stats* stats, void* work, size_t lwork,
             void* stream);

/*
 * posv_host -- jmg_posv on HOST buffers: the call copies lower(A) and B to the
 * device, solves there exactly as jmg_posv does (every step in the library's
 * kernels) and copies X back, returning once X is in host memory.  It is the
 * whole job as a caller without device-resident data sees it.
 *   A       host, n x n column-major, lda >= max(1, n).  The n x n block is
 *           transferred whole (one linear copy when lda == n); its strict upper
 *           triangle travels along but is never used.  (Skipping it would take
 *           one copy row per column, about 1 us each on GB300: more than the
 *           bytes it saves below n ~ 50000.)
 *   B       host, n x nrhs, ldb >= max(1, n); read only
 *   X       host, n x nrhs, ldx >= max(1, n); may be B itself.  Holds the
 *           solution on JMG_OK and the last iterate on JMG_ERR_NOT_CONVERGED;
 *           otherwise its contents are unspecified
 *   dtype   JMG_F64 (every mode) or JMG_F32 (prec NATIVE)
 *   info    HOST int: 0, or k > 0 when the leading minor of order k is not
 *           positive definite (the call then returns JMG_ERR_NOT_SPD)
 *   opt, stats  as jmg_posv; stats->h2d_bytes / d2h_bytes report the copies
 *   work    device, jmg_workspace_size(JMG_OP_POSV_HOST, n, nrhs, dtype, opt)
 *           bytes, 256-byte aligned: the device copies of A and B, then
 *           jmg_posv's own workspace.  Host A, B and X are neither kept nor
 *           registered; page-locked host memory (cudaHostAlloc,
 *           cudaHostRegister) copies fastest.
 * Synchronous: the call synchronises `stream` before it returns, on every
 * path that queued work, so the host buffers may be reused at once.
 */
int jmg_posv_host(int n, int nrhs, const void* A, int lda, const void* B, int ldb, void* X,
                  int ldx, int dtype, int* info, const jmg_options* opt, jmg_stats* stats,
                  void* work, size_t lwork, void* stream);

/*
 * posv_batched -- many small independent systems A_b X_b = B_b (b = 0 .. batch-1)
 * in one call: every A_b = L_b L_b^T in place, then X_b over B_b.  The paper's
 * potrs is a batched primitive of its framework ("Summary": it composes with
 * the framework's transformations, including vectorisation over a batch);
 * this is its small-matrix form, one CTA per system.
 *   n       order of every A_b, 0 <= n <= 128 (larger: JMG_ERR_UNSUPPORTED)
 *   A       device; A_b = A + b * strideA, column-major, lower read, becomes L_b;
 *           lda >= max(1, n), strideA >= lda * n (elements)
 *   B       device; B_b = B + b * strideB, n x nrhs, overwritten with X_b;
 *           ldb >= max(1, n), strideB >= ldb * nrhs (elements)
 *   dtype   JMG_F64 or JMG_F32 (the plain path in the storage type)
 *   info    device int[batch], written asynchronously: info[b] = 0, or k > 0 when
 *           the leading minor of order k of A_b is not positive definite (that
 *           B_b is then left unchanged)
 * Asynchronous; allocates nothing.
 */
int jmg_posv_batched(int n, int nrhs, int batch, void* A, int lda, long long strideA, void* B,
                     int ldb, long long strideB, int dtype, int* info, void* stream);

/*
 * logdet -- log det A = 2 sum_i log L_ii from a factor made by jmg_potrf
 * (paper: "Software design", potrs can also return log det A).
 *   dtype   of L: JMG_F64 or JMG_F32 (the sum is formed in FP64 either way)
 *   out     device double, written asynchronously
 */
int jmg_logdet(int n, const void* L, int lda, int dtype, double* out, void* stream);

/*
 * sym_grad -- adjoint of X = A^{-1} B with respect to the symmetric A:
 *     Abar = -(Bbar X^T + X Bbar^T) / 2         (n x n, full symmetric, FP64)
 * where Bbar = A^{-1} Xbar is the adjoint solve.  The paper exposes potrs as a
 * primitive that composes with the framework's transformations ("Summary");
 * this is reverse-mode differentiation of it.  Bbar, X: n x nrhs column-major
 * (ldb, ldx >= n); Abar: ldab >= n, every element of the n x n block written.
 * Asynchronous.
 */
int jmg_sym_grad(int n, int nrhs, const double* Bbar, int ldb, const double* X, int ldx,
                 double* Abar, int ldab, void* stream);

/*
 * rowmajor_to_colmajor -- in-place layout conversion (paper: "Local
 * memory-layout conversion": a row-major array of the framework becomes the
 * column-major buffer the solver wants, without a second full-sized copy).
 *   m, n    rows and columns of the matrix M (m, n >= 0)
 *   A       device, m * n elements: on entry M row-major (M(i, j) at i n + j),
 *           on exit M column-major (M(i, j) at i + j m, i.e. the buffer holds
 *           the row-major n x m matrix M^T); the logical matrix is unchanged
 *   dtype   JMG_F64 or JMG_F32 (the elements are moved bit for bit)
 *   work    device scratch, at least jmg_layout_workspace(m, n, dtype) bytes;
 *           a larger buffer lets more column batches run at once (the move is
 *           done in batches bounded by it)
 * colmajor_to_rowmajor is the inverse move (a column-major m x n M back to
 * row-major), with scratch jmg_layout_workspace(n, m, dtype).
 * Asynchronous.  Returns JMG_OK, -i for an illegal argument i, or
 * JMG_ERR_WORKSPACE.
 */
size_t jmg_layout_workspace(long long m, long long n, int dtype);
int jmg_rowmajor_to_colmajor(long long m, long long n, void* A, int dtype, void* work,
                             size_t lwork, void* stream);
int jmg_colmajor_to_rowmajor(long long m, long long n, void* A, int dtype, void* work,
                             size_t lwork, void* stream);

/* Human-readable name of a status code. */
const char* jmg_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* JMG_H */
