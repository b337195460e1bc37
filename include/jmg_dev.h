/*
 * jmg_dev.h -- kernel-level entry points of the SPD solver library, exported
 * for tests, benchmarks and profiling.  They run one building block of
 * jmg_potrf / jmg_posv in isolation, on caller-owned device memory, queued on
 * `stream` (a cudaStream_t passed as void*).  Conventions as in jmg.h.
 */
#ifndef JMG_DEV_H
#define JMG_DEV_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Trailing-matrix update on the tensor cores (the SYRK step of a right-looking
 * blocked Cholesky factorisation):
 *     C[i, j] -= sum_k PA[i, k] * PB[j, k]     for 0 <= j <= i < m, j < ncols
 * PA, PB: m x kext, ROW-major (k contiguous), leading dimension ldp elements,
 *   element type BF16 (prec JMG_PREC_BF16) or FP16 (JMG_PREC_FP16); kext and
 *   ldp multiples of 64; base addresses 16-byte aligned.  PB may equal PA.
 * C: FP32, column-major, ldc >= m; only the lower trapezoid (rows >= columns,
 *   columns < ncols <= m) is touched.
 * err: device int; set non-zero if a device-side wait ran out (the update is
 *   then incomplete).  Asynchronous.
 */
int jmg_dev_syrk_tc(int m, int ncols, int kext, const void* PA, const void* PB, int ldp,
                    int prec, float* C, int ldc, int* err, void* stream);

/*
 * FP8 (e4m3) variant with one power-of-two scale per 128-row tile of the panel
 * (with a 128-wide panel, kext = 128, that is one scale per 128 x 128 tile):
 *     C[i, j] -= 2^-(e[i/128] + e[j/128]) * sum_k Q[i, k] Q[j, k]
 *         for 0 <= j <= i < m, j < ncols
 * Q: m x kext e4m3 bytes, row-major, ldq bytes (kext, ldq multiples of 128;
 * 16-byte aligned); e: ceil(m/128) int8 exponents.  C, err as above.
 */
int jmg_dev_syrk_fp8(int m, int ncols, int kext, const void* Q, int ldq, const signed char* e,
                     float* C, int ldc, int* err, void* stream);

/*
 * The same with one set of exponents per 128-deep chunk of K (the two-level
 * factorisation applies several panels, each quantised with its own tile
 * scales, in one update):
 *     C[i, j] -= sum_c 2^-(e[c*lde + i/128] + e[c*lde + j/128]) * sum_{k in chunk c} Q[i, k] Q[j, k]
 * lde >= ceil(m/128) (0: every chunk uses e[0 .. ceil(m/128)); kext % 128 == 0.
 */
int jmg_dev_syrk_fp8_chunks(int m, int ncols, int kext, const void* Q, int ldq,
                            const signed char* e, int lde, float* C, int ldc, int* err,
                            void* stream);

/*
 * FP64 residual R = B - A X with A symmetric (lower(A) read), the kernel that
 * drives the refinement loop of jmg_posv.  X, B, R: n x nrhs column-major.
 * Also writes colmax[0..nrhs) = ||r_j||_inf, colmax[nrhs..2nrhs) = ||x_j||_inf,
 * colmax[2nrhs..3nrhs) = ||b_j||_inf.  work: jmg_dev_residual_workspace bytes.
 */
size_t jmg_dev_residual_workspace(int n, int nrhs);
int jmg_dev_residual(int n, int nrhs, const double* A, int lda, const double* X, int ldx,
                     const double* B, int ldb, double* R, int ldr, double* colmax,
                     void* work, size_t lwork, void* stream);

/*
 * The same residual with the product A X formed on the BF16 tensor cores by
 * error-free splitting into 8 slices of 7 bits per operand (Ozaki, Ogita,
 * Oishi and Rump 2012) and exact FP32 accumulation over windows of 256,
 * combined in FP64: FP64-accurate, and the kernel the refinement loop uses
 * when opt->resid selects it.  Arguments as jmg_dev_residual; `work` holds the
 * slices of A (16 n^2 bytes) and of X: jmg_dev_residual_split_workspace bytes.
 * `err` (device int) is set if a device-side wait ran out.
 */
size_t jmg_dev_residual_split_workspace(int n, int nrhs);
int jmg_dev_residual_split(int n, int nrhs, const double* A, int lda, const double* X, int ldx,
                           const double* B, int ldb, double* R, int ldr, double* colmax,
                           int* err, void* work, size_t lwork, void* stream);

/* ||A||_inf of the symmetric matrix held in lower(A) (FP64), to *out. */
int jmg_dev_norm_inf(int n, const double* A, int lda, double* out, void* work, size_t lwork,
                     void* stream);

/*
 * Throughput probes: `blocks` CTAs of 256 threads each run `iters` rounds of
 * independent dependent-chain arithmetic and store a checksum to sink[0..):
 *   kind 0: FP64 fused multiply-add (DFMA), 2 flops each, 8 chains per thread
 *   kind 1: FP64 mma.sync m8n8k4 (512 flops per warp instruction)
 *   kind 2: FP32 fused multiply-add
 * Returns the number of flops the launch performs in *flops.  The caller times
 * the launch (CUDA events) to get a rate.
 */
int jmg_dev_probe(int kind, int blocks, int iters, double* sink, double* flops, void* stream);

/* number of launches of this library's kernels queued since the process
 * started (host-side counter, incremented at every launch). */
long long jmg_dev_launch_count(void);

/*
 * Time limit of every device-side wait (the solves' flag waits and the
 * tensor-core kernels' mbarrier waits), in nanoseconds of %globaltimer; the
 * default is 2 s.  Sets it to `ns` (ns > 0; 0 only queries) and returns the
 * previous value.  Process-wide and read at each launch: change it only while
 * no call of this library is being issued from another thread.
 */
unsigned long long jmg_dev_set_wait_limit_ns(unsigned long long ns);

/*
 * Bounded-wait checks.  Each launches one kernel in a state where one of its
 * device-side waits is never satisfied, so the wait runs out after the current
 * limit and the kernel leaves through its abort path (no trap, no fault):
 *
 * trsv_leaderless: the one-launch forward solve L Y = B (dtype JMG_F64 or
 *   JMG_F32) with every ticket offset by one, so that no CTA takes the leading
 *   role and no block of Y is ever published: every helper's flag wait runs
 *   out.  `sync` holds jmg_workspace_size(JMG_OP_POTRS, n, nrhs, dtype, NULL)
 *   bytes; afterwards sync[0] == JMG_ERR_TIMEOUT and *info == -1 (info may be
 *   NULL).  B is left partly overwritten.
 *
 * syrk_tc_idle_producer: the tensor-core trailing update (arguments as
 *   jmg_dev_syrk_tc) with its copy producer idle: the MMA issuer's wait for the
 *   first stage runs out; afterwards *err != 0 and C is untouched.
 */
int jmg_dev_trsv_leaderless(int n, int nrhs, const void* L, int lda, void* B, int ldb, int dtype,
                            int* sync, int* info, void* stream);
int jmg_dev_syrk_tc_idle_producer(int m, int ncols, int kext, const void* PA, const void* PB,
                                  int ldp, int prec, float* C, int ldc, int* err, void* stream);

/*
 * The block-inverse triangular solves of the mixed path on a caller's FP32
 * factor: (L L^T) X = B in place on B (FP32, n x nrhs, column-major).  The
 * call copies lower(L) and B into `work` (the solves need W's upper triangle
 * and 128-byte aligned leading dimensions), forms the inverses of the 128 x 128
 * diagonal blocks and the chain's coupling blocks, runs the forward and the
 * backward solve and copies X back into B.  work: jmg_dev_sv_workspace(n, nrhs)
 * bytes, 256-byte aligned.  Asynchronous.
 */
size_t jmg_dev_sv_workspace(int n, int nrhs);
int jmg_dev_sv_potrs(int n, int nrhs, const float* L, int lda, float* B, int ldb, void* work,
                     size_t lwork, void* stream);

/*
 * The FP8 quantiser of the mixed factorisation on its own: the FP32 panel
 * L21 (m x kb, column-major, ldw) becomes Q (m x kb e4m3 bytes, row-major, ldq
 * >= kb) with one exponent per 128-row tile t:
 *     e_t = floor(log2(448 / amax_t)) clamped to [-126, 126] (0 when amax_t = 0),
 *     Q[i, c] = e4m3_rn_satfinite(L21[i, c] * 2^e_t)     (round to nearest even).
 * e: ceil(m / 128) int8.  Asynchronous.
 */
int jmg_dev_quant_fp8(int m, int kb, const float* L21, int ldw, void* Q, int ldq, signed char* e,
                      void* stream);

#ifdef __cplusplus
}
#endif

#endif /* JMG_DEV_H */
