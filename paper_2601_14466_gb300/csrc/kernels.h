// kernels.h -- internal launchers of the SPD solver's kernels (not exported).
#pragma once

#include <cuda.h>

#include <algorithm>

#include "common.cuh"

namespace jmg {

// Operand access modes of the tiled GEMM:
//   N: op(A)(i, l) = A[i + l*lda]            (column-major as stored)
//   T: op(A)(i, l) = A[l + i*lda]            (transposed)
//   S: op(A)(i, l) = A[max(i,l) + min(i,l)*lda]  (symmetric, lower stored;
//      i and l are absolute indices of the stored matrix)
enum Mode { MODE_N = 0, MODE_T = 1, MODE_S = 2 };

// Output of the tiled GEMM:
//   OUT_SUB:  C[i + j*ldc] -= acc                 (all tiles of the grid)
//   OUT_SUB_LOWER: same, lower-triangle tiles only and only i >= j written
//   OUT_PART: part[z][i + j*ldc] = acc            (split-K partial sums)
enum Out { OUT_SUB = 0, OUT_SUB_LOWER = 1, OUT_PART = 2 };

// ---- factorisation pieces (T = storage type; FP64 arithmetic in potf2)
int launch_potf2(double* A, int lda, int kb, int koff, int* info, cudaStream_t s);
int launch_potf2(float* A, int lda, int kb, int koff, int* info, cudaStream_t s);

// A21 (m x kb, in place) <- A21 * Lkk^{-T}; arithmetic in T.
int launch_trsm(double* A21, int lda, int m, int kb, const double* Lkk, const int* info,
                cudaStream_t s);
int launch_trsm(float* A21, int lda, int m, int kb, const float* Lkk, const int* info,
                cudaStream_t s);

// C (m x n) -= op(A) (m x k) * op(B) (k x n), T arithmetic.
// For OUT_SUB_LOWER, m == n and the tile grid covers the lower triangle.
// For OUT_PART, `C` is the partial buffer with `splits` slices of ldc*n.
template <typename T>
int launch_gemm(int m, int n, int k, const T* A, int lda, int amode, const T* B, int ldb,
                int bmode, T* C, int ldc, int out, int splits, const int* info, cudaStream_t s);

// Batched small systems (n <= 128): factor every A_b = L_b L_b^T in place
// (info[b], 0-based batch index) and solve (L_b L_b^T) X_b = B_b in place.
template <typename T>
int posv_small_batched(int n, int nrhs, int batch, T* A, int lda, long long sA, T* B, int ldb,
                       long long sB, int* info, cudaStream_t s);

// One-launch blocked solve with the whole factor, in place on B:
// trans == 0: L Y = B;  trans == 1: L^T X = B.  `sync` holds
// trsv_sync_ints(n, nrhs) ints of scratch: sync[0] is the error word (0, or
// JMG_ERR_TIMEOUT once a device-side wait ran out; the forward solve clears it,
// the backward solve keeps it and does nothing if it is set), then tickets,
// finished-block counters and per-block flags.  tkt0 != 0 is a test hook: every
// ticket is offset by tkt0, so no CTA leads and the helpers' bounded waits run
// out (g_wait_ns).
size_t trsv_sync_ints(int n, int nrhs);
template <typename T>
int launch_trsv_persist(int n, int nrhs, const T* L, int lda, T* B, int ldb, int trans, int* sync,
                        int* info, cudaStream_t s, int tkt0 = 0);
// (L L^T) X = B: forward then backward with launch_trsv_persist.
template <typename T>
int solve_llt(int n, int nrhs, const T* L, int lda, T* B, int ldb, int* sync, int* info,
              cudaStream_t s) {
  JMG_TRY(launch_trsv_persist<T>(n, nrhs, L, lda, B, ldb, 0, sync, info, s));
  return launch_trsv_persist<T>(n, nrhs, L, lda, B, ldb, 1, sync, info, s);
}

// ---- mixed-precision helpers
// W (FP32, ldw) <- lower(A) (FP64), lower triangle only; plus shift on the diagonal.
int launch_lower_to_f32(int n, const double* A, int lda, float* W, int ldw, double shift,
                        cudaStream_t s);
// Split FP32 panel L21 (m x kb, ldw) into 16-bit words, written into the
// extended operands PA / PB (row-major, m x kext, ldp) at K offset `koff`:
// for each pair p of the pair table, PA[:, p*kb + c] = word a_p, PB = word b_p.
int launch_split_words(int m, int kb, const float* L21, int ldw, int prec, int words, void* PA,
                       void* PB, int ldp, cudaStream_t s);
int split_pairs(int words);  // number of (a, b) word pairs used for `words`

// ---- refinement helpers
// R = B - A X (A symmetric, lower) in FP64 with split-K partials in `part`
// (splits * n * nrhs doubles), colmax[0..3 nrhs) = ||r||, ||x||, ||b|| per column.
int residual_splits(int n, int nrhs);
int launch_residual(int n, int nrhs, const double* A, int lda, const double* X, int ldx,
                    const double* B, int ldb, double* R, int ldr, double* colmax, double* part,
                    int splits, cudaStream_t s, cudaEvent_t ev0 = nullptr,
                    cudaEvent_t ev1 = nullptr);
// R = B - sum_z part[z] (B == nullptr: R = sum_z part[z]) and the column norms
int launch_resid_reduce(int n, int nrhs, int used, const double* part, const double* X, int ldx,
                        const double* B, int ldb, double* R, int ldr, double* colmax,
                        cudaStream_t s);

// ---- split (Ozaki) product on the BF16 tensor cores (k_ozaki.cu)
size_t oz_a_bytes(int n);             // slices of A
size_t oz_x_bytes(int n, int nrhs);   // slices of X and their exponents
int oz_splits(int n, int nrhs);       // K splits requested
int oz_splits_used(int n, int nrhs);  // K splits the grid ends up with (partials written)
// rowmax: n doubles (written); SA: oz_a_bytes(n)
int oz_prepare_a(int n, const double* A, int lda, double* rowmax, void* SA, cudaStream_t s);
// the slices alone, from row maxima already computed by launch_row_stats
int oz_slice_a(int n, const double* A, int lda, const double* rowmax, void* SA, cudaStream_t s);
// part[z] (z < oz_splits_used) = partial sums of A X; xwork: oz_x_bytes(n, nrhs)
int oz_product(int n, int nrhs, const void* SA, const double* rowmax, const double* X, int ldx,
               void* xwork, double* part, int* err, cudaStream_t s);

// Row sums and row maxima of |A| over full rows of the symmetric A (lower
// stored); either output may be null.
int launch_row_stats(int n, const double* A, int lda, double* rowsum, double* rowmax,
                     cudaStream_t s);
// *out = max_i v[i] (NaN propagates; v >= 0)
int launch_max_reduce(int n, const double* v, double* out, cudaStream_t s);
// ||A||_inf (lower stored) into *out; rowsum: n doubles of scratch.
int launch_norm_inf(int n, const double* A, int lda, double* rowsum, double* out,
                    cudaStream_t s);
// eta_j = colmax_r / (anorm * colmax_x + colmax_b); eta_out[0] = max_j, eta_out[1..] = eta_j
int launch_eta(int nrhs, const double* colmax, const double* anorm, double* eta_out,
               cudaStream_t s);
// D32[:, j] = fp32(R[:, j] / scale_j), scale_j = colmax_r[j] (1 if zero)
int launch_scale_to_f32(int n, int nrhs, const double* R, int ldr, const double* colmax_r,
                        float* D, int ldd, cudaStream_t s);
// X[:, j] += scale_j * D32[:, j]   (X FP64)
int launch_axpy_f32(int n, int nrhs, const float* D, int ldd, const double* colmax_r, double* X,
                    int ldx, cudaStream_t s);
// copy FP64 -> FP64 column-major blocks
int launch_copy2d(int n, int nrhs, const double* src, int lds, double* dst, int ldd,
                  cudaStream_t s);
// clear n doubles
int launch_zero(double* p, size_t n, cudaStream_t s);

// ---- preconditioned CG (FP64, columns independent)
int launch_dot_cols(int n, int nrhs, const double* U, int ldu, const double* V, int ldv,
                    double* out, cudaStream_t s);
int launch_pcg_step(int n, int nrhs, const double* P, const double* Q, const double* rz,
                    const double* pq, double* X, double* R, double* colmax, int* bad,
                    cudaStream_t s);
int launch_pcg_dir(int n, int nrhs, const double* Z, double* P, const double* rz_new,
                   const double* rz_old, cudaStream_t s);
int launch_scale_from_f32(int n, int nrhs, const float* D, int ldd, const double* colmax_r,
                          double* Z, cudaStream_t s);
int launch_diag_max(int n, const double* A, int lda, double* out, cudaStream_t s);

// ---- adjoint (k_grad.cu): G = -(Bb X^T + X Bb^T)/2, full symmetric n x n
int launch_sym_grad(int n, int nrhs, const double* Bb, int ldb, const double* X, int ldx, double* G,
                    int ldg, cudaStream_t s);

// ---- block-inverse solves with the FP32 factor of the mixed path (k_solve.cu)
// Bytes of the per-factorisation images (inverses of the diagonal blocks and the
// chain's coupling matrices) and ints of solve scratch.
size_t sv_image_bytes(int n);
size_t sv_sync_ints(int n, int nrhs);
// Once per factorisation of W (FP32, lower, ldw % 32 == 0, 16-byte aligned):
// mirror the strictly lower blocks into the upper triangle of W and write the
// images into SV (sv_image_bytes(n), 256-byte aligned).
int sv_prepare(int n, float* W, int ldw, float* SV, cudaStream_t s);
// trans == 0: L Y = D; trans == 1: L^T X = D, in place on D (FP32, n x nrhs,
// ldd % 32 == 0).  sync: sv_sync_ints(n, nrhs) ints; sync[0] is the error word
// (cleared by the forward solve, kept by the backward solve).  info: as
// launch_trsv_persist (may be NULL).
int sv_solve(int n, int nrhs, const float* W, int ldw, const float* SV, float* D, int ldd,
             int trans, int* sync, int* info, cudaStream_t s);
inline int sv_solve_llt(int n, int nrhs, const float* W, int ldw, const float* SV, float* D,
                        int ldd, int* sync, int* info, cudaStream_t s) {
  JMG_TRY(sv_solve(n, nrhs, W, ldw, SV, D, ldd, 0, sync, info, s));
  return sv_solve(n, nrhs, W, ldw, SV, D, ldd, 1, sync, info, s);
}

// ---- in-place row-major -> column-major conversion (k_layout.cu)
size_t layout_min_scratch(long long m, long long n, size_t esize);

// k_small.cu: the whole mixed posv for n <= 2048 in one persistent kernel
bool small_path_fits(int n, int nrhs);
size_t small_workspace(int n, int nrhs);
int small_posv(int n, int nrhs, const double* A, int lda, double* B, int ldb, int* info,
               const jmg_options& o, jmg_stats* st, void* work, cudaStream_t s);
int layout_r2c(long long m, long long n, void* A, int dtype, void* work, size_t lwork,
               cudaStream_t s);

// 2D tiled tensor map over a matrix with `inner` contiguous elements per line
// (leading dimension ld_bytes), `outer` lines; box box_inner x box_outer.
int make_tmap_2d(CUtensorMap* map, const void* base, unsigned long long inner,
                 unsigned long long outer, unsigned long long ld_bytes, unsigned box_inner,
                 unsigned box_outer, CUtensorMapDataType dt, CUtensorMapSwizzle sw);

// ---- tensor-core trailing update (k_tc.cu)
// C (m x ncols, lower trapezoid: rows >= columns) -= PA PB^T, PA/PB: m x kext
// row-major 16-bit words; ncols <= m.
// max_ctas > 0 caps the persistent grid (to leave SMs free for concurrent work).
// hold != 0 is a test hook: the TMA producer stays idle, so the kernel's first
// bounded wait runs out (g_wait_ns) and it returns through its abort path.
// kchunk (a multiple of 64 dividing kext; 0 = kext): K goes to the tensor-core
// accumulator in chunks of kchunk and the chunks add up in FP32 registers.
int launch_syrk_tc(int m, int ncols, int kext, const void* PA, const void* PB, int ldp, int prec,
                   float* C, int ldc, int* err, cudaStream_t s, int max_ctas = 0, int hold = 0,
                   int kchunk = 0);
// FP8 e4m3 variant: Q (m x kext bytes, row-major, ldq); K goes in chunks of 128,
// chunk c with its own exponents e + c * lde (one per 128-row tile; lde = 0: the
// same exponents for every chunk):
//     C -= sum_c 2^-(e_c[ti] + e_c[tj]) Q_ti,c Q_tj,c^T
int launch_syrk_fp8(int m, int ncols, int kext, const void* Q, int ldq, const signed char* e,
                    int lde, float* C, int ldc, int* err, cudaStream_t s, int max_ctas = 0);
// Quantise the FP32 panel L21 (m x kb, ldw) to e4m3 with one power-of-two scale
// per 128-row tile: e = floor(log2(448 / amax)) clamped to [-126, 126] (0 for an
// all-zero tile), Q = rn_satfinite(x * 2^e), row-major m x kb (ldq bytes).
int launch_quant_fp8(int m, int kb, const float* L21, int ldw, void* Q, int ldq, signed char* e,
                     cudaStream_t s);

}  // namespace jmg
