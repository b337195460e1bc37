// k_dense.cu -- CUDA-core kernels of the blocked Cholesky solver (sm_103a):
// diagonal-block factorisation, panel TRSM, tiled GEMM / SYRK / SYMM, blocked
// triangular solves, FP64 residual and the small helpers of the refinement loop.
//
// Paper: "Software design" -- potrs solves A x = b for SPD A by a Cholesky
// factorisation followed by the triangular solves.  The paper delegates both to
// cuSOLVERMp; the blocking below is the textbook right-looking scheme (factor
// the diagonal block, solve the panel below it, update the trailing matrix).
#include <map>
#include <mutex>
#include <utility>

#include "kernels.h"

namespace jmg {

long long g_launches = 0;
unsigned long long g_wait_ns = 2000000000ull;

int ensure_smem_raw(const void* func, int bytes) {
  int dev = 0;
  JMG_CUDA(cudaGetDevice(&dev));
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> raised;
  std::lock_guard<std::mutex> lock(mu);
  const auto key = std::make_pair(func, dev);
  const auto it = raised.find(key);
  if (it != raised.end() && it->second >= bytes) return JMG_OK;
  JMG_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  raised[key] = bytes;
  return JMG_OK;
}

// ============================================================================
// Diagonal-block factorisation L_kk L_kk^T = A_kk (kb <= 128), in place, as a
// blocked right-looking Cholesky over 32-column sub-blocks, one CTA:
//
//  1. the 32 x 32 diagonal sub-block is factored in FP64 whatever the storage
//     type T (double for the plain path, float for the FP32 working matrix of
//     the mixed path).  Its 528 lower elements sit in shared memory as FP64;
//     step j applies a_rc -= a_rj * a_cj / a_jj (= l_rj * l_cj) to every
//     element with c > j, handing the trailing triangle's elements (a range of
//     the packed column-major order) to consecutive threads so that FP64 work
//     is issued by full warps only; each column costs one barrier.  The owner
//     of a_(j+1)(j+1) forms 1 / a_(j+1)(j+1) in step j, the only operation on
//     the serial chain besides the updates (exact for the plain path; an FP32
//     seed plus one step of Newton's method for the mixed path, whose output is
//     rounded to FP32 anyway); sqrt(a_jj) and its reciprocal follow after the
//     last column;
//  2. the rows of the block below it solve x L_qq^T = a (triangular solve, one
//     thread per row, in T);
//  3. the rest of the block takes the symmetric rank-32 update C -= X X^T (in
//     T, 4 x 4 register tiles).
//
// In the mixed path only step 1 runs in FP64: steps 2 and 3 are the panel's
// share of the trailing update, which the tensor-core path rounds further
// anyway, and FP64 runs at 1/64 of the FP32 rate on this GPU.  A pivot that is
// not > 0 (or NaN) records info = koff + j + 1; the columns before it are
// written, the rest keep their input.
// ============================================================================
namespace pdiag {
constexpr int KB = 128;                  // largest diagonal block
constexpr int BS = 32;                   // FP64 sub-block
constexpr int TH = 256;
constexpr int LD = KB + 4;               // shared leading dimension: 16-byte aligned columns
constexpr int NEL = BS * (BS + 1) / 2;   // lower elements of a sub-block
static_assert(TH == 256, "the FP64 step's warp roles and its named barrier (224 threads) assume 8 warps");

// 1/d to about 44 bits for positive normal d with |log2 d| <= 100: the leading
// bits of d as an FP32 number (exponent rebiased, mantissa truncated, with
// integer operations that stay off the FP64 pipe, where a conversion costs as
// much as an FMA), rcp.approx on it, the FP32 result widened the same way, and
// one step of Newton's method for 1/d in FP64.
JMG_DEV double rcp_seeded(double d) {
  const int hi = __double2hiint(d);
  const unsigned lo = (unsigned)__double2loint(d);
  const int fb = ((((hi >> 20) & 0x7ff) - 896) << 23) | ((hi & 0xfffff) << 3) | (int)(lo >> 29);
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(__int_as_float(fb)));
  const int yb = __float_as_int(y);
  const double y0 =
      __hiloint2double(((((yb >> 23) & 0xff) + 896) << 20) | ((yb & 0x7fffff) >> 3), (yb & 7) << 29);
  return fma(y0, fma(-d, y0, 1.0), y0);
}

// 1 / d for the updates of step j (exact division for the plain path; for the
// mixed path the seeded Newton step above, whose result is rounded to FP32
// anyway).  Only this reciprocal sits on the serial chain of the steps; sqrt(d)
// is taken after the last step.  *bad is set when d is not positive (or NaN);
// the result is then finite garbage or non-finite, never a trap.
JMG_DEV double pivot_w(double d, bool exact, bool* bad) {
  const int hi = __double2hiint(d), e = (hi >> 20) & 0x7ff;
  if (!exact && hi >= 0 && e >= 1023 - 100 && e <= 1023 + 100) return rcp_seeded(d);
  *bad = !(d > 0.0);
  return 1.0 / d;
}

template <typename T>
JMG_DEV void load4(const T* p, T (&v)[4]);
template <>
JMG_DEV void load4<float>(const float* p, float (&v)[4]) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
}
template <>
JMG_DEV void load4<double>(const double* p, double (&v)[4]) {
  const double2 q0 = reinterpret_cast<const double2*>(p)[0];
  const double2 q1 = reinterpret_cast<const double2*>(p)[1];
  v[0] = q0.x, v[1] = q0.y, v[2] = q1.x, v[3] = q1.y;
}
}  // namespace pdiag

template <typename T>
JMG_DEV void potrf_diag_body(T* __restrict__ A, int lda, int kb, int koff,
                             int* __restrict__ info) {
  using namespace pdiag;
  extern __shared__ __align__(16) unsigned char sm_diag[];
  T* sa = reinterpret_cast<T*>(sm_diag);  // kb columns, LD apart: sa[c * LD + r] = a_rc
  __shared__ double s_l[BS], s_il[BS], s_u[2][BS];
  __shared__ T s_rinv[BS];
  __shared__ int fail;
  constexpr bool kExact = sizeof(T) == 8;
  const int t = threadIdx.x;
  if (t == 0) fail = *(volatile int*)info;  // one read, so every thread takes the same exit
  __syncthreads();
  if (fail != 0) return;  // an earlier block already failed
  for (int base = 0; base < kb * kb; base += TH * 16) {  // 16 independent loads per thread
    T v[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int idx = base + t + TH * q;
      const int i = idx % kb, j = idx / kb;
      v[q] = (idx < kb * kb && i >= j) ? A[(size_t)j * lda + i] : T(0);
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int idx = base + t + TH * q;
      if (idx < kb * kb) sa[(idx / kb) * LD + idx % kb] = v[q];
    }
  }
  // packed column-major lower order of a sub-block: element e <-> (row, column)
  __shared__ unsigned short s_rc[NEL];
  __shared__ double s64[BS * (BS + 1)];  // the FP64 sub-block: s64[c * (BS+1) + r]
  for (int e = t; e < NEL; e += TH) {
    int r = e, c = 0;
    while (r >= BS - c) r -= BS - c++;
    s_rc[e] = (unsigned short)((c << 8) | (c + r));
  }
  __syncthreads();

  for (int p = 0; p < kb; p += BS) {
    const int bs = min(BS, kb - p);
    // ---- 1. FP64 factor of the sub-block.  Step j updates every element
    // (r, c), c > j, of the trailing triangle: a_rc -= a_rj u_c with
    // u_c = a_cj w_j, w_j = 1/a_jj.  A warp-wide FP64 instruction occupies its
    // SM sub-partition's FP64 pipe for ~64 cycles whatever the active lanes,
    // and the pivots form a serial chain, so the work is split by warp and
    // the chain runs one column ahead of the rest:
    //  * warp 0 (the chain) keeps column j and w_j in registers (one lane per
    //    row); in step j it forms u, hands it to the trailing warps (named
    //    barrier U), finishes column j+1 (its update by column j) and takes
    //    pivot j+1 on every lane;
    //  * warps 1-3 and 5-7 (trailing) take u_j and update column j+2 first,
    //    release it (named barrier Y: the chain's input of step j+1), then
    //    the columns j+3.. (packed indices on consecutive threads);
    //  * warp 4, which shares warp 0's FP64 pipe, stays out.
    // The last step has no work, so both sides run steps 0..bs-2.  Each
    // barrier is passed the same number of times on both sides (U: bs-1,
    // Y: bs-2), and every arrival waits, through the other barrier, for the
    // other side to have passed the previous instance, so no instance can
    // count an arrival meant for the next.  Nothing leaves the loop early: a
    // pivot that is not positive is recorded (the first one wins) and the
    // columns from it on are dropped after the loop.  u alternates between
    // two buffers; the chain writes buffer j&1 only after passing Y of step
    // j-1, i.e. after the trailing warps have finished step j-2.
    for (int e = t; e < NEL; e += TH) {
      const int rc = s_rc[e], c = rc >> 8, r = rc & 255;
      if (r < bs) s64[c * (BS + 1) + r] = (double)sa[(p + c) * LD + p + r];
    }
    __syncthreads();
    const int warp = t >> 5, lane = t & 31;
    if (warp == 0) {
      const bool row = lane < bs;
      double colj = row ? s64[lane] : 0.0;  // column 0
      bool bad = false;
      double w = pivot_w(__shfl_sync(0xffffffffu, colj, 0), kExact, &bad);
      int fj = bad ? 0 : -1;  // first failing column of the sub-block
      for (int j = 0; j + 1 < bs; ++j) {
        const bool own = row && lane > j;  // rows below the diagonal of column j
        __syncwarp();
        if (j > 0) asm volatile("bar.sync 2, 224;" ::: "memory");  // column j+1 done to j-1
        double nxt = own ? s64[(j + 1) * (BS + 1) + lane] : 0.0;
        const double u = own ? colj * w : 0.0;
        if (own) s_u[j & 1][lane] = u;
        __syncwarp();
        asm volatile("bar.arrive 1, 224;" ::: "memory");
        nxt = fma(-colj, __shfl_sync(0xffffffffu, u, j + 1), nxt);
        if (own) s64[(j + 1) * (BS + 1) + lane] = nxt;
        bad = false;
        const double wn = pivot_w(__shfl_sync(0xffffffffu, nxt, j + 1), kExact, &bad);
        if (bad && fj < 0) fj = j + 1;
        colj = nxt;
        w = wn;
      }
      if (lane == 0 && fj >= 0) fail = p + fj + 1;
    } else if (warp != 4) {
      const int tq = warp < 4 ? t - 32 : t - 64;  // index among the trailing warps
      for (int j = 0; j + 1 < bs; ++j) {
        __syncwarp();
        asm volatile("bar.sync 1, 224;" ::: "memory");  // u_j and column j in place
        const double* cj = &s64[j * (BS + 1)];
        const double* uj = s_u[j & 1];
        if (j + 2 < bs) {
          if (tq >= j + 2 && tq < bs) {
            double* c2 = &s64[(j + 2) * (BS + 1)];
            c2[tq] = fma(-cj[tq], uj[j + 2], c2[tq]);
          }
          __syncwarp();
          asm volatile("bar.arrive 2, 224;" ::: "memory");
        }
        // first packed index of column j+3: sum of the column lengths before it
        const int c3 = j + 3;
        const int e3 = c3 >= BS ? NEL : c3 * BS - c3 * (c3 - 1) / 2;
        for (int e = e3 + tq; e < NEL; e += TH - 64) {
          const int rc = s_rc[e], c = rc >> 8, r = rc & 255;
          if (r >= bs) continue;
          s64[c * (BS + 1) + r] = fma(-cj[r], uj[c], s64[c * (BS + 1) + r]);
        }
      }
    }
    __syncthreads();
    const int jdone = fail ? fail - 1 - p : bs;  // columns of the sub-block that are final
    // L of the sub-block: l_cc = sqrt(a_cc), l_rc = a_rc / l_cc
    if (t < jdone) {
      const int c = t;
      const double a = s64[c * (BS + 1) + c];
      double l, il;
      if (kExact || a < 1e-30) {
        l = sqrt(a);
        il = 1.0 / l;
      } else {
        const double y0 = (double)rsqrtf((float)a);
        il = y0 * fma(-0.5 * a, y0 * y0, 1.5);  // one Newton step for d^{-1/2}
        l = a * il;
      }
      s_l[c] = l;
      s_il[c] = il;
    }
    __syncthreads();
    for (int e = t; e < NEL; e += TH) {
      const int rc = s_rc[e], c = rc >> 8, r = rc & 255;
      if (r < bs && c < jdone) {
        const T v = (T)(r == c ? s_l[c] : s64[c * (BS + 1) + r] * s_il[c]);
        sa[(p + c) * LD + p + r] = v;
        A[(size_t)(p + c) * lda + p + r] = v;
        if (r == c) s_rinv[c] = kExact ? (T)s_il[c] : (T)__frcp_rn((float)v);
      }
    }
    if (jdone < bs) break;  // (uniform: every thread read the same flag after the barrier)
    const int mr = kb - p - BS;
    if (mr <= 0) break;
    __syncthreads();

    // ---- 2. rows below the sub-block: x L_qq^T = a, one thread per row
    if (t < mr) {
      const int r = p + BS + t;
      T x[BS];
#pragma unroll
      for (int c = 0; c < BS; ++c) x[c] = sa[(p + c) * LD + r];
#pragma unroll
      for (int j = 0; j < BS; ++j) {
        x[j] *= s_rinv[j];
#pragma unroll
        for (int l = j + 1; l < BS; ++l) x[l] = fma(-x[j], sa[(p + j) * LD + p + l], x[l]);
      }
#pragma unroll
      for (int c = 0; c < BS; ++c) {
        sa[(p + c) * LD + r] = x[c];
        A[(size_t)(p + c) * lda + r] = x[c];
      }
    }
    __syncthreads();

    // ---- 3. trailing part of the block: C -= X X^T on 4 x 4 tiles (lower)
    {
      const int q0 = p + BS, nt = (mr + 3) / 4, ntiles = nt * (nt + 1) / 2;
      for (int tile = t; tile < ntiles; tile += TH) {
        int I = (int)((sqrtf(8.0f * (float)tile + 1.0f) - 1.0f) * 0.5f);
        while (I * (I + 1) / 2 > tile) --I;
        while ((I + 1) * (I + 2) / 2 <= tile) ++I;
        const int J = tile - I * (I + 1) / 2;
        const int r0 = q0 + 4 * I, c0 = q0 + 4 * J;
        T acc[4][4] = {};
#pragma unroll 8
        for (int k = 0; k < BS; ++k) {
          T xr[4], xc[4];
          load4(&sa[(p + k) * LD + r0], xr);  // rows past kb read padding, never stored
          load4(&sa[(p + k) * LD + c0], xc);
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) acc[i][jj] = fma(xr[i], xc[jj], acc[i][jj]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) {
            const int r = r0 + i, c = c0 + jj;
            if (r < kb && r >= c) sa[c * LD + r] -= acc[i][jj];
          }
      }
    }
    __syncthreads();
  }
  if (t == 0 && fail) atomicCAS(info, 0, koff + fail);
}

template <typename T>
__global__ void __launch_bounds__(pdiag::TH) k_potrf_diag(T* __restrict__ A, int lda, int kb,
                                                          int koff, int* __restrict__ info) {
  potrf_diag_body<T>(A, lda, kb, koff, info);
}

// Batched: CTA b factors the n x n system A + b * sA (n <= 128) with info[b].
template <typename T>
__global__ void __launch_bounds__(pdiag::TH) k_potrf_diag_batched(T* __restrict__ A, int lda,
                                                                  long long sA, int n,
                                                                  int* __restrict__ info) {
  potrf_diag_body<T>(A + (size_t)blockIdx.x * sA, lda, n, 0, info + blockIdx.x);
}

// Batched solve with the factors of k_potrf_diag_batched: CTA b solves
// (L_b L_b^T) X_b = B_b in place on B + b * sB, 64 right-hand sides per pass,
// one thread per right-hand side: forward then back substitution against L_b in
// shared memory (FP64 or FP32 as stored).  Systems with info[b] != 0 are left
// alone.
namespace pbat {
constexpr int TH = 64;
}
template <typename T>
__global__ void __launch_bounds__(pbat::TH) k_potrs_small(int n, int nrhs, const T* __restrict__ L,
                                                          int lda, long long sA, T* __restrict__ B,
                                                          int ldb, long long sB,
                                                          const int* __restrict__ info) {
  using pbat::TH;
  const int b = blockIdx.x;
  if (info[b] != 0) return;
  extern __shared__ __align__(16) unsigned char sm_small[];
  T* Ls = reinterpret_cast<T*>(sm_small);  // Ls[c * (n + 1) + r] = L(r, c)
  T* Xs = Ls + (size_t)n * (n + 1);        // Xs[r * (TH + 1) + t] = x_r of column t
  const int ldl = n + 1, ldx = TH + 1;
  const T* Lb = L + (size_t)b * sA;
  T* Bb = B + (size_t)b * sB;
  const int t = threadIdx.x;
  for (int idx = t; idx < n * n; idx += TH) {
    const int r = idx % n, c = idx / n;
    if (r >= c) Ls[c * ldl + r] = Lb[(size_t)c * lda + r];
  }
  for (int c0 = 0; c0 < nrhs; c0 += TH) {
    const int nc = min(TH, nrhs - c0);
    __syncthreads();  // L is in place; the previous pass is done with Xs
    for (int idx = t; idx < n * nc; idx += TH) {  // coalesced down the columns
      const int r = idx % n, c = idx / n;
      Xs[r * ldx + c] = Bb[(size_t)(c0 + c) * ldb + r];
    }
    __syncthreads();
    if (t < nc) {
      for (int i = 0; i < n; ++i) {  // L y = b
        const T y = Xs[i * ldx + t] / Ls[i * ldl + i];
        Xs[i * ldx + t] = y;
        for (int k = i + 1; k < n; ++k) Xs[k * ldx + t] -= Ls[i * ldl + k] * y;
      }
      for (int i = n - 1; i >= 0; --i) {  // L^T x = y
        const T x = Xs[i * ldx + t] / Ls[i * ldl + i];
        Xs[i * ldx + t] = x;
        for (int k = 0; k < i; ++k) Xs[k * ldx + t] -= Ls[k * ldl + i] * x;
      }
    }
    __syncthreads();
    for (int idx = t; idx < n * nc; idx += TH) {
      const int r = idx % n, c = idx / n;
      Bb[(size_t)(c0 + c) * ldb + r] = Xs[r * ldx + c];
    }
  }
}

template <typename T>
int posv_small_batched(int n, int nrhs, int batch, T* A, int lda, long long sA, T* B, int ldb,
                       long long sB, int* info, cudaStream_t s) {
  if (n > pdiag::KB) return JMG_ERR_UNSUPPORTED;
  JMG_CUDA(cudaMemsetAsync(info, 0, sizeof(int) * (size_t)batch, s));
  if (n == 0 || batch == 0) return JMG_OK;
  {
    auto k = k_potrf_diag_batched<T>;
    JMG_TRY(ensure_smem(k, (int)(pdiag::KB * pdiag::LD * sizeof(T))));
    k<<<batch, pdiag::TH, (size_t)n * pdiag::LD * sizeof(T), s>>>(A, lda, sA, n, info);
    JMG_TRY(launched());
  }
  if (nrhs == 0) return JMG_OK;
  auto k = k_potrs_small<T>;
  const size_t smem = sizeof(T) * ((size_t)n * (n + 1) + (size_t)n * (pbat::TH + 1));
  JMG_TRY(ensure_smem(k, (int)smem));
  k<<<batch, pbat::TH, smem, s>>>(n, nrhs, A, lda, sA, B, ldb, sB, info);
  return launched();
}
template int posv_small_batched<double>(int, int, int, double*, int, long long, double*, int,
                                        long long, int*, cudaStream_t);
template int posv_small_batched<float>(int, int, int, float*, int, long long, float*, int,
                                       long long, int*, cudaStream_t);

template <typename T>
static int potf2_impl(T* A, int lda, int kb, int koff, int* info, cudaStream_t s) {
  if (kb > pdiag::KB) return JMG_ERR_UNSUPPORTED;
  const size_t smem = (size_t)kb * pdiag::LD * sizeof(T);
  auto k = k_potrf_diag<T>;
  JMG_TRY(ensure_smem(k, (int)(pdiag::KB * pdiag::LD * sizeof(T))));
  k<<<1, pdiag::TH, smem, s>>>(A, lda, kb, koff, info);
  return launched();
}
int launch_potf2(double* A, int lda, int kb, int koff, int* info, cudaStream_t s) {
  return potf2_impl(A, lda, kb, koff, info, s);
}
int launch_potf2(float* A, int lda, int kb, int koff, int* info, cudaStream_t s) {
  return potf2_impl(A, lda, kb, koff, info, s);
}

// ============================================================================
// Panel TRSM: A21 (m x kb) <- A21 * Lkk^{-T}, in place.  Each CTA owns BR rows;
// row r of the result solves x_r Lkk^T = a_r by forward substitution over the
// columns j (x_rj = a_rj / L_jj, then a_rl -= x_rj L_lj for l > j).  Lkk sits in
// shared memory; threads are (row, column-group) pairs.
// ============================================================================
template <typename T, int BR>
__global__ void __launch_bounds__(256) k_trsm(T* __restrict__ A21, int lda, int m, int kb,
                                              const T* __restrict__ Lkk,
                                              const int* __restrict__ info) {
  if (*(volatile const int*)info != 0) return;
  extern __shared__ __align__(16) unsigned char sm_trsm[];
  T* Ls = reinterpret_cast<T*>(sm_trsm);  // kb x (kb+1), column-major
  const int ldl = kb + 1;
  T* Xs = Ls + (size_t)kb * ldl;  // kb columns x (BR+1)
  const int ldx = BR + 1;
  const int t = threadIdx.x;
  const int r0 = blockIdx.x * BR;
  for (int base = 0; base < kb * kb; base += 256 * 16) {  // 16 independent loads per thread
    T v[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int idx = base + t + 256 * q;
      const int i = idx % kb, j = idx / kb;
      v[q] = (idx < kb * kb && i >= j) ? Lkk[(size_t)j * lda + i] : T(0);
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int idx = base + t + 256 * q;
      if (idx < kb * kb) Ls[(idx / kb) * ldl + idx % kb] = v[q];
    }
  }
  for (int base = 0; base < BR * kb; base += 256 * 16) {
    T v[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int idx = base + t + 256 * q;
      const int i = idx % BR, j = idx / BR;
      v[q] = (idx < BR * kb && r0 + i < m) ? A21[(size_t)j * lda + r0 + i] : T(0);
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int idx = base + t + 256 * q;
      if (idx < BR * kb) Xs[(idx / BR) * ldx + idx % BR] = v[q];
    }
  }
  __syncthreads();
  constexpr int G = 256 / BR;
  const int r = t % BR, g = t / BR;
  for (int j = 0; j < kb; ++j) {
    if (g == 0) Xs[j * ldx + r] = Xs[j * ldx + r] / Ls[j * ldl + j];
    __syncthreads();
    const T xrj = Xs[j * ldx + r];
    for (int l = j + 1 + g; l < kb; l += G) Xs[l * ldx + r] -= xrj * Ls[j * ldl + l];
    __syncthreads();
  }
  for (int idx = t; idx < BR * kb; idx += blockDim.x) {
    int i = idx % BR, j = idx / BR;
    if (r0 + i < m) A21[(size_t)j * lda + r0 + i] = Xs[j * ldx + i];
  }
}

template <typename T, int BR>
static int trsm_impl(T* A21, int lda, int m, int kb, const T* Lkk, const int* info,
                     cudaStream_t s) {
  if (m <= 0) return JMG_OK;
  size_t smem = ((size_t)kb * (kb + 1) + (size_t)kb * (BR + 1)) * sizeof(T);
  auto k = k_trsm<T, BR>;
  JMG_TRY(ensure_smem(k, (int)smem));
  k<<<cdiv(m, BR), 256, smem, s>>>(A21, lda, m, kb, Lkk, info);
  return launched();
}
int launch_trsm(double* A21, int lda, int m, int kb, const double* Lkk, const int* info,
                cudaStream_t s) {
  return trsm_impl<double, 32>(A21, lda, m, kb, Lkk, info, s);
}
// FP32 panel TRSM of the mixed path (kb == KB): row r of the panel solves
// x Lkk^T = a by forward substitution, four threads per row (lanes 4r' .. 4r'+3
// of a warp), each owning 8 of every 32 columns.  Columns go in 32-wide chunks:
// chunk J first subtracts the finished chunks (x_k L_ck for k < 32J, an
// independent FMA per column: the bulk of the work, spread over the four
// threads), then solves its diagonal 32 x 32 block (x_k = a_k / L_kk by the
// owner, broadcast to the row's other three lanes by a shuffle, a_c -= x_k L_ck).
// The 64-row tile of the panel and L_kk (transposed, Lt[k][c] = L[c][k]) sit in
// shared memory; global traffic is coalesced down the columns.
namespace ptrsm {
constexpr int RB = 64, TH = 256, LDX = RB + 1;
}

template <int KB>
__global__ void __launch_bounds__(ptrsm::TH, 1) k_trsm_rows(float* __restrict__ A21, int lda, int m,
                                                        const float* __restrict__ Lkk,
                                                        const int* __restrict__ info) {
  using namespace ptrsm;
  if (*(volatile const int*)info != 0) return;
  extern __shared__ __align__(16) float sm_trows[];
  float(*Lt)[KB] = reinterpret_cast<float(*)[KB]>(sm_trows);            // KB x KB
  float(*Xt)[LDX] = reinterpret_cast<float(*)[LDX]>(sm_trows + KB * KB);  // KB x RB (column-major tile)
  float* rinv = sm_trows + KB * KB + KB * LDX;
  const int t = threadIdx.x;
  for (int base = 0; base < KB * KB; base += TH * 16) {  // 16 independent loads per thread
    float v[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int idx = base + t + TH * q;
      const int c = idx % KB, k = idx / KB;  // column k of L, row c
      v[q] = (idx < KB * KB && c >= k) ? Lkk[(size_t)k * lda + c] : 0.0f;
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int idx = base + t + TH * q;
      if (idx < KB * KB) Lt[idx / KB][idx % KB] = v[q];
    }
  }
  __syncthreads();  // Lt complete before its diagonal is read
  if (t < KB) rinv[t] = 1.0f / Lt[t][t];
  const int rl = t / 4, g = t % 4, lane = t % 32;
  // L_kk stays in shared memory; the CTA takes 64-row tiles in turn
  for (int r0 = blockIdx.x * RB; r0 < m; r0 += gridDim.x * RB) {
  __syncthreads();  // Lt, rinv ready; the previous tile's Xt is stored
  for (int base = 0; base < KB * RB; base += TH * 16) {
    float v[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int idx = base + t + TH * q;
      const int r = idx % RB, c = idx / RB;
      v[q] = (idx < KB * RB && r0 + r < m) ? A21[(size_t)c * lda + r0 + r] : 0.0f;
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int idx = base + t + TH * q;
      if (idx < KB * RB) Xt[idx / RB][idx % RB] = v[q];
    }
  }
  __syncthreads();
#pragma unroll 1
  for (int J = 0; J < KB / 32; ++J) {
    const int j0 = J * 32, cb = j0 + 8 * g;  // this thread's 8 columns
    float x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = Xt[cb + i][rl];
    // the finished chunks
#pragma unroll 4
    for (int k = 0; k < j0; ++k) {
      const float xk = Xt[k][rl];
      const float4 l0 = *reinterpret_cast<const float4*>(&Lt[k][cb]);
      const float4 l1 = *reinterpret_cast<const float4*>(&Lt[k][cb + 4]);
      x[0] = fmaf(-xk, l0.x, x[0]);
      x[1] = fmaf(-xk, l0.y, x[1]);
      x[2] = fmaf(-xk, l0.z, x[2]);
      x[3] = fmaf(-xk, l0.w, x[3]);
      x[4] = fmaf(-xk, l1.x, x[4]);
      x[5] = fmaf(-xk, l1.y, x[5]);
      x[6] = fmaf(-xk, l1.z, x[6]);
      x[7] = fmaf(-xk, l1.w, x[7]);
    }
    // the diagonal block of the chunk
#pragma unroll
    for (int kk = 0; kk < 32; ++kk) {
      const int k = j0 + kk, go = kk / 8, io = kk % 8;
      if (g == go) x[io] *= rinv[k];
      const float xk = __shfl_sync(0xffffffffu, x[io], (lane & ~3) | go);
      const float4 l0 = *reinterpret_cast<const float4*>(&Lt[k][cb]);
      const float4 l1 = *reinterpret_cast<const float4*>(&Lt[k][cb + 4]);
      const float l[8] = {l0.x, l0.y, l0.z, l0.w, l1.x, l1.y, l1.z, l1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (8 * g + i > kk) x[i] = fmaf(-xk, l[i], x[i]);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) Xt[cb + i][rl] = x[i];
    __syncwarp();  // the row's four lanes read these in the next chunks
  }
  __syncthreads();
  for (int idx = t; idx < KB * RB; idx += TH) {
    const int r = idx % RB, c = idx / RB;
    if (r0 + r < m) A21[(size_t)c * lda + r0 + r] = Xt[c][r];
  }
  }
}

int launch_trsm(float* A21, int lda, int m, int kb, const float* Lkk, const int* info,
                cudaStream_t s) {
  if (m <= 0) return JMG_OK;
  if (kb == 128 || kb == 64) {
    auto k = (kb == 128) ? k_trsm_rows<128> : k_trsm_rows<64>;
    const size_t smem = sizeof(float) * ((size_t)kb * kb + (size_t)kb * ptrsm::LDX + kb);
    JMG_TRY(ensure_smem(k, (int)smem));
    int dev = 0, nsm = 152, per_sm = 1;
    JMG_CUDA(cudaGetDevice(&dev));
    JMG_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    JMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, ptrsm::TH, smem));
    const int grid = std::max(1, std::min(cdiv(m, ptrsm::RB), std::max(per_sm, 1) * nsm));
    k<<<grid, ptrsm::TH, smem, s>>>(A21, lda, m, Lkk, info);
    return launched();
  }
  return trsm_impl<float, 64>(A21, lda, m, kb, Lkk, info, s);
}

// ============================================================================
// Tiled GEMM on the CUDA cores: C -= op(A) op(B) with 64 x BN output tiles,
// BK = 16, 256 threads, each thread a 4 x (BN/16) register tile.  Rows of a
// thread are tx + 16 q and columns ty + 16 q' so that shared-memory reads are
// conflict-free and global stores coalesce along a column.
// ============================================================================
constexpr int GBM = 64, GBK = 16;

template <typename T, int AMODE>
JMG_DEV T load_a(const T* __restrict__ A, int lda, int i, int l) {
  if (AMODE == MODE_N) return A[(size_t)l * lda + i];
  if (AMODE == MODE_T) return A[(size_t)i * lda + l];
  return (i >= l) ? A[(size_t)l * lda + i] : A[(size_t)i * lda + l];
}

template <typename T, int BN, int AMODE, int BMODE, int OUT>
__global__ void __launch_bounds__(256) k_gemm(int m, int n, int k, const T* __restrict__ A, int lda,
                                              const T* __restrict__ B, int ldb, T* __restrict__ C,
                                              int ldc, int kchunk, const int* __restrict__ info) {
  if (info && *(volatile const int*)info != 0) return;
  constexpr int TN = BN / 16;
  __shared__ T As[GBK][GBM + 1];
  __shared__ T Bs[GBK][BN + 1];
  int ti, tj;
  if (OUT == OUT_SUB_LOWER) {
    tri_index(blockIdx.x, ti, tj);
  } else {
    ti = blockIdx.x;
    tj = blockIdx.y;
  }
  const int i0 = ti * GBM, j0 = tj * BN;
  const int kbeg = (OUT == OUT_PART) ? blockIdx.z * kchunk : 0;
  const int kend = (OUT == OUT_PART) ? min(k, kbeg + kchunk) : k;
  const int t = threadIdx.x, tx = t % 16, ty = t / 16;
  T acc[4][TN];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int p = 0; p < TN; ++p) acc[q][p] = T(0);

  for (int l0 = kbeg; l0 < kend; l0 += GBK) {
    // ---- A tile: GBM x GBK
    // coalesce along the stored column: rows for N (and S tiles that reach the
    // lower triangle), k for T (and S tiles wholly above the diagonal)
    const bool a_rowfast = (AMODE == MODE_N) || (AMODE == MODE_S && !(i0 + GBM - 1 < l0));
#pragma unroll
    for (int q = 0; q < (GBM * GBK) / 256; ++q) {
      int idx = t + 256 * q;
      int ii, ll;
      if (a_rowfast) {
        ii = idx % GBM;
        ll = idx / GBM;
      } else {
        ll = idx % GBK;
        ii = idx / GBK;
      }
      int gi = i0 + ii, gl = l0 + ll;
      As[ll][ii] = (gi < m && gl < kend) ? load_a<T, AMODE>(A, lda, gi, gl) : T(0);
    }
    // ---- B tile: GBK x BN
#pragma unroll
    for (int q = 0; q < (GBK * BN + 255) / 256; ++q) {
      int idx = t + 256 * q;
      if (idx < GBK * BN) {
        int ll, jj;
        if (BMODE == MODE_N) {
          ll = idx % GBK;
          jj = idx / GBK;
        } else {
          jj = idx % BN;
          ll = idx / BN;
        }
        int gl = l0 + ll, gj = j0 + jj;
        T v = T(0);
        if (gl < kend && gj < n)
          v = (BMODE == MODE_N) ? B[(size_t)gj * ldb + gl] : B[(size_t)gl * ldb + gj];
        Bs[ll][jj] = v;
      }
    }
    __syncthreads();
#pragma unroll
    for (int l = 0; l < GBK; ++l) {
      T a[4], b[TN];
#pragma unroll
      for (int q = 0; q < 4; ++q) a[q] = As[l][tx + 16 * q];
#pragma unroll
      for (int p = 0; p < TN; ++p) b[p] = Bs[l][ty + 16 * p];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int p = 0; p < TN; ++p) acc[q][p] = fma(a[q], b[p], acc[q][p]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    int gi = i0 + tx + 16 * q;
    if (gi >= m) continue;
#pragma unroll
    for (int p = 0; p < TN; ++p) {
      int gj = j0 + ty + 16 * p;
      if (gj >= n) continue;
      if (OUT == OUT_PART) {
        C[(size_t)blockIdx.z * ldc * n + (size_t)gj * ldc + gi] = acc[q][p];
      } else {
        if (OUT == OUT_SUB_LOWER && gi < gj) continue;
        C[(size_t)gj * ldc + gi] -= acc[q][p];
      }
    }
  }
}

template <typename T, int BN, int AMODE, int BMODE, int OUT>
static int gemm_launch4(int m, int n, int k, const T* A, int lda, const T* B, int ldb, T* C,
                        int ldc, int splits, const int* info, cudaStream_t s) {
  dim3 grid;
  int kchunk = k;
  if (OUT == OUT_SUB_LOWER) {
    long long tiles = tri_tiles(cdiv(m, GBM));
    grid = dim3((unsigned)tiles, 1, 1);
  } else {
    grid = dim3(cdiv(m, GBM), cdiv(n, BN), 1);
    if (OUT == OUT_PART) {
      kchunk = (int)round_up((size_t)cdiv(k, splits), GBK);
      grid.z = cdiv(k, kchunk);
    }
  }
  k_gemm<T, BN, AMODE, BMODE, OUT><<<grid, 256, 0, s>>>(m, n, k, A, lda, B, ldb, C, ldc, kchunk,
                                                        info);
  return launched();
}

template <typename T, int AMODE, int BMODE, int OUT>
static int gemm_bn(int m, int n, int k, const T* A, int lda, const T* B, int ldb, T* C, int ldc,
                   int splits, const int* info, cudaStream_t s) {
  if (OUT == OUT_SUB_LOWER || n > 32)
    return gemm_launch4<T, 64, AMODE, BMODE, OUT>(m, n, k, A, lda, B, ldb, C, ldc, splits, info, s);
  if (n > 16)
    return gemm_launch4<T, 32, AMODE, BMODE, OUT>(m, n, k, A, lda, B, ldb, C, ldc, splits, info, s);
  return gemm_launch4<T, 16, AMODE, BMODE, OUT>(m, n, k, A, lda, B, ldb, C, ldc, splits, info, s);
}

template <typename T>
int launch_gemm(int m, int n, int k, const T* A, int lda, int amode, const T* B, int ldb,
                int bmode, T* C, int ldc, int out, int splits, const int* info, cudaStream_t s) {
  if (m <= 0 || n <= 0 || k <= 0) return JMG_OK;
#define JMG_G(AM, BM, OU) \
  if (amode == AM && bmode == BM && out == OU) \
    return gemm_bn<T, AM, BM, OU>(m, n, k, A, lda, B, ldb, C, ldc, splits, info, s);
  JMG_G(MODE_N, MODE_T, OUT_SUB_LOWER)  // SYRK: C -= P P^T
  JMG_G(MODE_N, MODE_N, OUT_SUB)        // forward-solve update: B -= L Y
  JMG_G(MODE_T, MODE_N, OUT_SUB)        // back-solve update: B -= L^T X
  JMG_G(MODE_S, MODE_N, OUT_PART)       // symmetric residual partials
  JMG_G(MODE_N, MODE_T, OUT_SUB)        // general C -= A B^T
#undef JMG_G
  return JMG_ERR_UNSUPPORTED;
}
template int launch_gemm<double>(int, int, int, const double*, int, int, const double*, int, int,
                                 double*, int, int, int, const int*, cudaStream_t);
template int launch_gemm<float>(int, int, int, const float*, int, int, const float*, int, int,
                                float*, int, int, int, const int*, cudaStream_t);

// ============================================================================
// FP64 residual R = B - A X (A symmetric, lower stored): split-K partial sums of
// A X through the tiled GEMM (mode S), then a fixed-order reduction that also
// records the per-column infinity norms of r, x and b.
// ============================================================================
int residual_splits(int n, int nrhs) {
  // enough CTAs for ~8 per SM on 152 SMs, never chunks shorter than 256
  long long tiles = (long long)cdiv(n, GBM) * cdiv(nrhs, nrhs > 32 ? 64 : (nrhs > 16 ? 32 : 16));
  long long want = 152LL * 8;
  int splits = (int)((want + tiles - 1) / tiles);
  int maxs = max(1, n / 256);
  return max(1, min(splits, maxs));
}

__global__ void k_resid_reduce(int n, int nrhs, int splits, const double* __restrict__ part,
                               const double* __restrict__ X, int ldx, const double* __restrict__ B,
                               int ldb, double* __restrict__ R, int ldr, double* __restrict__ colmax) {
  const int c = blockIdx.y;
  double rm = 0.0, xm = 0.0, bm = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int z = 0; z < splits; ++z) acc += part[(size_t)z * n * nrhs + (size_t)c * n + i];
    // B == nullptr: plain product (PCG's Q = A P) instead of the residual
    double b = B ? B[(size_t)c * ldb + i] : 0.0;
    double r = B ? b - acc : acc;
    R[(size_t)c * ldr + i] = r;
    double x = X[(size_t)c * ldx + i];
    rm = (isnan(r) || isnan(rm)) ? NAN : fmax(rm, fabs(r));
    xm = (isnan(x) || isnan(xm)) ? NAN : fmax(xm, fabs(x));
    bm = fmax(bm, fabs(b));
  }
  // warp then block max
  for (int o = 16; o > 0; o >>= 1) {
    double a = __shfl_xor_sync(0xffffffffu, rm, o);
    rm = (isnan(a) || isnan(rm)) ? NAN : fmax(rm, a);
    a = __shfl_xor_sync(0xffffffffu, xm, o);
    xm = (isnan(a) || isnan(xm)) ? NAN : fmax(xm, a);
    bm = fmax(bm, __shfl_xor_sync(0xffffffffu, bm, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomic_max_nonneg(&colmax[c], rm);
    atomic_max_nonneg(&colmax[nrhs + c], xm);
    atomic_max_nonneg(&colmax[2 * nrhs + c], bm);
  }
}

int launch_resid_reduce(int n, int nrhs, int used, const double* part, const double* X, int ldx,
                        const double* B, int ldb, double* R, int ldr, double* colmax,
                        cudaStream_t s) {
  dim3 grid(min(cdiv(n, 256), 64), nrhs);
  k_resid_reduce<<<grid, 256, 0, s>>>(n, nrhs, used, part, X, ldx, B, ldb, R, ldr, colmax);
  return launched();
}

int launch_residual(int n, int nrhs, const double* A, int lda, const double* X, int ldx,
                    const double* B, int ldb, double* R, int ldr, double* colmax, double* part,
                    int splits, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1) {
  if (n <= 0 || nrhs <= 0) return JMG_OK;
  JMG_CUDA(cudaMemsetAsync(colmax, 0, sizeof(double) * 3 * nrhs, s));
  if (ev0) JMG_CUDA(cudaEventRecord(ev0, s));
  JMG_TRY(launch_gemm<double>(n, nrhs, n, A, lda, MODE_S, X, ldx, MODE_N, part, n, OUT_PART, splits,
                              nullptr, s));
  if (ev1) JMG_CUDA(cudaEventRecord(ev1, s));
  // number of splits actually used by the GEMM grid
  int kchunk = (int)round_up((size_t)cdiv(n, splits), GBK);
  int used = cdiv(n, kchunk);
  dim3 grid(min(cdiv(n, 256), 64), nrhs);
  k_resid_reduce<<<grid, 256, 0, s>>>(n, nrhs, used, part, X, ldx, B, ldb, R, ldr, colmax);
  return launched();
}

// Row statistics of the symmetric A from its lower triangle:
//   rowsum[i] = sum_j |a_ij|   (NaN propagates; ||A||_inf = max_i rowsum[i])
//   rowmax[i] = max_j |a_ij| truncated to its upper 32 bits (sign, exponent
//               and 20 leading fraction bits): the same binary exponent as the
//               maximum, which is all the row scales of the split residual use
// over the full row j = 0..n-1.  One CTA per strip of 32 columns j reads them
// down from the diagonal in 1024-row chunks (long contiguous runs of each
// column, 16 loads in flight per thread).  Entry a_rj (r > j) adds to row r --
// kept per thread for its four rows of the chunk and flushed with one atomic
// per row and chunk -- and to row j (its mirror), kept per thread for the
// strip's 32 columns and reduced across the CTA at the end; a_jj adds once.
// The maxima are taken on the upper 32 bits of |a| as unsigned integers,
// which order like the values (NaN above every finite value).
__global__ void __launch_bounds__(256, 1) k_row_stats(int n, const double* __restrict__ A,
                                                      int lda, double* __restrict__ rowsum,
                                                      double* __restrict__ rowmax) {
  constexpr int W = 32, U = 4, TH = 256, JB = 4;
  __shared__ double red_s[TH / 32][W];
  __shared__ unsigned red_m[TH / 32][W];
  const int j0 = blockIdx.x * W;
  const int jn = min(W, n - j0);
  const int t = threadIdx.x, lane = t % 32, warp = t / 32;
  double cs[W];
  unsigned cm[W];
#pragma unroll
  for (int jj = 0; jj < W; ++jj) cs[jj] = 0.0, cm[jj] = 0u;
  for (int rb = j0; rb < n; rb += TH * U) {
    double rs[U];
    unsigned rm[U];
#pragma unroll
    for (int u = 0; u < U; ++u) rs[u] = 0.0, rm[u] = 0u;
    const double* base = A + (size_t)j0 * lda + rb + t;  // (column j0, row rb + t)
#pragma unroll
    for (int jb = 0; jb < W; jb += JB) {
      double v[JB][U];
#pragma unroll
      for (int q = 0; q < JB; ++q)  // JB x U independent loads
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int j = j0 + jb + q, r = rb + t + TH * u;
          v[q][u] = (jb + q < jn && r >= j && r < n) ? fabs(base[(jb + q) * lda + TH * u]) : 0.0;
        }
#pragma unroll
      for (int q = 0; q < JB; ++q)
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int j = j0 + jb + q, r = rb + t + TH * u;
          const unsigned hi = (unsigned)__double2hiint(v[q][u]);
          rs[u] += v[q][u];
          rm[u] = max(rm[u], hi);
          if (r > j) {
            cs[jb + q] += v[q][u];
            cm[jb + q] = max(cm[jb + q], hi);
          }
        }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int r = rb + t + TH * u;
      if (r < n) {
        if (rowsum) atomicAdd(&rowsum[r], rs[u]);
        if (rowmax) atomicMax(reinterpret_cast<unsigned*>(&rowmax[r]) + 1, rm[u]);
      }
    }
  }
  // the mirrored part of rows j0 .. j0+31: reduce the column sums over the CTA
#pragma unroll
  for (int jj = 0; jj < W; ++jj) {
    double a = cs[jj];
    unsigned m = cm[jj];
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    }
    if (lane == jj) {
      red_s[warp][jj] = a;
      red_m[warp][jj] = m;
    }
  }
  __syncthreads();
  if (t < jn) {
    double a = 0.0;
    unsigned m = 0u;
#pragma unroll
    for (int w = 0; w < TH / 32; ++w) {
      a += red_s[w][t];
      m = max(m, red_m[w][t]);
    }
    if (rowsum) atomicAdd(&rowsum[j0 + t], a);
    if (rowmax) atomicMax(reinterpret_cast<unsigned*>(&rowmax[j0 + t]) + 1, m);
  }
}

int launch_row_stats(int n, const double* A, int lda, double* rowsum, double* rowmax,
                     cudaStream_t s) {
  if (n <= 0) return JMG_OK;
  if (rowsum) JMG_CUDA(cudaMemsetAsync(rowsum, 0, sizeof(double) * n, s));
  if (rowmax) JMG_CUDA(cudaMemsetAsync(rowmax, 0, sizeof(double) * n, s));
  k_row_stats<<<cdiv(n, 32), 256, 0, s>>>(n, A, lda, rowsum, rowmax);
  return launched();
}

__global__ void k_max_reduce(int n, const double* __restrict__ v, double* __restrict__ out) {
  double m = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    m = (isnan(v[i]) || isnan(m)) ? NAN : fmax(m, v[i]);
  for (int o = 16; o > 0; o >>= 1) {
    double a = __shfl_xor_sync(0xffffffffu, m, o);
    m = (isnan(a) || isnan(m)) ? NAN : fmax(m, a);
  }
  if ((threadIdx.x & 31) == 0) atomic_max_nonneg(out, m);
}

int launch_max_reduce(int n, const double* v, double* out, cudaStream_t s) {
  JMG_CUDA(cudaMemsetAsync(out, 0, sizeof(double), s));
  if (n <= 0) return JMG_OK;
  k_max_reduce<<<min(cdiv(n, 256), 152), 256, 0, s>>>(n, v, out);
  return launched();
}

int launch_norm_inf(int n, const double* A, int lda, double* rowsum, double* out,
                    cudaStream_t s) {
  JMG_TRY(launch_row_stats(n, A, lda, rowsum, nullptr, s));
  return launch_max_reduce(n, rowsum, out, s);
}

__global__ void k_eta(int nrhs, const double* __restrict__ colmax, const double* __restrict__ anorm,
                      double* __restrict__ eta) {
  // single warp
  double worst = 0.0;
  for (int c = threadIdx.x; c < nrhs; c += 32) {
    double rn = colmax[c], xn = colmax[nrhs + c], bn = colmax[2 * nrhs + c];
    double den = (*anorm) * xn + bn;
    double e = den > 0.0 ? rn / den : (rn > 0.0 ? INFINITY : 0.0);
    if (isnan(rn) || isnan(xn)) e = NAN;
    eta[1 + c] = e;
    worst = (isnan(e) || isnan(worst)) ? NAN : fmax(worst, e);
  }
  for (int o = 16; o > 0; o >>= 1) {
    double a = __shfl_xor_sync(0xffffffffu, worst, o);
    worst = (isnan(a) || isnan(worst)) ? NAN : fmax(worst, a);
  }
  if (threadIdx.x == 0) eta[0] = worst;
}

int launch_eta(int nrhs, const double* colmax, const double* anorm, double* eta_out,
               cudaStream_t s) {
  k_eta<<<1, 32, 0, s>>>(nrhs, colmax, anorm, eta_out);
  return launched();
}

// ============================================================================
// Conversions used by the mixed-precision path.
// ============================================================================
__global__ void k_lower_to_f32(int n, const double* __restrict__ A, int lda, float* __restrict__ W,
                               int ldw, double shift) {
  // one CTA per column, rows j..n-1
  const int j = blockIdx.x;
  for (int i = j + threadIdx.x; i < n; i += blockDim.x) {
    double v = A[(size_t)j * lda + i];
    if (i == j) v += shift;
    W[(size_t)j * ldw + i] = (float)v;
  }
}

int launch_lower_to_f32(int n, const double* A, int lda, float* W, int ldw, double shift,
                        cudaStream_t s) {
  if (n <= 0) return JMG_OK;
  k_lower_to_f32<<<n, 256, 0, s>>>(n, A, lda, W, ldw, shift);
  return launched();
}

// word pairs (a, b) with a + b < words, ordered by significance
__constant__ int c_pair_a[6] = {0, 0, 1, 0, 1, 2};
__constant__ int c_pair_b[6] = {0, 1, 0, 2, 1, 0};
int split_pairs(int words) { return words <= 1 ? 1 : (words == 2 ? 3 : 6); }

template <typename H>
JMG_DEV H to16(float v);
template <>
JMG_DEV __nv_bfloat16 to16<__nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}
template <>
JMG_DEV __half to16<__half>(float v) {
  return __float2half_rn(v);
}
template <typename H>
JMG_DEV float from16(H v);
template <>
JMG_DEV float from16<__nv_bfloat16>(__nv_bfloat16 v) {
  return __bfloat162float(v);
}
template <>
JMG_DEV float from16<__half>(__half v) {
  return __half2float(v);
}

// 32 x 32 tiles through shared memory: read down the stored columns of L21,
// write along the rows of the row-major extended operands.
template <typename H>
__global__ void k_split_words(int m, int kb, const float* __restrict__ L21, int ldw, int npairs,
                              H* __restrict__ PA, H* __restrict__ PB, int ldp) {
  __shared__ float tile[32][33];
  const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    int c = c0 + ty + 8 * q, r = r0 + tx;
    tile[ty + 8 * q][tx] = (r < m && c < kb) ? L21[(size_t)c * ldw + r] : 0.0f;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    int r = r0 + ty + 8 * q, c = c0 + tx;
    if (r >= m || c >= kb) continue;
    float rem = tile[tx][ty + 8 * q];
    H w[3];
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      w[u] = to16<H>(rem);
      rem = rem - from16<H>(w[u]);
    }
    for (int p = 0; p < npairs; ++p) {
      PA[(size_t)r * ldp + p * kb + c] = w[c_pair_a[p]];
      if (PB) PB[(size_t)r * ldp + p * kb + c] = w[c_pair_b[p]];
    }
  }
}

int launch_split_words(int m, int kb, const float* L21, int ldw, int prec, int words, void* PA,
                       void* PB, int ldp, cudaStream_t s) {
  if (m <= 0) return JMG_OK;
  int np = split_pairs(words);
  dim3 grid(cdiv(m, 32), cdiv(kb, 32)), block(32, 8);
  if (prec == JMG_PREC_FP16)
    k_split_words<__half><<<grid, block, 0, s>>>(m, kb, L21, ldw, np, (__half*)PA,
                                                 np > 1 ? (__half*)PB : nullptr, ldp);
  else
    k_split_words<__nv_bfloat16><<<grid, block, 0, s>>>(m, kb, L21, ldw, np, (__nv_bfloat16*)PA,
                                                        np > 1 ? (__nv_bfloat16*)PB : nullptr,
                                                        ldp);
  return launched();
}

__global__ void k_scale_to_f32(int n, const double* __restrict__ R, int ldr,
                               const double* __restrict__ colmax_r, float* __restrict__ D, int ldd) {
  const int c = blockIdx.y;
  double sc = colmax_r[c];
  double inv = (sc > 0.0 && isfinite(sc)) ? 1.0 / sc : 1.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    D[(size_t)c * ldd + i] = (float)(R[(size_t)c * ldr + i] * inv);
}

int launch_scale_to_f32(int n, int nrhs, const double* R, int ldr, const double* colmax_r,
                        float* D, int ldd, cudaStream_t s) {
  dim3 grid(min(cdiv(n, 256), 64), nrhs);
  k_scale_to_f32<<<grid, 256, 0, s>>>(n, R, ldr, colmax_r, D, ldd);
  return launched();
}

__global__ void k_axpy_f32(int n, const float* __restrict__ D, int ldd,
                           const double* __restrict__ colmax_r, double* __restrict__ X, int ldx) {
  const int c = blockIdx.y;
  double sc = colmax_r[c];
  if (!(sc > 0.0 && isfinite(sc))) sc = 1.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    X[(size_t)c * ldx + i] += sc * (double)D[(size_t)c * ldd + i];
}

int launch_axpy_f32(int n, int nrhs, const float* D, int ldd, const double* colmax_r, double* X,
                    int ldx, cudaStream_t s) {
  dim3 grid(min(cdiv(n, 256), 64), nrhs);
  k_axpy_f32<<<grid, 256, 0, s>>>(n, D, ldd, colmax_r, X, ldx);
  return launched();
}

int launch_copy2d(int n, int nrhs, const double* src, int lds, double* dst, int ldd,
                  cudaStream_t s) {
  JMG_CUDA(cudaMemcpy2DAsync(dst, sizeof(double) * ldd, src, sizeof(double) * lds,
                             sizeof(double) * n, nrhs, cudaMemcpyDeviceToDevice, s));
  return JMG_OK;
}

int launch_zero(double* p, size_t n, cudaStream_t s) {
  JMG_CUDA(cudaMemsetAsync(p, 0, sizeof(double) * n, s));
  return JMG_OK;
}

}  // namespace jmg

namespace jmg {

// ============================================================================
// Vector kernels of the preconditioned conjugate gradient refinement (FP64,
// one right-hand side per column, columns independent).
// ============================================================================

// out[c] = sum_i U[i,c] V[i,c]; one CTA per column, fixed reduction order.
__global__ void __launch_bounds__(256) k_dot_cols(int n, const double* __restrict__ U, int ldu,
                                                  const double* __restrict__ V, int ldv,
                                                  double* __restrict__ out) {
  __shared__ double part[256];
  const int c = blockIdx.x;
  double a = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) a = fma(U[(size_t)c * ldu + i], V[(size_t)c * ldv + i], a);
  part[threadIdx.x] = a;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = part[0];
}

int launch_dot_cols(int n, int nrhs, const double* U, int ldu, const double* V, int ldv,
                    double* out, cudaStream_t s) {
  k_dot_cols<<<nrhs, 256, 0, s>>>(n, U, ldu, V, ldv, out);
  return launched();
}

// alpha_c = rz_c / pq_c (0 when pq_c <= 0, which also raises *bad);
// X += alpha P, R -= alpha Q; colmax[0..nrhs) = ||R||, [nrhs..2nrhs) = ||X||.
__global__ void k_pcg_step(int n, const double* __restrict__ P, const double* __restrict__ Q,
                           const double* __restrict__ rz, const double* __restrict__ pq,
                           double* __restrict__ X, double* __restrict__ R, int nrhs,
                           double* __restrict__ colmax, int* __restrict__ bad) {
  const int c = blockIdx.y;
  const double den = pq[c];
  double alpha = 0.0;
  if (den > 0.0 && isfinite(den)) {
    alpha = rz[c] / den;
  } else if (rz[c] != 0.0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(bad, 1);
  }
  double rm = 0.0, xm = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const size_t o = (size_t)c * n + i;
    const double x = fma(alpha, P[o], X[o]);
    const double r = fma(-alpha, Q[o], R[o]);
    X[o] = x;
    R[o] = r;
    rm = (isnan(r) || isnan(rm)) ? NAN : fmax(rm, fabs(r));
    xm = (isnan(x) || isnan(xm)) ? NAN : fmax(xm, fabs(x));
  }
  for (int o = 16; o > 0; o >>= 1) {
    double a = __shfl_xor_sync(0xffffffffu, rm, o);
    rm = (isnan(a) || isnan(rm)) ? NAN : fmax(rm, a);
    a = __shfl_xor_sync(0xffffffffu, xm, o);
    xm = (isnan(a) || isnan(xm)) ? NAN : fmax(xm, a);
  }
  if ((threadIdx.x & 31) == 0) {
    atomic_max_nonneg(&colmax[c], rm);
    atomic_max_nonneg(&colmax[nrhs + c], xm);
  }
}

int launch_pcg_step(int n, int nrhs, const double* P, const double* Q, const double* rz,
                    const double* pq, double* X, double* R, double* colmax, int* bad,
                    cudaStream_t s) {
  JMG_CUDA(cudaMemsetAsync(colmax, 0, sizeof(double) * 2 * nrhs, s));
  dim3 grid(std::min(cdiv(n, 256), 64), nrhs);
  k_pcg_step<<<grid, 256, 0, s>>>(n, P, Q, rz, pq, X, R, nrhs, colmax, bad);
  return launched();
}

// P = Z + (rz_new / rz_old) P   (beta = 0 when rz_old == 0); then rz_old = rz_new
__global__ void k_pcg_dir(int n, const double* __restrict__ Z, double* __restrict__ P,
                          const double* __restrict__ rz_new, const double* __restrict__ rz_old) {
  const int c = blockIdx.y;
  const double beta = (rz_old[c] != 0.0) ? rz_new[c] / rz_old[c] : 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const size_t o = (size_t)c * n + i;
    P[o] = fma(beta, P[o], Z[o]);
  }
}

int launch_pcg_dir(int n, int nrhs, const double* Z, double* P, const double* rz_new,
                   const double* rz_old, cudaStream_t s) {
  dim3 grid(std::min(cdiv(n, 256), 64), nrhs);
  k_pcg_dir<<<grid, 256, 0, s>>>(n, Z, P, rz_new, rz_old);
  return launched();
}

// Z = scale_c * D32 (FP64 from the FP32 preconditioner output)
__global__ void k_scale_from_f32(int n, const float* __restrict__ D, int ldd,
                                 const double* __restrict__ colmax_r, double* __restrict__ Z) {
  const int c = blockIdx.y;
  double sc = colmax_r[c];
  if (!(sc > 0.0 && isfinite(sc))) sc = 1.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    Z[(size_t)c * n + i] = sc * (double)D[(size_t)c * ldd + i];
}

int launch_scale_from_f32(int n, int nrhs, const float* D, int ldd, const double* colmax_r,
                          double* Z, cudaStream_t s) {
  dim3 grid(std::min(cdiv(n, 256), 64), nrhs);
  k_scale_from_f32<<<grid, 256, 0, s>>>(n, D, ldd, colmax_r, Z);
  return launched();
}

// max_i A_ii (A_ii > 0 expected; NaN wins) into *out (must be zeroed)
__global__ void k_diag_max(int n, const double* __restrict__ A, int lda, double* __restrict__ out) {
  double m = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double v = A[(size_t)i * lda + i];
    m = (isnan(v) || isnan(m)) ? NAN : fmax(m, fabs(v));
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double a = __shfl_xor_sync(0xffffffffu, m, o);
    m = (isnan(a) || isnan(m)) ? NAN : fmax(m, a);
  }
  if ((threadIdx.x & 31) == 0) atomic_max_nonneg(out, m);
}

int launch_diag_max(int n, const double* A, int lda, double* out, cudaStream_t s) {
  JMG_CUDA(cudaMemsetAsync(out, 0, sizeof(double), s));
  k_diag_max<<<std::max(1, std::min(cdiv(n, 256), 64)), 256, 0, s>>>(n, A, lda, out);
  return launched();
}

}  // namespace jmg

#include <cuda_fp8.h>

namespace jmg {

// ============================================================================
// FP8 quantisation of the panel with one power-of-two scale per 128-row tile
// (the 128 x 128 tiles of a 128-wide panel): one CTA per tile finds amax,
// picks e = floor(log2(448 / amax)) (448 = largest finite e4m3) clamped to
// [-126, 126], and writes q = e4m3_rn_satfinite(x * 2^e) row-major.
// ============================================================================
__global__ void __launch_bounds__(256) k_quant_fp8(int m, int kb, const float* __restrict__ L21,
                                                   int ldw, unsigned char* __restrict__ Q, int ldq,
                                                   signed char* __restrict__ ex) {
  // the tile goes through shared memory (column c at c * 129): read along the
  // columns of L21 (coalesced, 16 loads in flight per thread, amax on the way),
  // written along the rows of Q (four codes per 32-bit store)
  extern __shared__ float qtile[];
  constexpr int LDT = 129;
  __shared__ float red[8];
  __shared__ int s_e;
  const int r0 = blockIdx.x * 128;
  const int rows = min(128, m - r0);
  const int t = threadIdx.x;
  float amax = 0.0f;
  for (int base = 0; base < 128 * kb; base += 256 * 16) {
    float v[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int idx = base + t + 256 * q, i = idx & 127, c = idx >> 7;
      v[q] = (idx < 128 * kb && i < rows) ? L21[(size_t)c * ldw + r0 + i] : 0.0f;
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int idx = base + t + 256 * q;
      if (idx < 128 * kb) {
        qtile[(idx >> 7) * LDT + (idx & 127)] = v[q];
        amax = fmaxf(amax, fabsf(v[q]));
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  if ((t & 31) == 0) red[t / 32] = amax;
  __syncthreads();
  if (t == 0) {
    float a = red[0];
    for (int w = 1; w < 8; ++w) a = fmaxf(a, red[w]);
    int e = 0;
    if (a > 0.0f && isfinite(a)) {
      e = (int)floorf(log2f(448.0f / a));
      // guard the rounding of log2f: keep a * 2^e <= 448
      while (e > -126 && ldexpf(a, e) > 448.0f) --e;
      e = max(-126, min(126, e));
    }
    s_e = e;
    ex[blockIdx.x] = (signed char)e;
  }
  __syncthreads();
  const int e = s_e, kq = kb / 4;
  for (int idx = t; idx < rows * kq; idx += 256) {
    const int i = idx / kq, c = (idx % kq) * 4;
    unsigned int w = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float v = ldexpf(qtile[(c + u) * LDT + i], e);
      w |= (unsigned int)(unsigned char)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3)
           << (8 * u);
    }
    *reinterpret_cast<unsigned int*>(Q + (size_t)(r0 + i) * ldq + c) = w;
  }
}

int launch_quant_fp8(int m, int kb, const float* L21, int ldw, void* Q, int ldq, signed char* e,
                     cudaStream_t s) {
  if (m <= 0) return JMG_OK;
  if (kb % 4 || ldq % 4 || (reinterpret_cast<uintptr_t>(Q) & 3)) return JMG_ERR_ALIGN;
  const int smem = (int)sizeof(float) * kb * 129;
  JMG_TRY(ensure_smem(k_quant_fp8, smem));
  k_quant_fp8<<<cdiv(m, 128), 256, smem, s>>>(m, kb, L21, ldw, (unsigned char*)Q, ldq, e);
  return launched();
}

}  // namespace jmg
