// k_trsv.cu -- blocked triangular solves with the Cholesky factor, one launch
// per direction (paper: "Software design", the solve step of potrs):
//
//   forward   L Y = B :  Y_b = L_bb^{-1} (B_b - sum_{j<b} L_bj Y_j)
//   backward  L^T X = Y: X_b = L_bb^{-T} (Y_b - sum_{j>b} L_jb^T X_j)
//
// Block rows of 32.  CTAs take block rows in dependency order from an atomic
// ticket, so every block a CTA waits for belongs to a CTA that is already
// running: progress is guaranteed without co-residency assumptions.  A CTA
// accumulates the products with the finished blocks as their flags appear
// (acquire loads, bounded by globaltimer), then solves its 32 x 32 diagonal
// block by substitution (one lane per right-hand side, in registers) and
// publishes its rows (release).  Small blocks keep the serial chain -- one
// 32 x 32 product, one substitution and one publish per block -- short; the
// right-hand sides are split into groups (grid.y) that run independently.
#include <algorithm>

#include "kernels.h"

namespace jmg {

namespace trsv {
constexpr int NBK = 32;  // block rows (also the K chunk: one chunk per dependency block)
constexpr int TH = 128;
constexpr uint64_t WAIT_NS = 2000000000ull;

// right-hand sides per CTA: all of them (up to 64) for FP32, 16 for FP64
template <typename T>
struct Cfg;
template <>
struct Cfg<float> {
  static constexpr int NR = 64;
};
template <>
struct Cfg<double> {
  static constexpr int NR = 16;
};

template <typename T>
struct Smem {
  static constexpr int NR = Cfg<T>::NR;
  T Ls[2][NBK][NBK + 1];  // dependency blocks of L (double-buffered): Ls[buf][k][i]
  T Ys[NBK][NR + 1];      // finished solution rows of the dependency block
  T Ss[NBK][NR + 1];      // the block's right-hand sides
  T Ld[NBK][NBK + 1];     // diagonal block: Ld[r][c] = L(r0 + r, r0 + c)
  T rinv[NBK];            // 1 / L_ii
  int b, abort;
};

JMG_DEV int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
JMG_DEV void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// asynchronous global -> shared copies of one element (L is final while the
// kernel runs, so caching it in L1 is safe)
JMG_DEV void cp_async_elem(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src)
               : "memory");
}
JMG_DEV void cp_async_elem(double* dst, const double* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src)
               : "memory");
}
JMG_DEV void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
JMG_DEV void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
JMG_DEV void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
}  // namespace trsv

template <typename T>
__global__ void __launch_bounds__(trsv::TH)
    k_trsv_persist(int n, int nrhs, const T* __restrict__ L, int lda, T* __restrict__ B, int ldb,
                   int trans, int* __restrict__ tickets, int* __restrict__ flags,
                   int* __restrict__ err, int* __restrict__ info) {
  using namespace trsv;
  constexpr int NR = Cfg<T>::NR, CP = NR / 8;  // thread: rows tx, tx+16; cols ty + 8p
  if (info && *(volatile int*)info != 0) return;  // no factor: leave B alone
  extern __shared__ __align__(16) unsigned char sm_raw_trsv[];
  Smem<T>& S = *reinterpret_cast<Smem<T>*>(sm_raw_trsv);
  const int nblk = cdiv_dev(n, NBK);
  const int grp = blockIdx.y;
  const int c0 = grp * NR;
  const int ncol = min(NR, nrhs - c0);
  int* flag = flags + (size_t)grp * nblk;
  const int t = threadIdx.x, tx = t % 16, ty = t / 16;

  while (true) {
    if (t == 0) {
      S.b = atomicAdd(&tickets[grp], 1);
      S.abort = 0;
    }
    __syncthreads();
    const int tk = S.b;
    if (tk >= nblk) break;
    const int b = trans ? nblk - 1 - tk : tk;
    const int r0 = b * NBK, rows = min(NBK, n - r0);
    const T* Lbb = L + (size_t)r0 * lda + r0;  // diagonal block

    // the diagonal block is final: start copying it now, it is needed last
    for (int idx = t; idx < NBK * NBK; idx += TH) {
      const int r = idx % NBK, c = idx / NBK;  // down a column of L
      if (r < rows && c < rows && r >= c)
        cp_async_elem(&S.Ld[r][c], &Lbb[(size_t)c * lda + r]);
      else
        S.Ld[r][c] = T(0);
    }
    cp_async_commit();

    T acc[2][CP];
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int p = 0; p < CP; ++p) {
        const int i = tx + 16 * q, c = ty + 8 * p;
        acc[q][p] = (i < rows && c < ncol) ? B[(size_t)(c0 + c) * ldb + r0 + i] : T(0);
      }
    if (t < NBK) S.rinv[t] = (t < rows) ? T(1) / __ldg(&Lbb[(size_t)t * lda + t]) : T(0);
    // (rinv past the last row is 0, so padded rows of the substitution stay 0)

    // ---- products with the finished blocks, in dependency order.  The next
    // block of L (final, no flag needed) is copied asynchronously into the
    // other buffer while the current one is multiplied; rows of Y are read
    // (L2 only: other SMs wrote them) after the flag of their block.
    const int ndep = trans ? (nblk - 1 - b) : b;
    auto issue_L = [&](int dd, int buf) {
      const int j = trans ? (nblk - 1 - dd) : dd;
      const int j0 = j * NBK, jrows = min(NBK, n - j0);
      for (int idx = t; idx < NBK * NBK; idx += TH) {
        const int i = trans ? idx / NBK : idx % NBK;
        const int kk = trans ? idx % NBK : idx / NBK;
        T* dst = &S.Ls[buf][kk][i];
        if (i < rows && kk < jrows)
          cp_async_elem(dst, trans ? &L[(size_t)(r0 + i) * lda + j0 + kk]
                                   : &L[(size_t)(j0 + kk) * lda + r0 + i]);
        else
          *dst = T(0);
      }
      cp_async_commit();
    };
    if (ndep > 0) issue_L(0, 0);
    int buf = 0;
    for (int d = 0; d < ndep; ++d, buf ^= 1) {
      const int j = trans ? (nblk - 1 - d) : d;
      const int j0 = j * NBK, jrows = min(NBK, n - j0);
      if (t == 0) {
        if (!ld_acquire(&flag[j])) {
          const uint64_t t0 = globaltimer_ns();
          while (!ld_acquire(&flag[j])) {
            if (globaltimer_ns() - t0 > WAIT_NS || *(volatile int*)err) {
              S.abort = 1;
              atomicExch(err, 1);
              if (info) atomicCAS(info, 0, -1);  // the solve is incomplete
              break;
            }
            __nanosleep(32);
          }
        }
      }
      __syncthreads();
      if (S.abort) break;
      for (int idx = t; idx < NBK * NR; idx += TH) {
        const int kk = idx % NBK, c = idx / NBK;
        S.Ys[kk][c] = (kk < jrows && c < ncol) ? __ldcg(&B[(size_t)(c0 + c) * ldb + j0 + kk]) : T(0);
      }
      if (d + 1 < ndep) {
        issue_L(d + 1, buf ^ 1);
        cp_async_wait1();  // this block's copies (and the diagonal block's) have landed
      } else {
        cp_async_wait0();
      }
      __syncthreads();
#pragma unroll 8
      for (int kk = 0; kk < NBK; ++kk) {
        T a[2], y[CP];
#pragma unroll
        for (int q = 0; q < 2; ++q) a[q] = S.Ls[buf][kk][tx + 16 * q];
#pragma unroll
        for (int p = 0; p < CP; ++p) y[p] = S.Ys[kk][ty + 8 * p];
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
          for (int p = 0; p < CP; ++p) acc[q][p] -= a[q] * y[p];
      }
      __syncthreads();
    }
    if (S.abort) {
      cp_async_wait0();  // no copy of ours may land after the CTA moves on
      break;
    }
    cp_async_wait0();  // the diagonal block has landed (when there was no dependency)

    // ---- the diagonal block: one lane per right-hand side, in registers
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int p = 0; p < CP; ++p) S.Ss[tx + 16 * q][ty + 8 * p] = acc[q][p];
    __syncthreads();
    if (t < NR) {
      const int c = t;
      T s[NBK];
#pragma unroll
      for (int r = 0; r < NBK; ++r) s[r] = S.Ss[r][c];
      if (!trans) {
#pragma unroll
        for (int i = 0; i < NBK; ++i) {
          const T y = s[i] * S.rinv[i];  // rinv is 0 past the last row
          s[i] = y;
#pragma unroll
          for (int k = i + 1; k < NBK; ++k) s[k] -= S.Ld[k][i] * y;
        }
      } else {
#pragma unroll
        for (int i = NBK - 1; i >= 0; --i) {
          const T x = s[i] * S.rinv[i];
          s[i] = x;
#pragma unroll
          for (int k = 0; k < i; ++k) s[k] -= S.Ld[i][k] * x;
        }
      }
#pragma unroll
      for (int r = 0; r < NBK; ++r) S.Ss[r][c] = s[r];
    }
    __syncthreads();
    for (int idx = t; idx < NBK * NR; idx += TH) {  // coalesced down the columns
      const int r = idx % NBK, c = idx / NBK;
      if (r < rows && c < ncol) B[(size_t)(c0 + c) * ldb + r0 + r] = S.Ss[r][c];
    }
    // ---- publish
    __threadfence();
    __syncthreads();
    if (t == 0) st_release(&flag[b], 1);
  }
}

size_t trsv_sync_ints(int n, int nrhs) {
  // sized for the smaller of the per-type groups (16 right-hand sides) and
  // 32-row blocks
  const int groups = cdiv(nrhs, 16), nblk = cdiv(n, trsv::NBK);
  return (size_t)groups * (1 + nblk) + 1;  // tickets, flags, error word
}

template <typename T>
int launch_trsv_persist(int n, int nrhs, const T* L, int lda, T* B, int ldb, int trans,
                        int* sync, int* info, cudaStream_t s) {
  if (n <= 0 || nrhs <= 0) return JMG_OK;
  const int groups = cdiv(nrhs, trsv::Cfg<T>::NR), nblk = cdiv(n, trsv::NBK);
  int* tickets = sync;
  int* flags = sync + groups;
  int* err = flags + (size_t)groups * nblk;
  JMG_CUDA(cudaMemsetAsync(sync, 0, sizeof(int) * trsv_sync_ints(n, nrhs), s));
  const size_t smem = sizeof(trsv::Smem<T>);
  auto k = k_trsv_persist<T>;
  static int done_attr[2] = {0, 0};
  const int which = sizeof(T) == 8;
  if (!done_attr[which]) {
    JMG_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    done_attr[which] = 1;
  }
  // one CTA per block row and group when they all fit; the tickets keep the
  // dependency order either way
  int dev = 0, nsm = 152, per_sm = 1;
  JMG_CUDA(cudaGetDevice(&dev));
  JMG_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  JMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, trsv::TH, smem));
  per_sm = per_sm < 1 ? 1 : per_sm;
  const int slots = nsm * per_sm;
  const int gx = std::max(1, std::min(nblk, slots / groups));
  k<<<dim3(gx, groups), trsv::TH, smem, s>>>(n, nrhs, L, lda, B, ldb, trans, tickets,
                                                     flags, err, info);
  return launched();
}
template int launch_trsv_persist<float>(int, int, const float*, int, float*, int, int, int*,
                                        int*, cudaStream_t);
template int launch_trsv_persist<double>(int, int, const double*, int, double*, int, int, int*,
                                         int*, cudaStream_t);

}  // namespace jmg
