// k_trsv.cu -- blocked triangular solves with the Cholesky factor, one launch
// per direction (paper: "Software design", the solve step of potrs):
//
//   forward   L Y = B :  Y_b = L_bb^{-1} (B_b - sum_{j<b} L_bj Y_j)
//   backward  L^T X = Y: X_b = L_bb^{-T} (Y_b - sum_{j>b} L_jb^T X_j)
//
// Block rows of 32.  CTAs take block rows in dependency order from an atomic
// ticket, so every block a CTA waits for belongs to a CTA that is already
// running: progress is guaranteed without co-residency assumptions.  Blocks
// finish in ticket order (block b needs block b-1), so one monotonic counter
// per group of right-hand sides says how many blocks are final.  A CTA reads
// the counter (acquire, bounded by globaltimer) and multiplies with every
// finished block it has not used yet, up to two per step, while the blocks of
// L it needs next are already being copied (cp.async ring, L is final).  It
// then solves its 32 x 32 diagonal block by substitution (one lane per
// right-hand side, in registers), stores its rows and advances the counter
// (release).  The right-hand sides are split into groups (grid.y) that run
// independently.
#include <algorithm>

#include "kernels.h"

namespace jmg {

namespace trsv {
constexpr int NBK = 32;   // block rows
constexpr int TH = 128;
constexpr int KCH = 2;    // finished blocks multiplied per step (at most)
constexpr int RING = 4;   // blocks of L in flight or in use
constexpr uint64_t WAIT_NS = 2000000000ull;

// right-hand sides per CTA (all of them, up to 64, for FP32; 16 for FP64) and
// the register tile of the products: TM rows x TN columns per thread
template <typename T>
struct Cfg;
template <>
struct Cfg<float> {
  static constexpr int NR = 64, TM = 4, TN = 4, PAD = 4;
};
template <>
struct Cfg<double> {
  static constexpr int NR = 16, TM = 2, TN = 2, PAD = 2;
};

template <typename T>
struct Smem {
  static constexpr int NR = Cfg<T>::NR, PAD = Cfg<T>::PAD;
  T Ls[RING][NBK][NBK + PAD];  // blocks of L: Ls[slot][k][i] = factor entry (row i, col k)
  T Ys[KCH][NBK][NR + PAD];    // finished rows of Y; Ys[0] is reused for the block's own rows
  T Ld[NBK][NBK + 1];          // diagonal block: Ld[r][c] = L(r0 + r, r0 + c)
  T rinv[NBK];                 // 1 / L_ii
  int b, ready, abort;
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
// wait until at most n of the most recent groups are pending (n <= 3)
JMG_DEV void cp_async_wait(int n) {
  switch (n) {
    case 0: asm volatile("cp.async.wait_group 0;" ::: "memory"); break;
    case 1: asm volatile("cp.async.wait_group 1;" ::: "memory"); break;
    case 2: asm volatile("cp.async.wait_group 2;" ::: "memory"); break;
    default: asm volatile("cp.async.wait_group 3;" ::: "memory"); break;
  }
}

template <typename T, int N>
struct Vec;
template <>
struct Vec<float, 4> {
  JMG_DEV static void load(const float* p, float (&v)[4]) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
  }
};
template <>
struct Vec<double, 2> {
  JMG_DEV static void load(const double* p, double (&v)[2]) {
    const double2 q = *reinterpret_cast<const double2*>(p);
    v[0] = q.x, v[1] = q.y;
  }
};
}  // namespace trsv

template <typename T>
__global__ void __launch_bounds__(trsv::TH)
    k_trsv_persist(int n, int nrhs, const T* __restrict__ L, int lda, T* __restrict__ B, int ldb,
                   int trans, int* __restrict__ tickets, int* __restrict__ done,
                   int* __restrict__ err, int* __restrict__ info) {
  using namespace trsv;
  constexpr int NR = Cfg<T>::NR, TM = Cfg<T>::TM, TN = Cfg<T>::TN;
  constexpr int RG = NBK / TM;  // row groups; column groups = TH / RG
  static_assert(RG * (NR / TN) == TH, "thread tile does not cover the block");
  if (info && *(volatile int*)info != 0) return;  // no factor: leave B alone
  extern __shared__ __align__(16) unsigned char sm_raw_trsv[];
  Smem<T>& S = *reinterpret_cast<Smem<T>*>(sm_raw_trsv);
  const int nblk = cdiv_dev(n, NBK);
  const int grp = blockIdx.y;
  const int c0 = grp * NR;
  const int ncol = min(NR, nrhs - c0);
  int* cnt = done + grp;
  const int t = threadIdx.x;
  const int ti = (t % RG) * TM, tj = (t / RG) * TN;  // this thread's tile of the products

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

    // ---- products with the finished blocks, in dependency order (the d-th
    // dependency is the block of ticket d)
    const int ndep = tk;
    auto issue_L = [&](int d) {  // one cp.async group per block of L
      const int j = trans ? nblk - 1 - d : d;
      const int j0 = j * NBK, jrows = min(NBK, n - j0);
      T(*dst)[NBK + Cfg<T>::PAD] = S.Ls[d % RING];
      for (int idx = t; idx < NBK * NBK; idx += TH) {
        const int i = trans ? idx / NBK : idx % NBK;
        const int kk = trans ? idx % NBK : idx / NBK;
        if (i < rows && kk < jrows)
          cp_async_elem(&dst[kk][i], trans ? &L[(size_t)(r0 + i) * lda + j0 + kk]
                                           : &L[(size_t)(j0 + kk) * lda + r0 + i]);
        else
          dst[kk][i] = T(0);
      }
      cp_async_commit();
    };
    // this thread's tile of the block's right-hand sides; the products are
    // subtracted from it
    T acc[TM][TN];
#pragma unroll
    for (int j = 0; j < TN; ++j)
#pragma unroll
      for (int i = 0; i < TM; ++i)
        acc[i][j] = (ti + i < rows && tj + j < ncol) ? B[(size_t)(c0 + tj + j) * ldb + r0 + ti + i]
                                                     : T(0);
    if (t < NBK) S.rinv[t] = (t < rows) ? T(1) / __ldg(&Lbb[(size_t)t * lda + t]) : T(0);
    // (rinv past the last row is 0, so padded rows of the substitution stay 0)
    int pf = 0;  // blocks of L issued
    for (; pf < min(ndep, RING - KCH); ++pf) issue_L(pf);
    for (int d = 0; d < ndep;) {
      if (t == 0) {
        int have = ld_acquire(cnt);
        if (have <= d) {
          const uint64_t t0 = globaltimer_ns();
          while ((have = ld_acquire(cnt)) <= d) {
            if (globaltimer_ns() - t0 > WAIT_NS || *(volatile int*)err) {
              S.abort = 1;
              atomicExch(err, 1);
              if (info) atomicCAS(info, 0, -1);  // the solve is incomplete
              break;
            }
            __nanosleep(32);
          }
        }
        S.ready = min(min(have, ndep), d + KCH);
      }
      __syncthreads();
      if (S.abort) break;
      const int ready = S.ready;
      // rows of Y (L2 only: other SMs wrote them)
      {
        constexpr int PER = NBK * NR / TH;  // elements per thread and block
        T v[KCH][PER];
#pragma unroll
        for (int q = 0; q < KCH; ++q) {  // all loads first, then the stores
          const int j = trans ? nblk - 1 - (d + q) : d + q;
          const int j0 = j * NBK;
#pragma unroll
          for (int e = 0; e < PER; ++e) {
            const int idx = t + TH * e, kk = idx % NBK, c = idx / NBK;
            v[q][e] = (q < ready - d && j0 + kk < n && c < ncol)
                          ? __ldcg(&B[(size_t)(c0 + c) * ldb + j0 + kk])
                          : T(0);
          }
        }
#pragma unroll
        for (int q = 0; q < KCH; ++q)
#pragma unroll
          for (int e = 0; e < PER; ++e) {
            const int idx = t + TH * e;
            S.Ys[q][idx % NBK][idx / NBK] = v[q][e];
          }
      }
      for (; pf < min(ndep, ready + RING - KCH); ++pf) issue_L(pf);
      cp_async_wait(pf - ready);  // blocks d .. ready-1 (and the diagonal block) have landed
      __syncthreads();
      for (int q = 0; q < ready - d; ++q) {
        T(*Lq)[NBK + Cfg<T>::PAD] = S.Ls[(d + q) % RING];
#pragma unroll 8
        for (int kk = 0; kk < NBK; ++kk) {
          T a[TM], y[TN];
          Vec<T, TM>::load(&Lq[kk][ti], a);
          Vec<T, TN>::load(&S.Ys[q][kk][tj], y);
#pragma unroll
          for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) acc[i][j] = fma(-a[i], y[j], acc[i][j]);
        }
      }
      __syncthreads();  // the ring slots and Ys are free again
      d = ready;
    }
    if (S.abort) {
      cp_async_wait(0);  // no copy of ours may land after the CTA moves on
      break;
    }
    cp_async_wait(0);  // the diagonal block has landed (when there was no dependency)

    // ---- the diagonal block: right-hand side minus the products, then one
    // lane per right-hand side solves the 32 x 32 system in registers
    T(*Ss)[NR + Cfg<T>::PAD] = S.Ys[0];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) Ss[ti + i][tj + j] = acc[i][j];
    __syncthreads();
    if (t < NR) {
      const int c = t;
      T s[NBK];
#pragma unroll
      for (int r = 0; r < NBK; ++r) s[r] = Ss[r][c];
      if (!trans) {
#pragma unroll
        for (int i = 0; i < NBK; ++i) {
          const T y = s[i] * S.rinv[i];
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
      for (int r = 0; r < NBK; ++r) Ss[r][c] = s[r];
    }
    __syncthreads();
    for (int idx = t; idx < NBK * NR; idx += TH) {  // coalesced down the columns
      const int r = idx % NBK, c = idx / NBK;
      if (r < rows && c < ncol) B[(size_t)(c0 + c) * ldb + r0 + r] = Ss[r][c];
    }
    // ---- publish: every thread's stores, then one release of the counter
    __syncthreads();
    if (t == 0) {
      __threadfence();
      st_release(cnt, tk + 1);
    }
  }
}

size_t trsv_sync_ints(int n, int nrhs) {
  (void)n;
  // per group of right-hand sides (sized for the smaller, FP64, groups of 16):
  // a ticket counter and a counter of finished blocks; then the error word
  const int groups = cdiv(std::max(nrhs, 1), 16);
  return (size_t)groups * 2 + 1;
}

template <typename T>
int launch_trsv_persist(int n, int nrhs, const T* L, int lda, T* B, int ldb, int trans,
                        int* sync, int* info, cudaStream_t s) {
  if (n <= 0 || nrhs <= 0) return JMG_OK;
  const int groups = cdiv(nrhs, trsv::Cfg<T>::NR), nblk = cdiv(n, trsv::NBK);
  int* tickets = sync;
  int* done = sync + groups;
  int* err = done + groups;
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
  k<<<dim3(gx, groups), trsv::TH, smem, s>>>(n, nrhs, L, lda, B, ldb, trans, tickets, done, err,
                                             info);
  return launched();
}
template int launch_trsv_persist<float>(int, int, const float*, int, float*, int, int, int*,
                                        int*, cudaStream_t);
template int launch_trsv_persist<double>(int, int, const double*, int, double*, int, int, int*,
                                         int*, cudaStream_t);

}  // namespace jmg
