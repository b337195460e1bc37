// k_trsv.cu -- blocked triangular solves with the Cholesky factor, one launch
// per direction (paper: "Software design", the solve step of potrs):
//
//   forward   L Y = B :  Y_b = L_bb^{-1} (B_b - sum_{j<b} L_bj Y_j)
//   backward  L^T X = Y: X_b = L_bb^{-T} (Y_b - sum_{j>b} L_jb^T X_j)
//
// Block rows of 128.  CTAs take block rows in dependency order from an atomic
// ticket, so every block a CTA waits for belongs to a CTA that is already
// running: progress is guaranteed without co-residency assumptions.  A CTA
// accumulates the products with the finished blocks as their flags appear
// (acquire loads, bounded by globaltimer), then solves its diagonal block by
// substitution in 32-row sub-blocks and publishes its rows (release).  The
// right-hand sides are split into groups of 16 columns (grid.y) that run
// independently, which shortens the serial chain per group.
#include <algorithm>

#include "kernels.h"

namespace jmg {

namespace trsv {
constexpr int NBK = 128;  // block rows
constexpr int NR = 16;    // right-hand sides per group
constexpr int KC = 32;    // K chunk of the off-diagonal products
constexpr int SB = 32;    // substitution sub-block
constexpr uint64_t WAIT_NS = 2000000000ull;

template <typename T>
struct Smem {
  T Ld[NBK][NBK + 1];  // diagonal block (lower), row-major by row index
  T Ls[KC][NBK + 1];   // off-diagonal chunk: Ls[k][i]
  T Ys[KC][NR + 1];    // finished solution chunk
  T Ss[NBK][NR + 1];   // the block's right-hand sides
  T rinv[NBK];         // 1 / L_ii
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
template <typename T>
JMG_DEV T ldcg(const T* p) {
  return __ldcg(p);
}
}  // namespace trsv

template <typename T>
__global__ void __launch_bounds__(256) k_trsv_persist(int n, int nrhs, const T* __restrict__ L,
                                                      int lda, T* __restrict__ B, int ldb,
                                                      int trans, int* __restrict__ tickets,
                                                      int* __restrict__ flags,
                                                      int* __restrict__ err,
                                                      int* __restrict__ info) {
  using namespace trsv;
  if (info && *(volatile int*)info != 0) return;  // no factor: leave B alone
  extern __shared__ __align__(16) unsigned char sm_raw_trsv[];
  Smem<T>& S = *reinterpret_cast<Smem<T>*>(sm_raw_trsv);
  const int nblk = cdiv_dev(n, NBK);
  const int grp = blockIdx.y;
  const int c0 = grp * NR;
  const int ncol = min(NR, nrhs - c0);
  int* flag = flags + (size_t)grp * nblk;
  const int t = threadIdx.x, tx = t % 32, ty = t / 32;  // rows tx + 32q, cols ty + 8p

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

    T acc[4][2];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const int i = tx + 32 * q, c = ty + 8 * p;
        acc[q][p] = (i < rows && c < ncol) ? B[(size_t)(c0 + c) * ldb + r0 + i] : T(0);
      }

    // ---- off-diagonal products as a stream of 32-column chunks; the next
    // chunk of L (final, no flag needed) is prefetched into registers while
    // the current one is multiplied.  Y chunks are read after the flag of
    // their block was acquired.
    constexpr int LQ = KC * NBK / 256, YQ = KC * NR / 256;
    const int ndep = trans ? (nblk - 1 - b) : b;
    T lv[LQ];
    auto load_L = [&](int dd, int kk0) {
      const int j = trans ? (nblk - 1 - dd) : dd;
      const int j0 = j * NBK, jrows = min(NBK, n - j0);
#pragma unroll
      for (int q = 0; q < LQ; ++q) {
        const int idx = t + 256 * q;
        const int i = trans ? idx / KC : idx % NBK;
        const int kk = trans ? idx % KC : idx / NBK;
        const int gk = kk0 + kk;
        T v = T(0);
        if (i < rows && gk < jrows)
          v = trans ? L[(size_t)(r0 + i) * lda + j0 + gk] : L[(size_t)(j0 + gk) * lda + r0 + i];
        lv[q] = v;
      }
    };
    int d = 0, k0 = 0;
    if (ndep > 0) load_L(0, 0);
    while (d < ndep) {
      const int j = trans ? (nblk - 1 - d) : d;
      const int j0 = j * NBK, jrows = min(NBK, n - j0);
      if (k0 == 0) {
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
              __nanosleep(64);
            }
          }
        }
        __syncthreads();
        if (S.abort) break;
      }
      T yv[YQ];
#pragma unroll
      for (int q = 0; q < YQ; ++q) {
        const int idx = t + 256 * q;
        const int kk = idx % KC, c = idx / KC, gk = k0 + kk;
        yv[q] = (gk < jrows && c < ncol) ? ldcg(&B[(size_t)(c0 + c) * ldb + j0 + gk]) : T(0);
      }
#pragma unroll
      for (int q = 0; q < LQ; ++q) {
        const int idx = t + 256 * q;
        const int i = trans ? idx / KC : idx % NBK;
        const int kk = trans ? idx % KC : idx / NBK;
        S.Ls[kk][i] = lv[q];
      }
#pragma unroll
      for (int q = 0; q < YQ; ++q) {
        const int idx = t + 256 * q;
        S.Ys[idx % KC][idx / KC] = yv[q];
      }
      __syncthreads();
      int nd = d, nk0 = k0 + KC;
      if (nk0 >= jrows) {
        nd = d + 1;
        nk0 = 0;
      }
      if (nd < ndep) load_L(nd, nk0);
#pragma unroll 8
      for (int kk = 0; kk < KC; ++kk) {
        T a[4], y[2];
#pragma unroll
        for (int q = 0; q < 4; ++q) a[q] = S.Ls[kk][tx + 32 * q];
#pragma unroll
        for (int p = 0; p < 2; ++p) y[p] = S.Ys[kk][ty + 8 * p];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int p = 0; p < 2; ++p) acc[q][p] -= a[q] * y[p];
      }
      __syncthreads();
      d = nd;
      k0 = nk0;
    }
    if (S.abort) break;

    // ---- diagonal block: right-hand sides and L_bb to shared memory
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int p = 0; p < 2; ++p) S.Ss[tx + 32 * q][ty + 8 * p] = acc[q][p];
    for (int base = 0; base < NBK * NBK; base += 256 * 16) {  // 16 loads in flight
      T v[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int idx = base + t + 256 * q;
        const int i = idx % NBK, k = idx / NBK;  // column k, row i: coalesced down a column
        v[q] = (i < rows && k < rows && i >= k) ? L[(size_t)(r0 + k) * lda + r0 + i] : T(0);
      }
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int idx = base + t + 256 * q;
        S.Ld[idx % NBK][idx / NBK] = v[q];
      }
    }
    __syncthreads();
    if (t < NBK) S.rinv[t] = (t < rows) ? T(1) / S.Ld[t][t] : T(0);
    __syncthreads();

    // ---- substitution, 32-row sub-blocks: warp 0 (lane = column) solves the
    // sub-block in registers, then all threads update the remaining rows
    const int nsb = cdiv_dev(rows, SB);
    for (int u = 0; u < nsb; ++u) {
      const int sb = trans ? (nsb - 1 - u) : u;
      const int s0 = sb * SB;
      if (t < NR) {
        const int c = t;
        T s[SB];
#pragma unroll
        for (int r = 0; r < SB; ++r) s[r] = (s0 + r < rows) ? S.Ss[s0 + r][c] : T(0);
        if (!trans) {
#pragma unroll
          for (int i = 0; i < SB; ++i) {
            if (s0 + i < rows) {
              const T y = s[i] * S.rinv[s0 + i];
              s[i] = y;
#pragma unroll
              for (int k = i + 1; k < SB; ++k) s[k] -= S.Ld[s0 + k][s0 + i] * y;
            }
          }
        } else {
#pragma unroll
          for (int i = SB - 1; i >= 0; --i) {
            if (s0 + i < rows) {
              const T x = s[i] * S.rinv[s0 + i];
              s[i] = x;
#pragma unroll
              for (int k = 0; k < i; ++k) s[k] -= S.Ld[s0 + i][s0 + k] * x;
            }
          }
        }
#pragma unroll
        for (int r = 0; r < SB; ++r)
          if (s0 + r < rows) S.Ss[s0 + r][c] = s[r];
      }
      __syncthreads();
      // remaining rows: forward rows below the sub-block, backward rows above
      const int lo = trans ? 0 : s0 + SB, hi = trans ? s0 : rows;
      for (int idx = t; idx < (hi - lo) * NR; idx += 256) {
        const int k = lo + idx / NR, c = idx % NR;
        T v = S.Ss[k][c];
#pragma unroll 8
        for (int i = 0; i < SB; ++i) {
          if (s0 + i < rows) v -= (trans ? S.Ld[s0 + i][k] : S.Ld[k][s0 + i]) * S.Ss[s0 + i][c];
        }
        S.Ss[k][c] = v;
      }
      __syncthreads();
    }

    // ---- publish
    for (int idx = t; idx < NBK * NR; idx += 256) {
      const int i = idx % NBK, c = idx / NBK;
      if (i < rows && c < ncol) B[(size_t)(c0 + c) * ldb + r0 + i] = S.Ss[i][c];
    }
    __threadfence();
    __syncthreads();
    if (t == 0) st_release(&flag[b], 1);
  }
}

size_t trsv_sync_ints(int n, int nrhs) {
  const int groups = cdiv(nrhs, trsv::NR), nblk = cdiv(n, trsv::NBK);
  return (size_t)groups * (1 + nblk) + 1;  // tickets, flags, error word
}

template <typename T>
int launch_trsv_persist(int n, int nrhs, const T* L, int lda, T* B, int ldb, int trans,
                        int* sync, int* info, cudaStream_t s) {
  if (n <= 0 || nrhs <= 0) return JMG_OK;
  const int groups = cdiv(nrhs, trsv::NR), nblk = cdiv(n, trsv::NBK);
  int* tickets = sync;
  int* flags = sync + groups;
  int* err = flags + (size_t)groups * nblk;
  JMG_CUDA(cudaMemsetAsync(sync, 0, sizeof(int) * trsv_sync_ints(n, nrhs), s));
  const size_t smem = sizeof(trsv::Smem<T>);
  static int done_attr[2] = {0, 0};
  auto k = k_trsv_persist<T>;
  const int which = sizeof(T) == 8;
  if (!done_attr[which]) {
    JMG_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    done_attr[which] = 1;
  }
  int dev = 0, nsm = 152, per_sm = 1;
  JMG_CUDA(cudaGetDevice(&dev));
  JMG_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  JMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, smem));
  per_sm = per_sm < 1 ? 1 : per_sm;
  const int slots = nsm * per_sm;
  const int gx = std::max(1, std::min(nblk, slots / groups));
  k<<<dim3(gx, groups), 256, smem, s>>>(n, nrhs, L, lda, B, ldb, trans, tickets, flags, err,
                                        info);
  return launched();
}
template int launch_trsv_persist<float>(int, int, const float*, int, float*, int, int, int*,
                                        int*, cudaStream_t);
template int launch_trsv_persist<double>(int, int, const double*, int, double*, int, int, int*,
                                         int*, cudaStream_t);

}  // namespace jmg
