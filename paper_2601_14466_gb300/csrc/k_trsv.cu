// k_trsv.cu -- blocked triangular solves with the Cholesky factor, one launch
// per direction (paper: "Software design", the solve step of potrs):
//
//   forward   L Y = B :  Y_b = L_bb^{-1} (B_b - sum_{j<b} L_bj Y_j)
//   backward  L^T X = Y: X_b = L_bb^{-T} (Y_b - sum_{j>b} L_jb^T X_j)
//
// Block rows of 32, taken in dependency order d = 0, 1, ... (b = d forward,
// b = nblk-1-d backward).  The serial chain runs in ONE CTA, the leader: for
// each block it takes the partial right-hand side P_d, subtracts the products
// with the LAG-1 blocks it finished last (kept in shared memory), solves the
// 32 x 32 diagonal block by substitution (one lane per right-hand side), keeps
// the rows and publishes them (store, then a release of a counter of finished
// blocks).  Every other CTA is a helper: block d >= LAG gets
//     P_d = B_d - sum_{j <= d-LAG} L_dj Y_j
// from the published rows as they appear (acquire loads of the counter,
// bounded by globaltimer), written in place over B_d, and flags it (release).
// The leader thus never waits for another SM's rows of the last LAG-1 blocks,
// only for P_d, which the helpers finish LAG-1 blocks ahead.
//
// Roles come from an atomic ticket in order (ticket 0 leads; ticket t helps
// block LAG + t - 1), so the leader is running before any helper, and a helper
// of block d depends only on the leader, which depends only on helpers of
// lower blocks, all of which took their tickets earlier: no co-residency
// assumption beyond the leader's.  The right-hand sides are split into groups
// (grid.y) that run independently, each with its own leader.
#include <algorithm>

#include "kernels.h"

namespace jmg {

namespace trsv {
constexpr int NBK = 32;   // block rows
constexpr int TH = 320;   // leader: 8 compute warps, a publishing warp and a fetching warp
constexpr int CT = 256;   // compute threads
constexpr int LAG = 3;    // blocks the leader multiplies itself: d-1 .. d-LAG+1
constexpr int KCH = 2;    // finished blocks a helper multiplies per step (at most)
constexpr int RING = 4;   // helper: blocks of L in flight or in use (KCH + 2)

// right-hand sides per group (all of them, up to 64, for FP32; 16 for FP64),
// the register tile of the products (TM rows x TN columns per thread), and the
// row padding of the blocks of L (rows stay 16-byte aligned for the vector
// loads).  Row-of-Y buffers are padded by one element (a row stride of
// 1 mod 32 words keeps column-wise accesses free of bank conflicts).
template <typename T>
struct Cfg;
template <>
struct Cfg<float> {
  static constexpr int NR = 64, TM = 2, TN = 4, PADL = 4;
};
template <>
struct Cfg<double> {
  static constexpr int NR = 16, TM = 2, TN = 1, PADL = 2;
};

constexpr int PADY = 1;

template <typename T>
struct Helper {
  static constexpr int NR = Cfg<T>::NR, PADL = Cfg<T>::PADL;
  T Ls[RING][NBK][NBK + PADL];  // blocks of L: Ls[slot][k][i] = factor entry (row i, col k)
  T Ys[KCH][NBK][NR + PADY];    // finished rows of Y
};
template <typename T>
struct Leader {
  static constexpr int NR = Cfg<T>::NR, PADL = Cfg<T>::PADL;
  static constexpr int PB = (NBK * (NR + PADY) + NR - 1) / NR;  // >= NBK: also holds Ss
  T Lo[2][LAG - 1][NBK][NBK + PADL];  // off-diagonal blocks of the next two steps, [k][i]
  T Ld[2][NBK][NBK + 1];             // diagonal blocks: Ld[r][c] = L(r0 + r, r0 + c)
  T Yr[LAG - 1][NBK][NR + PADY];      // the last LAG-1 solved blocks (ring)
  T Pb[2][NR][PB];                   // P_d column-major (Pb[c][r]); then reused as Ss[r][c]
  T rinv[2][NBK];
};
template <typename T>
struct Smem {
  union {
    Helper<T> h;
    Leader<T> l;
  };
  int ticket, ready, abort;
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
JMG_DEV void bar_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
JMG_DEV void bar_arrive(int id, int count) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
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
struct Vec<float, 1> {
  JMG_DEV static void load(const float* p, float (&v)[1]) { v[0] = *p; }
};
template <>
struct Vec<float, 2> {
  JMG_DEV static void load(const float* p, float (&v)[2]) {
    const float2 q = *reinterpret_cast<const float2*>(p);
    v[0] = q.x, v[1] = q.y;
  }
};
template <>
struct Vec<double, 2> {
  JMG_DEV static void load(const double* p, double (&v)[2]) {
    const double2 q = *reinterpret_cast<const double2*>(p);
    v[0] = q.x, v[1] = q.y;
  }
};
template <>
struct Vec<double, 1> {
  JMG_DEV static void load(const double* p, double (&v)[1]) { v[0] = *p; }
};

// Bounded spin of thread 0 until *p > d (acquire).  On expiry (limit_ns of
// %globaltimer), or when another CTA raised the error word, flags the abort:
// the solve is then incomplete.
template <typename T>
JMG_DEV void wait_gt(const int* p, int d, int* err, int* info, Smem<T>& S, uint64_t limit_ns) {
  int have = ld_acquire(p);
  if (have <= d) {
    const uint64_t t0 = globaltimer_ns();
    while ((have = ld_acquire(p)) <= d) {
      if (globaltimer_ns() - t0 > limit_ns || *(volatile int*)err) {
        S.abort = 1;
        atomicExch(err, JMG_ERR_TIMEOUT);
        if (info) atomicCAS(info, 0, -1);
        break;
      }
      __nanosleep(32);
    }
  }
  S.ready = have;
}

// Copy the 32 x 32 block of L that multiplies rows r0.. (rows, row count `rows`)
// with the solved block j into dst[k][i] (transposed for the backward solve).
template <typename T, int LD, int NT>
JMG_DEV void copy_offdiag(T (*dst)[LD], const T* L, int lda, int n, int r0, int rows, int j,
                          int trans, int t) {
  const int j0 = j * NBK, jrows = min(NBK, n - j0);
  for (int idx = t; idx < NBK * NBK; idx += NT) {
    const int i = trans ? idx / NBK : idx % NBK;
    const int kk = trans ? idx % NBK : idx / NBK;
    if (i < rows && kk < jrows)
      cp_async_elem(&dst[kk][i], trans ? &L[(size_t)(r0 + i) * lda + j0 + kk]
                                       : &L[(size_t)(j0 + kk) * lda + r0 + i]);
    else
      dst[kk][i] = T(0);
  }
}

// acc (TM x TN tile at rows ti, columns tj) -= Lq Yq over one 32-wide block
template <typename T, int LDL, int LDY>
JMG_DEV void block_product(const T (*Lq)[LDL], const T (*Yq)[LDY], int ti, int tj,
                           T (&acc)[Cfg<T>::TM][Cfg<T>::TN]) {
  constexpr int TM = Cfg<T>::TM, TN = Cfg<T>::TN;
#pragma unroll 8
  for (int kk = 0; kk < NBK; ++kk) {
    T a[TM], y[TN];
    Vec<T, TM>::load(&Lq[kk][ti], a);
#pragma unroll
    for (int j = 0; j < TN; ++j) y[j] = Yq[kk][tj + j];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[i][j] = fma(-a[i], y[j], acc[i][j]);
  }
}
}  // namespace trsv

template <typename T>
__global__ void __launch_bounds__(trsv::TH, 2)
    k_trsv_persist(int n, int nrhs, const T* __restrict__ L, int lda, T* __restrict__ B, int ldb,
                   int trans, int g0, int* __restrict__ tickets, int* __restrict__ done,
                   int* __restrict__ pflag, int* __restrict__ err, int* __restrict__ info,
                   unsigned long long wait_ns, int tkt0) {
  using namespace trsv;
  constexpr int NR = Cfg<T>::NR, TM = Cfg<T>::TM, TN = Cfg<T>::TN, PADL = Cfg<T>::PADL;
  constexpr int RG = NBK / TM;  // row groups; column groups = TH / RG
  static_assert(RG * (NR / TN) == CT, "thread tile does not cover the block");
  if (info && *(volatile int*)info != 0) return;  // no factor: leave B alone
  if (*(volatile int*)err != 0) return;           // the other direction gave up
  extern __shared__ __align__(16) unsigned char sm_raw_trsv[];
  Smem<T>& S = *reinterpret_cast<Smem<T>*>(sm_raw_trsv);
  const int nblk = cdiv_dev(n, NBK);
  const int grp = g0 + blockIdx.y;
  const int c0 = grp * NR;
  const int ncol = min(NR, nrhs - c0);
  int* cnt = done + grp;
  int* pf = pflag + (size_t)grp * nblk;
  const int t = threadIdx.x;
  const int ti = (t % RG) * TM, tj = (t / RG) * TN;  // this thread's tile of the products
  auto blk = [&](int d) { return trans ? nblk - 1 - d : d; };

  if (t == 0) {
    S.ticket = atomicAdd(&tickets[grp], 1) + tkt0;
    S.abort = 0;
  }
  __syncthreads();
  if (S.ticket == 0) {
    // ================================================================ leader
    // Warps 0-7 compute and store each solved block; warp 8 publishes it (fence,
    // release of the counter); warp 9 fetches P_d (after its flag) into Pb, so
    // the serial chain never waits for a global round trip of its own.  Named
    // barriers: 1 + (d & 1) = "P_d is in Pb[d & 1]" (warp 9 arrives, compute
    // waits), 3 + (d & 1) = "Y_d is stored" (compute arrives, warps 8 and 9
    // wait; warp 9 then refills the P buffer of step d), 5 = compute warps only.
    // Each id is reused two steps later, after every participant passed it.
    Leader<T>& M = S.l;
    constexpr int NA = CT + 32, NB = CT + 64;  // participants of barriers A and B
    if (t >= CT + 32) {
      // ---------------------------------------------------- fetching warp
      const int lane = t - CT - 32;
      auto fetch = [&](int d) -> bool {  // P_d -> Pb[d & 1]; false on abort
        if (d >= LAG) {
          if (lane == 0) wait_gt(&pf[d], 0, err, info, S, wait_ns);
          __syncwarp();
          if (ld_shared_volatile(&S.abort)) return false;
        }
        const int b = blk(d), r0 = b * NBK, rows = min(NBK, n - r0);
        constexpr int H = NR > 32 ? 32 : NR;  // columns per batch of independent loads
#pragma unroll
        for (int h = 0; h < NR; h += H) {
          T v[H];
#pragma unroll
          for (int c = 0; c < H; ++c)  // lane = row: one coalesced column per load
            v[c] = (lane < rows && h + c < ncol)
                       ? __ldcg(&B[(size_t)(c0 + h + c) * ldb + r0 + lane])
                       : T(0);
#pragma unroll
          for (int c = 0; c < H; ++c) M.Pb[d & 1][h + c][lane] = v[c];
        }
        return true;
      };
      (void)fetch(0);  // (blocks below LAG need no flag)
      bar_arrive(1, NA);
      if (nblk > 1) {
        (void)fetch(1);
        bar_arrive(2, NA);
      }
      for (int d = 0; d < nblk; ++d) {
        bar_sync(3 + (d & 1), NB);  // step d is done with Pb[d & 1]
        if (d + 2 < nblk) {
          const bool ok = fetch(d + 2);
          bar_arrive(1 + (d & 1), NA);  // (compute sees the abort flag after this)
          if (!ok) {
            bar_sync(3 + ((d + 1) & 1), NB);  // the last step compute finishes
            break;
          }
        }
      }
    } else if (t >= CT) {
      // ---------------------------------------------------- publishing warp
      for (int d = 0; d < nblk; ++d) {
        bar_sync(3 + (d & 1), NB);  // Y_d is stored (by the compute warps)
        if (ld_shared_volatile(&S.abort)) break;
        if (t == CT) {
          __threadfence();
          st_release(cnt, d + 1);
        }
      }
    } else {
      // ---------------------------------------------------- compute warps
      auto prefetch = [&](int d, int buf) {  // the blocks of L that step d needs (L is final)
        const int b = blk(d), r0 = b * NBK, rows = min(NBK, n - r0);
        const T* Lbb = L + (size_t)r0 * lda + r0;
        for (int idx = t; idx < NBK * NBK; idx += CT) {
          const int r = idx % NBK, c = idx / NBK;  // down a column of L
          if (r < rows && c < rows && r >= c)
            cp_async_elem(&M.Ld[buf][r][c], &Lbb[(size_t)c * lda + r]);
          else
            M.Ld[buf][r][c] = T(0);
        }
        for (int e = 1; e < LAG; ++e) {
          if (d - e < 0) continue;
          copy_offdiag<T, NBK + PADL, CT>(M.Lo[buf][e - 1], L, lda, n, r0, rows, blk(d - e), trans, t);
        }
        cp_async_commit();
      };
      prefetch(0, 0);
      for (int d = 0; d < nblk; ++d) {
        const int buf = d & 1;
        const int b = blk(d), rows = min(NBK, n - b * NBK);
        bar_sync(1 + buf, NA);  // P_d is in Pb[buf]
        if (ld_shared_volatile(&S.abort)) break;
        T acc[TM][TN];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] = M.Pb[buf][tj + j][ti + i];
        if (d + 1 < nblk) {
          prefetch(d + 1, buf ^ 1);
          cp_async_wait(1);  // step d's blocks of L
        } else {
          cp_async_wait(0);
        }
        bar_sync(5, CT);
        if (t < NBK) M.rinv[buf][t] = (t < rows) ? T(1) / M.Ld[buf][t][t] : T(0);
        for (int e = 1; e < LAG; ++e)
          if (d - e >= 0)
            block_product<T, NBK + PADL, NR + PADY>(M.Lo[buf][e - 1], M.Yr[(d - e) % (LAG - 1)], ti,
                                                  tj, acc);
        // (every thread read its P_d tile before the barrier above: Ss may overwrite it)
        T(*Ss)[NR + PADY] = reinterpret_cast<T(*)[NR + PADY]>(&M.Pb[buf][0][0]);
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) Ss[ti + i][tj + j] = acc[i][j];
        bar_sync(5, CT);
        if (t < NR) {  // one lane per right-hand side
          const int c = t;
          T s[NBK];
#pragma unroll
          for (int r = 0; r < NBK; ++r) s[r] = Ss[r][c];
          const T(*Ld)[NBK + 1] = M.Ld[buf];
          const T* rinv = M.rinv[buf];  // 0 past the last row: padded rows stay 0
          if (!trans) {
#pragma unroll
            for (int i = 0; i < NBK; ++i) {
              const T y = s[i] * rinv[i];
              s[i] = y;
#pragma unroll
              for (int k = i + 1; k < NBK; ++k) s[k] -= Ld[k][i] * y;
            }
          } else {
#pragma unroll
            for (int i = NBK - 1; i >= 0; --i) {
              const T x = s[i] * rinv[i];
              s[i] = x;
#pragma unroll
              for (int k = 0; k < i; ++k) s[k] -= Ld[i][k] * x;
            }
          }
          T(*Y)[NR + PADY] = M.Yr[d % (LAG - 1)];
#pragma unroll
          for (int r = 0; r < NBK; ++r) Y[r][c] = s[r];
        }
        bar_sync(5, CT);
        {
          const int r0 = b * NBK;
          const T(*Y)[NR + PADY] = M.Yr[d % (LAG - 1)];
          for (int idx = t; idx < NBK * NR; idx += CT) {  // coalesced down the columns
            const int r = idx % NBK, c = idx / NBK;
            if (r < rows && c < ncol) B[(size_t)(c0 + c) * ldb + r0 + r] = Y[r][c];
          }
        }
        bar_arrive(3 + buf, NB);  // Y_d is stored (the next products read Yr after barrier 1/2)
      }
    }
    cp_async_wait(0);  // nothing of ours may land after the CTA ends
    return;
  }

  // ================================================================ helpers
  Helper<T>& H = S.h;
  while (true) {
    const int d = LAG + S.ticket - 1;  // block (in dependency order) of this ticket
    if (d >= nblk) break;
    const int b = blk(d), r0 = b * NBK, rows = min(NBK, n - r0);
    const int ndep = d - LAG + 1;  // dependencies j = 0 .. d-LAG
    auto issue_L = [&](int j) {
      copy_offdiag<T, NBK + PADL, TH>(H.Ls[j % RING], L, lda, n, r0, rows, blk(j), trans, t);
      cp_async_commit();
    };
    T acc[TM][TN];
#pragma unroll
    for (int j = 0; j < TN; ++j)
#pragma unroll
      for (int i = 0; i < TM; ++i)
        acc[i][j] = (ti + i < rows && tj + j < ncol) ? B[(size_t)(c0 + tj + j) * ldb + r0 + ti + i]
                                                     : T(0);
    int pfd = 0;  // blocks of L issued
    for (; pfd < min(ndep, RING - KCH); ++pfd) issue_L(pfd);
    for (int j = 0; j < ndep;) {
      if (t == 0) wait_gt(cnt, j, err, info, S, wait_ns);
      __syncthreads();
      if (S.abort) break;
      const int ready = min(min(S.ready, ndep), j + KCH);
      if (t < CT) {
        constexpr int PER = NBK * NR / CT;  // elements per compute thread and block
        T v[KCH][PER];
#pragma unroll
        for (int q = 0; q < KCH; ++q) {  // all loads first, then the stores
          const int jb = blk(j + q), jr0 = jb * NBK;
#pragma unroll
          for (int e = 0; e < PER; ++e) {
            const int idx = t + CT * e, kk = idx % NBK, c = idx / NBK;
            v[q][e] = (q < ready - j && jr0 + kk < n && c < ncol)
                          ? __ldcg(&B[(size_t)(c0 + c) * ldb + jr0 + kk])
                          : T(0);
          }
        }
#pragma unroll
        for (int q = 0; q < KCH; ++q)
#pragma unroll
          for (int e = 0; e < PER; ++e) {
            const int idx = t + CT * e;
            H.Ys[q][idx % NBK][idx / NBK] = v[q][e];
          }
      }
      for (; pfd < min(ndep, ready + RING - KCH); ++pfd) issue_L(pfd);
      cp_async_wait(pfd - ready);  // blocks j .. ready-1 have landed
      __syncthreads();
      if (t < CT)
        for (int q = 0; q < ready - j; ++q)
          block_product<T, NBK + PADL, NR + PADY>(H.Ls[(j + q) % RING], H.Ys[q], ti, tj, acc);
      __syncthreads();  // the ring slots and Ys are free again
      j = ready;
    }
    cp_async_wait(0);  // no copy of ours may land after the CTA moves on
    if (S.abort) break;
    // P_d over B_d, then the flag
#pragma unroll
    for (int j = 0; j < TN; ++j)
#pragma unroll
      for (int i = 0; i < TM; ++i)
        if (ti + i < rows && tj + j < ncol) B[(size_t)(c0 + tj + j) * ldb + r0 + ti + i] = acc[i][j];
    __syncthreads();
    if (t == 0) {
      __threadfence();
      st_release(&pf[d], 1);
      S.ticket = atomicAdd(&tickets[grp], 1) + tkt0;
    }
    __syncthreads();
  }
}

size_t trsv_sync_ints(int n, int nrhs) {
  // the error word first; then per group of right-hand sides (sized for the
  // smaller, FP64, groups of 16): a ticket counter, a counter of finished
  // blocks and one flag per block (P_d ready)
  const int groups = cdiv(std::max(nrhs, 1), 16);
  return 1 + (size_t)groups * (2 + cdiv(std::max(n, 1), trsv::NBK));
}

template <typename T>
int launch_trsv_persist(int n, int nrhs, const T* L, int lda, T* B, int ldb, int trans,
                        int* sync, int* info, cudaStream_t s, int tkt0) {
  if (n <= 0 || nrhs <= 0) return JMG_OK;
  const int groups = cdiv(nrhs, trsv::Cfg<T>::NR), nblk = cdiv(n, trsv::NBK);
  int* err = sync;
  int* tickets = sync + 1;
  int* done = tickets + groups;
  int* pflag = done + groups;
  // the forward solve clears the error word with the rest; the backward solve
  // keeps it, so that it returns at once after a forward solve that gave up
  JMG_CUDA(cudaMemsetAsync(sync + (trans ? 1 : 0), 0,
                           sizeof(int) * (trsv_sync_ints(n, nrhs) - (trans ? 1 : 0)), s));
  const size_t smem = sizeof(trsv::Smem<T>);
  auto k = k_trsv_persist<T>;
  JMG_TRY(ensure_smem(k, (int)smem));
  // a leader plus one helper per block when they all fit; the tickets keep the
  // dependency order either way.  A leader waits for its helpers, so every
  // launch keeps all of its CTAs resident: groups go in batches of at most
  // slots / 2, each with at least two CTAs.
  int dev = 0, nsm = 152, per_sm = 1;
  JMG_CUDA(cudaGetDevice(&dev));
  JMG_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  JMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, trsv::TH, smem));
  per_sm = per_sm < 1 ? 1 : per_sm;
  const int slots = nsm * per_sm;
  const int want = 1 + std::max(0, nblk - trsv::LAG);
  const int batch = std::max(1, std::min(groups, slots / 2));
  for (int g0 = 0; g0 < groups; g0 += batch) {
    const int gn = std::min(batch, groups - g0);
    const int gx = std::max(2, std::min(want, slots / gn));
    k<<<dim3(gx, gn), trsv::TH, smem, s>>>(n, nrhs, L, lda, B, ldb, trans, g0, tickets, done,
                                           pflag, err, info, g_wait_ns, tkt0);
    JMG_TRY(launched());
  }
  return JMG_OK;
}
template int launch_trsv_persist<float>(int, int, const float*, int, float*, int, int, int*,
                                        int*, cudaStream_t, int);
template int launch_trsv_persist<double>(int, int, const double*, int, double*, int, int, int*,
                                         int*, cudaStream_t, int);

}  // namespace jmg
