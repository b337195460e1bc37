// k_solve.cu -- triangular solves with the FP32 factor of the mixed-precision
// path by a block-inverse chain (paper: "Software design", the solve step of
// potrs; here it applies the preconditioner M = L L^T of the refinement loop).
//
// Blocks of BS = 128 rows, taken in dependency order d = 0, 1, ... (block
// b = d forward, b = nblk-1-d backward).  With the inverse of each diagonal
// block formed once per factorisation,
//
//   forward   Y_b = Li_b P_b - M1_b Y_{b-1} - M2_b Y_{b-2},
//             P_b = B_b - sum_{j <= b-3} L_bj Y_j,
//             Li_b = L_bb^{-1},  Me_b = Li_b L_{b,b-e};
//   backward  X_b = Li_b^T Q_b - N1_b X_{b+1} - N2_b X_{b+2},
//             Q_b = Y_b - sum_{j >= b+3} L_jb^T X_j,  Ne_b = Li_b^T L_{b+e,b}^T,
//
// so the serial chain is products only (no substitution), three per block.
//
// One launch per direction and per group of at most 64 right-hand sides.
// Roles come from an atomic ticket in order: tickets 0 .. G-1 are LEADERS, one
// per 16 right-hand sides, each running the chain above for its columns;
// every later ticket is a HELPER of one block (in dependency order), forming
// P_b for all columns of the launch from the finished blocks as the leaders
// publish them, writing it in place over B_b and raising a flag.  A leader
// waits only for the flags of blocks whose helpers took earlier tickets, and a
// helper only for the leaders, so any number of resident CTAs makes progress.
//
// Data movement is asynchronous copies only:
//  * blocks of L come by TMA from the factor W in a 128-byte-swizzled,
//    row-contiguous ("K-major") image: helper block (b, j) is the box at rows
//    j*128.., columns b*128.. of W.  For the backward solve that is L_jb^T read
//    from the lower triangle; for the forward solve it is L_bj, which
//    sv_prepare mirrors into the upper triangle of W once per factorisation;
//  * the right-hand-side blocks (n x nrhs column-major D, ldd % 32 == 0) come
//    by TMA;
//  * the leaders' matrices Li, Me, Ne are stored by sv_prepare as ready
//    swizzled images (6 per block) and arrive by bulk copies in 16 KB slabs.
// Products are FP32 FMAs on the CUDA cores.  Every wait (flags of other CTAs,
// mbarriers) is bounded by the runtime wait limit; on expiry the CTA raises the
// error word and info = -1 and every role of the CTA leaves its loop.
#include <algorithm>

#include "kernels.h"
#include "tc_ptx.cuh"

namespace jmg {
namespace sv {

constexpr int BS = 128;            // block rows
constexpr int LAG = 3;             // blocks the leader multiplies itself: d-1, d-2
constexpr int CG = 8;              // right-hand sides per leader
constexpr int NMAX = 64;           // right-hand sides per launch
constexpr int TH = 352;            // 8 compute warps, producer, publisher, fetcher
constexpr int NCOMP = 256;
constexpr int TILE_F = BS * BS;    // floats per tile image
constexpr int SLAB_F = 32 * BS;    // floats per 128-byte-wide k-slab (16 KB)
constexpr int NIMG = 6;            // images per block: Li, M1, M2, Li^T, N1, N2
constexpr int LSLOTS = 8;          // leader: slab ring
constexpr int HSLOTS = 2;          // helper: tile ring
// The compute warps split the k range of every product (each warp reads only
// its part of a block, so shared memory is read about once per product) and
// the columns; partial sums meet once per step (leader) or per block (helper).
// Leader: L_KG k-groups of L_KLEN k each x L_CQ column groups of L_CT.
constexpr int L_CQ = CG >= 16 ? 2 : 1, L_CT = CG / L_CQ, L_KG = 8 / L_CQ, L_KLEN = BS / L_KG;
constexpr int L_SLAB_READERS = (32 / L_KLEN) * L_CQ;  // warps that read each slab
// dynamic shared memory: helper = 2 x (64 KB tile + up to 32 KB of Y);
// leader = 8 x 16 KB slabs + 2 P buffers + 3 Y buffers + 3 partial-sum
// buffers (16 columns x 512 B each)
constexpr int YB = NMAX * BS * 4;  // bytes of one helper Y buffer (32 KB)
constexpr int HELPER_BYTES = HSLOTS * (TILE_F * 4 + YB);
constexpr int LEADER_BYTES = LSLOTS * SLAB_F * 4 + (5 + L_KG - 1) * CG * BS * 4;
constexpr int DATA_BYTES = HELPER_BYTES > LEADER_BYTES ? HELPER_BYTES : LEADER_BYTES;
constexpr int SMEM_BYTES = DATA_BYTES + 1024 /* alignment */ + 256 /* barriers */;

// float offset of element (i, k) in a swizzled K-major tile image: slab k/32,
// row i (128 bytes), 16-byte chunk ((k%32)/4) XOR (i%8), word k%4
__host__ __device__ inline int img_off(int i, int k) {
  return (k >> 5) * SLAB_F + i * 32 + ((((k & 31) >> 2) ^ (i & 7)) << 2) + (k & 3);
}

}  // namespace sv

// ============================================================================
// Preparation, once per factorisation
// ============================================================================

// Mirror the strictly-lower 128 x 128 blocks of W into its upper triangle:
// W(c, r) = W(r, c) for every pair of blocks (bi > bj), through 32 x 32 tiles
// in shared memory.  One CTA per block pair.
__global__ void __launch_bounds__(256) k_sv_mirror(int n, float* __restrict__ W, int ldw) {
  __shared__ float t[32][33];
  int bi, bj;
  tri_index(blockIdx.x, bi, bj);
  ++bi;  // strictly lower pairs: tri_index enumerates bj <= bi over nblk-1 rows
  const int r0 = bi * sv::BS, c0 = bj * sv::BS;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int q = 0; q < 16; ++q) {
    const int a = q >> 2, bq = q & 3;
    const int rr = r0 + 32 * a, cc = c0 + 32 * bq;  // source tile: rows rr.., cols cc..
#pragma unroll
    for (int y = ty; y < 32; y += 8) {
      const int r = rr + tx, c = cc + y;  // lanes down a column
      t[y][tx] = (r < n && c < n) ? W[(size_t)c * ldw + r] : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int y = ty; y < 32; y += 8) {
      const int r = rr + y, c = cc + tx;  // destination W(c, r): lanes along c
      if (r < n && c < n) W[(size_t)r * ldw + c] = t[tx][y];
    }
    __syncthreads();
  }
}

// Inverse of each diagonal block in FP64 (in-place lower triangular inversion,
// columns right to left), written as the swizzled images Li_b (slot 0) and
// Li_b^T (slot 3).  Rows and columns past n are the identity.
__global__ void __launch_bounds__(128) k_sv_inv(int n, const float* __restrict__ W, int ldw,
                                                float* __restrict__ SV) {
  extern __shared__ __align__(16) double As[];  // column-major, leading dimension 129
  __shared__ double x[sv::BS];
  constexpr int LD = sv::BS + 1;
  const int b = blockIdx.x, r0 = b * sv::BS, rows = min(sv::BS, n - r0);
  const int t = threadIdx.x;
  for (int c = 0; c < sv::BS; ++c) {
    double v;
    if (t < rows && c < rows)
      v = t >= c ? (double)W[(size_t)(r0 + c) * ldw + r0 + t] : 0.0;
    else
      v = (t == c) ? 1.0 : 0.0;
    As[c * LD + t] = v;
  }
  __syncthreads();
  for (int j = sv::BS - 1; j >= 0; --j) {
    if (t > j) x[t] = As[j * LD + t];
    __syncthreads();
    const double djj = 1.0 / As[j * LD + j];
    if (t > j) {
      double s = 0.0;
      for (int k = j + 1; k <= t; ++k) s = fma(As[k * LD + t], x[k], s);
      As[j * LD + t] = -djj * s;
    }
    __syncthreads();
    if (t == j) As[j * LD + j] = djj;
    __syncthreads();
  }
  float* li = SV + ((size_t)b * sv::NIMG + 0) * sv::TILE_F;
  float* lt = SV + ((size_t)b * sv::NIMG + 3) * sv::TILE_F;
  for (int f = t; f < sv::TILE_F; f += blockDim.x) {
    // decode the image position f -> (i, k)
    const int s = f / sv::SLAB_F, rem = f % sv::SLAB_F, i = rem >> 5, q = rem & 31;
    const int k = 32 * s + (((q >> 2) ^ (i & 7)) << 2) + (q & 3);
    li[f] = (float)As[k * LD + i];  // Li(i, k)
    lt[f] = (float)As[i * LD + k];  // Li(k, i)
  }
}

// The chain's coupling matrices, FP32 products of 128 x 128 blocks:
//   slot 1/2: M_e = Li_b L_{b,b-e}          (forward, e = 1, 2)
//   slot 4/5: N_e = Li_b^T L_{b+e,b}^T      (backward, e = 1, 2)
// blockIdx.x = block b, blockIdx.y = 0..3 -> (M1, M2, N1, N2).  Li / Li^T come
// from the images written by k_sv_inv.
__global__ void __launch_bounds__(256) k_sv_couple(int n, const float* __restrict__ W, int ldw,
                                                   float* __restrict__ SV) {
  extern __shared__ __align__(16) float sm_couple[];
  float* Ai = sm_couple;                // [i][m] dense, leading dimension 132
  float* Bk = sm_couple + 128 * 132;    // [m][k] dense, leading dimension 132
  constexpr int LD = 132;
  const int b = blockIdx.x, which = blockIdx.y;
  const int nblk = cdiv_dev(n, sv::BS);
  const int e = 1 + (which & 1);
  const bool fwd = which < 2;
  const int nb = fwd ? b - e : b + e;  // the neighbouring block
  float* out = SV + ((size_t)b * sv::NIMG + (fwd ? e : 3 + e)) * sv::TILE_F;
  const int t = threadIdx.x;
  if (nb < 0 || nb >= nblk) {  // no neighbour: the image stays unused; clear it
    for (int f = t; f < sv::TILE_F; f += blockDim.x) out[f] = 0.0f;
    return;
  }
  const float* li = SV + ((size_t)b * sv::NIMG + (fwd ? 0 : 3)) * sv::TILE_F;
  for (int f = t; f < sv::TILE_F; f += blockDim.x) {
    const int i = f >> 7, m = f & 127;
    Ai[i * LD + m] = li[sv::img_off(i, m)];
  }
  const int r0 = b * sv::BS, q0 = nb * sv::BS;
  for (int f = t; f < sv::TILE_F; f += blockDim.x) {
    // lanes along the contiguous index of W in either case
    const int k = fwd ? f >> 7 : f & 127, m = fwd ? f & 127 : f >> 7;
    float v;
    if (fwd)  // L_{b,b-e}(m, k) = W(r0 + m, q0 + k)
      v = (r0 + m < n && q0 + k < n) ? W[(size_t)(q0 + k) * ldw + r0 + m] : 0.0f;
    else  // L_{b+e,b}^T(m, k) = W(q0 + k, r0 + m)
      v = (r0 + m < n && q0 + k < n) ? W[(size_t)(r0 + m) * ldw + q0 + k] : 0.0f;
    Bk[m * LD + k] = v;
  }
  __syncthreads();
  // 256 threads x (8 rows x 8 columns): rows ty*8.., columns tx + 16 q
  const int tx = t & 15, ty = t >> 4;
  float acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[a][c] = 0.0f;
  for (int m = 0; m < sv::BS; ++m) {
    float av[8], bv[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) av[a] = Ai[(ty * 8 + a) * LD + m];
#pragma unroll
    for (int c = 0; c < 8; ++c) bv[c] = Bk[m * LD + tx + 16 * c];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int c = 0; c < 8; ++c) acc[a][c] = fmaf(av[a], bv[c], acc[a][c]);
  }
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int c = 0; c < 8; ++c) out[sv::img_off(ty * 8 + a, tx + 16 * c)] = acc[a][c];
}

// ============================================================================
// The solve
// ============================================================================
namespace sv {

struct Ctl {
  int ticket, abort;
  int copied;  // leader: steps whose Y the publisher has copied to global memory
};

JMG_DEV int ld_acq(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
JMG_DEV void st_rel(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
JMG_DEV void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}
JMG_DEV void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// Barrier of the compute warps that also ORs a flag across them: every compute
// thread gets the same answer, so they all leave a loop at the same step.
JMG_DEV bool bar_or(int id, int count, bool v) {
  int r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.b32 q, %1, 0;\n\t"
      "bar.red.or.pred p, %2, %3, q;\n\t"
      "selp.b32 %0, 1, 0, p;\n\t}"
      : "=r"(r)
      : "r"((int)v), "r"(id), "r"(count)
      : "memory");
  return r != 0;
}

JMG_DEV void bar_sync_named(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Raise the CTA's abort flag and the launch's error word (and info).
JMG_DEV void raise(Ctl& C, int* err, int* info) {
  C.abort = 1;
  atomicExch(err, JMG_ERR_TIMEOUT);
  if (info) atomicCAS(info, 0, -1);
}

// Bounded wait for an mbarrier phase.  Gives up (false) when the CTA aborts,
// another CTA raised the error word, or `limit` ns pass; in the last two cases
// it raises the CTA's abort flag itself, so every role of the CTA stops soon.
JMG_DEV bool wait_bar(uint64_t* bar, uint32_t parity, Ctl& C, int* err, int* info,
                      uint64_t limit) {
  if (tc::mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  while (true) {
    if (tc::mbar_try_wait(bar, parity)) return true;
    if (ld_shared_volatile(&C.abort)) return false;
    if (*(volatile const int*)err || globaltimer_ns() - t0 > limit) {
      raise(C, err, info);
      return false;
    }
  }
}

// Bounded wait until every one of the G ints at p is >= v (acquire); on
// failure as wait_bar.
JMG_DEV bool wait_ge(const int* p, int G, int v, Ctl& C, int* err, int* info, uint64_t limit) {
  uint64_t t0 = 0;
  for (int g = 0; g < G; ++g) {
    while (ld_acq(p + g) < v) {
      if (t0 == 0) t0 = globaltimer_ns();
      if (ld_shared_volatile(&C.abort)) return false;
      if (*(volatile const int*)err || globaltimer_ns() - t0 > limit) {
        raise(C, err, info);
        return false;
      }
      __nanosleep(32);
    }
  }
  return true;
}

// acc[r][c] += sign * sum over chunks ch0 .. ch1-1 (4 k each) of one 32-wide
// k-slab of T(i, k) * V(k, c): T a swizzled tile slab (rows i = lane + 32 r),
// V column-major with leading dimension BS (columns c0 + c).  Only rows r in
// [r_lo, r_hi] are formed: a lower triangular T has no entries in slab s above
// row group s, an upper triangular one none below it.
template <int CT, bool NEG>
JMG_DEV void slab_product(const float* __restrict__ slab, const float* __restrict__ V, int ks,
                          int ch0, int ch1, int c0, int lane, int r_lo, int r_hi,
                          float (&acc)[4][CT]) {
  const float sg = NEG ? -1.0f : 1.0f;  // folds into the multiply-adds
#pragma unroll 1
  for (int ch = ch0; ch < ch1; ++ch) {
    float4 a[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int i = lane + 32 * r;
      a[r] = *reinterpret_cast<const float4*>(slab + i * 32 + ((ch ^ (i & 7)) << 2));
    }
#pragma unroll
    for (int c = 0; c < CT; ++c) {
      const float4 v = *reinterpret_cast<const float4*>(V + (size_t)(c0 + c) * BS + ks + 4 * ch);
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        if (r < r_lo || r > r_hi) continue;
        float t = acc[r][c];
        t = fmaf(sg * a[r].x, v.x, t);
        t = fmaf(sg * a[r].y, v.y, t);
        t = fmaf(sg * a[r].z, v.z, t);
        t = fmaf(sg * a[r].w, v.w, t);
        acc[r][c] = t;
      }
    }
  }
}

}  // namespace sv

// CT: helper columns per compute warp (N_pad = 8 CT right-hand sides per launch).
template <int CT>
__global__ void __launch_bounds__(sv::TH, 1)
    k_sv_solve(const __grid_constant__ CUtensorMap tmW, const __grid_constant__ CUtensorMap tmDh,
               const __grid_constant__ CUtensorMap tmDl, int n, int ncol, int cb,
               const float* __restrict__ SV, float* __restrict__ D, int ldd, int trans,
               int* __restrict__ sync, int* __restrict__ info, unsigned long long wait_ns) {
  using namespace sv;
  extern __shared__ __align__(1024) unsigned char sm_raw_sv[];
  unsigned char* sm =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(sm_raw_sv) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + DATA_BYTES);
  __shared__ Ctl C;
  const int nblk = cdiv_dev(n, BS);
  const int G = cdiv_dev(ncol, CG);
  int* err = sync;
  int* tickets = sync + 1;
  int* cnt = sync + 2;           // G leader counters
  int* pflag = sync + 2 + G;     // one flag per block (dependency order)
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  if (info && *(volatile int*)info != 0) return;
  if (*(volatile int*)err != 0) return;
  auto blk = [&](int d) { return trans ? nblk - 1 - d : d; };

  if (t == 0) {
    C.ticket = atomicAdd(tickets, 1);
    C.abort = 0;
    C.copied = 0;
  }
  __syncthreads();
  const int ticket = C.ticket;

  if (ticket < G) {
    // ====================================================================== leader
    const int g = ticket, c0 = g * CG;
    const int ncg = min(CG, ncol - c0);
    float* slabs = reinterpret_cast<float*>(sm);
    float* Ps = slabs + LSLOTS * SLAB_F;  // 2 x [CG][BS]
    float* Yr = Ps + 2 * CG * BS;         // 3 x [CG][BS]
    float* red = Yr + 3 * CG * BS;        // (L_KG - 1) x [CG][BS] partial sums
    uint64_t* sfull = bars;
    uint64_t* sempty = bars + LSLOTS;
    uint64_t* pfull = bars + 2 * LSLOTS;
    uint64_t* pempty = pfull + 2;
    uint64_t* ystored = pempty + 2;
    if (t == 0) {
      for (int s = 0; s < LSLOTS; ++s) {
        tc::mbar_init(&sfull[s], 1);
        tc::mbar_init(&sempty[s], L_SLAB_READERS);
      }
      for (int s = 0; s < 2; ++s) {
        tc::mbar_init(&pfull[s], 1);
        tc::mbar_init(&pempty[s], 8);
      }
      tc::mbar_init(ystored, L_CQ);       // the warps of k-group 0 store Y
      tc::fence_mbar_init();
    }
    __syncthreads();
    // images of step d, in the order the compute warps use them
    auto tiles_of = [&](int d, int* idx) {
      int m = 0;
      idx[m++] = trans ? 3 : 0;
      if (d >= 2) idx[m++] = trans ? 5 : 2;
      if (d >= 1) idx[m++] = trans ? 4 : 1;
      return m;
    };
    if (warp == 8) {
      // ------------------------------------------------------------ producer
      if (lane == 0) {
        long long gs = 0;
        bool ok = true;
        for (int d = 0; d < nblk && ok; ++d) {
          const int b = blk(d);
          int idx[3];
          const int m = tiles_of(d, idx);
          for (int q = 0; q < m && ok; ++q) {
            const float* src = SV + ((size_t)b * NIMG + idx[q]) * TILE_F;
            for (int s = 0; s < 4; ++s, ++gs) {
              const int slot = (int)(gs % LSLOTS);
              if (gs >= LSLOTS &&
                  !wait_bar(&sempty[slot], (uint32_t)((gs / LSLOTS) - 1) & 1, C, err, info, wait_ns)) {
                ok = false;
                break;
              }
              tc::mbar_expect_tx(&sfull[slot], SLAB_F * 4);
              bulk_load(slabs + slot * SLAB_F, src + s * SLAB_F, SLAB_F * 4, &sfull[slot]);
            }
          }
        }
        if (!ok) raise(C, err, info);
        // let every copy issued land before the CTA ends
        for (long long q = (gs > LSLOTS ? gs - LSLOTS : 0); q < gs; ++q)
          (void)tc::mbar_wait(&sfull[q % LSLOTS], (uint32_t)(q / LSLOTS) & 1, wait_ns);
      }
    } else if (warp == 10) {
      // ------------------------------------------------------------ fetcher of P_b
      if (lane == 0) {
        int issued = 0;
        bool ok = true;
        for (int d = 0; d < nblk; ++d) {
          const int b = blk(d), buf = d & 1;
          if (d >= 2 && !wait_bar(&pempty[buf], (uint32_t)((d >> 1) - 1) & 1, C, err, info, wait_ns)) {
            ok = false;
            break;
          }
          if (d >= LAG) {
            if (!wait_ge(&pflag[d], 1, 1, C, err, info, wait_ns)) {
              ok = false;
              break;
            }
            fence_proxy_async_global();
          }
          tc::mbar_expect_tx(&pfull[buf], CG * BS * 4);
          tc::tma_load_2d(Ps + buf * CG * BS, &tmDl, b * BS, cb + c0, &pfull[buf]);
          ++issued;
        }
        if (!ok) raise(C, err, info);
        for (int d = (issued > 2 ? issued - 2 : 0); d < issued; ++d)
          (void)tc::mbar_wait(&pfull[d & 1], (uint32_t)(d >> 1) & 1, wait_ns);
      }
    } else if (warp == 9) {
      // ------------------------------------------------------------ publisher
      // Y_b goes from shared memory to global memory here, off the chain: every
      // lane fences its own stores, then the counter is released
      for (int d = 0; d < nblk; ++d) {
        bool ok = true;
        if (lane == 0) ok = wait_bar(ystored, (uint32_t)d & 1, C, err, info, wait_ns);
        if (!__shfl_sync(0xffffffffu, ok ? 1 : 0, 0)) break;
        const float* Yw = Yr + (d % 3) * CG * BS;
        const int r0 = blk(d) * BS;
        for (int c = 0; c < ncg; ++c)
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const int i = lane + 32 * r;
            if (r0 + i < n) D[(size_t)(cb + c0 + c) * ldd + r0 + i] = Yw[c * BS + i];
          }
        __threadfence();
        __syncwarp();
        if (lane == 0) {
          st_rel(&cnt[g], d + 1);
          *(volatile int*)&C.copied = d + 1;  // Yr[d % 3] may be overwritten
        }
      }
    } else {
      // ------------------------------------------------------------ compute warps
      const int kg = warp / L_CQ;           // k-group: k in [kg L_KLEN, (kg + 1) L_KLEN)
      const int cw = (warp % L_CQ) * L_CT;  // this warp's columns (of the leader's CG)
      const int ks = kg * L_KLEN;
      const int sl = ks >> 5, ch0 = (ks & 31) >> 2, ch1 = ch0 + L_KLEN / 4;
      long long gs = 0;
      for (int d = 0; d < nblk; ++d) {
        const int b = blk(d), buf = d & 1;
        bool ok = wait_bar(&pfull[buf], (uint32_t)(d >> 1) & 1, C, err, info, wait_ns);
        float acc[4][L_CT];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < L_CT; ++c) acc[r][c] = 0.0f;
        int idx[3];
        const int m = tiles_of(d, idx);
        for (int q = 0; q < m; ++q, gs += 4) {
          const float* V = q == 0 ? Ps + buf * CG * BS
                                  : Yr + ((d - (q == 1 && m == 3 ? 2 : 1)) % 3) * CG * BS;
          const long long gk = gs + sl;  // the slab of the block holding this k range
          const int slot = (int)(gk % LSLOTS);
          if (ok) ok = wait_bar(&sfull[slot], (uint32_t)(gk / LSLOTS) & 1, C, err, info, wait_ns);
          // Li (lower): row groups sl..3 of slab sl; Li^T (upper): 0..sl
          if (ok && q == 0)
            slab_product<L_CT, true>(slabs + slot * SLAB_F, V, 32 * sl, ch0, ch1, cw, lane,
                                     trans ? 0 : sl, trans ? sl : 3, acc);
          else if (ok)
            slab_product<L_CT, false>(slabs + slot * SLAB_F, V, 32 * sl, ch0, ch1, cw, lane, 0,
                                      3, acc);
          __syncwarp();
          if (lane == 0) {
            tc::mbar_arrive(&sempty[slot]);
            if (q == 0) tc::mbar_arrive(&pempty[buf]);  // P_b is no longer needed
          }
        }
        // acc (summed over the k-groups) = -(Li P) + M2 Y_{d-2} + M1 Y_{d-1} = -Y_b
        if (kg > 0) {
          float* R = red + (kg - 1) * CG * BS;
#pragma unroll
          for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < L_CT; ++c) R[(cw + c) * BS + lane + 32 * r] = acc[r][c];
        }
        bar_sync_named(1, NCOMP);
        if (kg == 0) {
          // Yr[d % 3] last held Y of step d-3: the publisher must have copied it
          if (d >= 3 && ok) {
            if (lane == 0) {
              const uint64_t t0 = globaltimer_ns();
              while (ld_shared_volatile(&C.copied) < d - 2) {
                if (ld_shared_volatile(&C.abort)) break;
                if (*(volatile const int*)err || globaltimer_ns() - t0 > wait_ns) {
                  raise(C, err, info);
                  break;
                }
              }
            }
            __syncwarp();
          }
          float* Yw = Yr + (d % 3) * CG * BS;
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const int i = lane + 32 * r;
#pragma unroll
            for (int c = 0; c < L_CT; ++c) {
              float v = acc[r][c];
#pragma unroll
              for (int q = 0; q < L_KG - 1; ++q) v += red[q * CG * BS + (cw + c) * BS + i];
              Yw[(cw + c) * BS + i] = -v;
            }
          }
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(ystored);
        }
        // all compute warps agree whether to go on (and Y_b and the partial
        // buffers are settled before the next step)
        if (bar_or(1, NCOMP, !ok || ld_shared_volatile(&C.abort))) {
          if (t == 0 && !ld_shared_volatile(&C.abort)) raise(C, err, info);
          break;
        }
      }
    }
    return;
  }

  // ======================================================================== helpers
  // compute warps: CQH column groups of CTH columns x KGH k-groups of KLEN
  constexpr int NP = 8 * CT;                 // right-hand sides of this launch, padded
  constexpr int CTH = NP < 16 ? NP : 16;
  constexpr int CQH = NP / CTH, KGH = 8 / CQH, KLEN = BS / KGH;
  float* ringL = reinterpret_cast<float*>(sm);                      // 2 x 64 KB
  float* ringY = ringL + HSLOTS * TILE_F;                           // 2 x [NMAX][BS]
  float* red = ringL;  // partial sums at the end of a block (the ring is idle then)
  uint64_t* full = bars;
  uint64_t* empty = bars + HSLOTS;
  uint64_t* hdone = bars + 2 * HSLOTS;
  uint64_t* tnext = hdone + 1;
  __shared__ int s_go;
  if (t == 0) {
    for (int s = 0; s < HSLOTS; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 8);
    }
    tc::mbar_init(hdone, 8);
    tc::mbar_init(tnext, 1);
    tc::fence_mbar_init();
  }
  __syncthreads();
  if (warp > 8) return;  // the publisher and fetcher warps have no helper duty
  long long gq = 0;      // tiles issued (producer) / consumed (compute), all tickets
  int my_ticket = ticket;
  for (int round = 0;; ++round) {
    const int d = my_ticket - G + LAG;  // block (dependency order) of this ticket
    if (d >= nblk) break;
    const int b = blk(d), r0 = b * BS;
    const int ndep = d - LAG + 1;  // dependencies in order 0 .. d-LAG
    if (warp == 8) {
      // ------------------------------------------------------------ producer
      bool ok = true;
      if (lane == 0) {
        for (int q = 0; q < ndep; ++q) {
          const int slot = (int)(gq % HSLOTS);
          if (gq >= HSLOTS &&
              !wait_bar(&empty[slot], (uint32_t)((gq / HSLOTS) - 1) & 1, C, err, info, wait_ns)) {
            ok = false;
            break;
          }
          const int j = blk(q);
          // one phase per slot: both copies' bytes, then the arrival once the
          // second copy is issued (the block of L does not wait for the chain)
          tc::mbar_expect_tx_only(&full[slot], TILE_F * 4 + NP * BS * 4);
          for (int s = 0; s < 4; ++s)
            tc::tma_load_2d(ringL + slot * TILE_F + s * SLAB_F, &tmW, j * BS + 32 * s, r0,
                            &full[slot]);
          ok = wait_ge(cnt, G, q + 1, C, err, info, wait_ns);
          if (ok) fence_proxy_async_global();
          // (on failure the block is still copied, so that the phase completes
          // and no copy is left in flight when the CTA ends)
          tc::tma_load_2d(ringY + slot * (NMAX * BS), &tmDh, j * BS, cb, &full[slot]);
          tc::mbar_arrive(&full[slot]);
          ++gq;
          if (!ok) break;
        }
        // P_b is stored once the compute warps arrive: publish it, take the next ticket
        if (ok) ok = wait_bar(hdone, (uint32_t)round & 1, C, err, info, wait_ns);
        if (ok) {
          __threadfence();  // the compute warps' stores of P_b, observed through hdone
          st_rel(&pflag[d], 1);
          C.ticket = atomicAdd(tickets, 1);
        }
        s_go = ok ? 1 : 0;
        tc::mbar_arrive(tnext);  // release the compute warps either way
      }
      __syncwarp();
      gq = __shfl_sync(0xffffffffu, gq, 0);
      if (!__shfl_sync(0xffffffffu, ok ? 1 : 0, 0)) break;
      my_ticket = C.ticket;
    } else {
      // ------------------------------------------------------------ compute warps
      const int cq = warp % CQH, kg = warp / CQH;
      const int cw = cq * CTH, k0 = kg * KLEN;
      float acc[4][CTH];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int i = lane + 32 * r;
#pragma unroll
        for (int c = 0; c < CTH; ++c)
          acc[r][c] = (kg == 0 && r0 + i < n && cw + c < ncol)
                          ? D[(size_t)(cb + cw + c) * ldd + r0 + i]
                          : 0.0f;
      }
      bool ok = true;
      for (int q = 0; q < ndep; ++q, ++gq) {
        const int slot = (int)(gq % HSLOTS);
        if (ok) ok = wait_bar(&full[slot], (uint32_t)(gq / HSLOTS) & 1, C, err, info, wait_ns);
        if (ok) {
          const float* Lt = ringL + slot * TILE_F;
          const float* Yt = ringY + slot * (NMAX * BS);
#pragma unroll
          for (int kk = k0; kk < k0 + KLEN; kk += 32) {  // P -= L_bj Y_j over this k range
            const int ch0 = (kk & 31) >> 2;
            const int ch1 = KLEN >= 32 ? 8 : ch0 + KLEN / 4;
            slab_product<CTH, true>(Lt + (kk >> 5) * SLAB_F, Yt, kk & ~31, ch0, ch1, cw, lane,
                                    0, 3, acc);
          }
        }
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&empty[slot]);
      }
      // partial sums of the k-groups meet in shared memory, over the tile ring:
      // once every compute warp has left the ring it is idle (the producer waits
      // for hdone before it copies again)
      bar_sync_named(2, NCOMP);
      if (ok && kg > 0) {
        float* R = red + (kg - 1) * NP * BS;
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < CTH; ++c) R[(cw + c) * BS + lane + 32 * r] = acc[r][c];
      }
      const bool bad = bar_or(2, NCOMP, !ok || ld_shared_volatile(&C.abort));
      if (!bad && kg == 0) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int i = lane + 32 * r;
#pragma unroll
          for (int c = 0; c < CTH; ++c) {
            float v = acc[r][c];
            for (int q = 0; q < KGH - 1; ++q) v += red[q * NP * BS + (cw + c) * BS + i];
            if (r0 + i < n && cw + c < ncol) D[(size_t)(cb + cw + c) * ldd + r0 + i] = v;
          }
        }
        __threadfence();  // each lane's own stores of P_b, before the hand-off
      }
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(hdone);
      // the producer's verdict and the next ticket, agreed by every compute warp
      const bool got = wait_bar(tnext, (uint32_t)round & 1, C, err, info, wait_ns);
      if (bar_or(2, NCOMP, bad || !got || !ld_shared_volatile(&s_go))) break;
      my_ticket = C.ticket;
    }
  }
  // let every copy this CTA issued land before it ends
  if (warp == 8 && lane == 0)
    for (long long q = (gq > HSLOTS ? gq - HSLOTS : 0); q < gq; ++q)
      (void)tc::mbar_wait(&full[q % HSLOTS], (uint32_t)(q / HSLOTS) & 1, wait_ns);
}

// ============================================================================
// Host side
// ============================================================================
size_t sv_image_bytes(int n) {
  return (size_t)cdiv(std::max(n, 1), sv::BS) * sv::NIMG * sv::TILE_F * sizeof(float);
}

size_t sv_sync_ints(int n, int nrhs) {
  (void)nrhs;  // one launch at a time reuses the same words
  return 2 + sv::NMAX / sv::CG + (size_t)cdiv(std::max(n, 1), sv::BS);
}

int sv_prepare(int n, float* W, int ldw, float* SV, cudaStream_t s) {
  if (n <= 0) return JMG_OK;
  if (ldw % 32 || (reinterpret_cast<uintptr_t>(W) & 15) || (reinterpret_cast<uintptr_t>(SV) & 255))
    return JMG_ERR_ALIGN;
  const int nblk = cdiv(n, sv::BS);
  if (nblk > 1) {
    k_sv_mirror<<<(unsigned)tri_tiles(nblk - 1), 256, 0, s>>>(n, W, ldw);
    JMG_TRY(launched());
  }
  const int inv_smem = sv::BS * (sv::BS + 1) * (int)sizeof(double);
  JMG_TRY(ensure_smem(k_sv_inv, inv_smem));
  k_sv_inv<<<nblk, 128, inv_smem, s>>>(n, W, ldw, SV);
  JMG_TRY(launched());
  const int cp_smem = 2 * 128 * 132 * (int)sizeof(float);
  JMG_TRY(ensure_smem(k_sv_couple, cp_smem));
  k_sv_couple<<<dim3(nblk, 4), 256, cp_smem, s>>>(n, W, ldw, SV);
  return launched();
}

template <int CT>
static int sv_launch(const CUtensorMap& mw, const CUtensorMap& mdh, const CUtensorMap& mdl, int n,
                     int ncol, int cb, const float* SV, float* D, int ldd, int trans, int* sync,
                     int* info, int grid, cudaStream_t s) {
  JMG_TRY(ensure_smem(k_sv_solve<CT>, sv::SMEM_BYTES));
  k_sv_solve<CT><<<grid, sv::TH, sv::SMEM_BYTES, s>>>(mw, mdh, mdl, n, ncol, cb, SV, D, ldd, trans,
                                                      sync, info, g_wait_ns);
  return launched();
}

int sv_solve(int n, int nrhs, const float* W, int ldw, const float* SV, float* D, int ldd,
             int trans, int* sync, int* info, cudaStream_t s) {
  if (n <= 0 || nrhs <= 0) return JMG_OK;
  if (ldw % 32 || ldd % 32 || (reinterpret_cast<uintptr_t>(W) & 15) ||
      (reinterpret_cast<uintptr_t>(D) & 15) || (reinterpret_cast<uintptr_t>(SV) & 15))
    return JMG_ERR_ALIGN;
  const int nblk = cdiv(n, sv::BS);
  int dev = 0, nsm = 152;
  JMG_CUDA(cudaGetDevice(&dev));
  JMG_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  CUtensorMap mw, mdl;
  JMG_TRY(make_tmap_2d(&mw, W, (unsigned long long)n, (unsigned long long)n,
                       (unsigned long long)ldw * 4, 32, sv::BS, CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                       CU_TENSOR_MAP_SWIZZLE_128B));
  JMG_TRY(make_tmap_2d(&mdl, D, (unsigned long long)n, (unsigned long long)nrhs,
                       (unsigned long long)ldd * 4, sv::BS, sv::CG,
                       CU_TENSOR_MAP_DATA_TYPE_FLOAT32, CU_TENSOR_MAP_SWIZZLE_NONE));
  for (int cb = 0; cb < nrhs; cb += sv::NMAX) {
    const int ncol = std::min(sv::NMAX, nrhs - cb);
    const int ct = ncol > 32 ? 8 : ncol > 16 ? 4 : ncol > 8 ? 2 : 1;
    CUtensorMap mdh;
    JMG_TRY(make_tmap_2d(&mdh, D, (unsigned long long)n, (unsigned long long)nrhs,
                         (unsigned long long)ldd * 4, sv::BS, 8 * ct,
                         CU_TENSOR_MAP_DATA_TYPE_FLOAT32, CU_TENSOR_MAP_SWIZZLE_NONE));
    // the error word survives every launch but the first forward one
    const int keep = (trans || cb > 0) ? 1 : 0;
    JMG_CUDA(cudaMemsetAsync(sync + keep, 0, sizeof(int) * (sv_sync_ints(n, nrhs) - keep), s));
    const int G = cdiv(ncol, sv::CG);
    const int helpers = std::max(0, nblk - sv::LAG);
    const int grid = std::max(G, std::min(nsm, G + helpers));
    int st;
    switch (ct) {
      case 8: st = sv_launch<8>(mw, mdh, mdl, n, ncol, cb, SV, D, ldd, trans, sync, info, grid, s); break;
      case 4: st = sv_launch<4>(mw, mdh, mdl, n, ncol, cb, SV, D, ldd, trans, sync, info, grid, s); break;
      case 2: st = sv_launch<2>(mw, mdh, mdl, n, ncol, cb, SV, D, ldd, trans, sync, info, grid, s); break;
      default: st = sv_launch<1>(mw, mdh, mdl, n, ncol, cb, SV, D, ldd, trans, sync, info, grid, s); break;
    }
    JMG_TRY(st);
  }
  return JMG_OK;
}

}  // namespace jmg
