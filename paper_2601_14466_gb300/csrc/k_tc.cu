// k_tc.cu -- trailing-matrix update of the mixed-precision Cholesky factorisation
// on the 5th-generation tensor cores (tcgen05, sm_103a).
//
//     C[i, j] -= sum_k PA[i, k] * PB[j, k]        (lower-triangle tiles only)
//
// PA / PB are the panel L21 split into 16-bit words (BF16 or FP16) and laid out
// row-major, K contiguous, so both operands are "K-major".  With several words
// the pairs (hi*hi, hi*lo, lo*hi, ...) are concatenated along K, so one GEMM with
// K' = pairs * kb applies all of them to the same FP32 accumulator.
//
// Persistent: one CTA per SM walks the 128 x 128 output tiles of the lower
// trapezoid, 320 threads:
//   warp 0 (one lane): TMA producer -- 128 x 64 tiles of PA and PB per stage,
//                       128-byte swizzle, mbarrier transaction counts;
//   warp 1 (one lane): MMA issuer   -- tcgen05.mma kind::f16, M=128 N=128 K=16
//                       (or kind::f8f6f4, K=32), FP32 accumulators in TMEM, two
//                       of them so the MMAs of the next tile overlap the
//                       epilogue of this one;
//   warps 2-9:         epilogue     -- tcgen05.ld 32 lanes x 32 columns, then
//                       C -= acc with coalesced column accesses (lane = row);
//                       with FP8 every 128-deep chunk of K carries its own
//                       power-of-two tile scales, so the chunks accumulate in
//                       TMEM one at a time and the epilogue adds them scaled;
//                       two warps per TMEM lane quarter, 64 columns each.  They
//                       prefetch the next tile's C into L2 before they drain
//                       this one, so the read-modify-write of C meets L2.
// Every mbarrier wait is bounded by `wait_ns` (globaltimer); on expiry the
// kernel raises *err, drains its own copies, frees TMEM and returns without
// touching C.
//
// The paper runs these updates inside cuSOLVERMp (FP32/FP64, "Software
// design"); the split-word tensor-core form is this library's own design.
#include <algorithm>

#include "kernels.h"
#include "tc_ptx.cuh"

namespace jmg {
namespace tc {

constexpr int BM = 128, BN = 128, BK = 64;  // BK: 64 x 16-bit = one 128-byte swizzle row
constexpr int TILE_BYTES = BM * BK * 2;  // 16 KiB
constexpr int STAGE_BYTES = 2 * TILE_BYTES;

// Tile b of the lower trapezoid {(ti, tj): tj <= ti < TI, tj < TJ}, enumerated
// row by row: the first TJ rows form a triangle, every later row has TJ tiles.
JMG_DEV void trap_index(int b, int TJ, int& ti, int& tj) {
  const int tri = TJ * (TJ + 1) / 2;
  if (b < tri) {
    tri_index(b, ti, tj);
  } else {
    const int q = b - tri;
    ti = TJ + q / TJ;
    tj = q % TJ;
  }
}


// Persistent, warp-specialised update.  320 threads:
//   warp 0: TMA producer (one lane), warp 1: MMA issuer (one lane),
//   warps 2-9: epilogue; warp w reads TMEM lanes 32 (w % 4) .. +31, columns
//   64 ((w - 2) / 4) .. +63 of the accumulator.
// Two TMEM accumulators (2 x 128 columns): the MMAs of tile i+1 run while the
// epilogue drains tile i.  Barriers: full/empty per smem stage, acc_full /
// acc_empty per accumulator.
constexpr int PSTAGES = 6;
constexpr int PTHREADS = 320;
constexpr int EPI_WARPS = 8;
constexpr int PSMEM_BYTES = PSTAGES * STAGE_BYTES + 1024 + 512;
constexpr uint32_t PTMEM_COLS = 256;

// KIND 0: kind::f16 (BF16 / FP16 words, 64 elements = 128 bytes per stage row,
//         K = 16 per instruction); ab_fmt selects BF16 (1) or FP16 (0).
// KIND 1: kind::f8f6f4 with E4M3 operands (128 elements per stage row, K = 32
//         per instruction); the accumulator of tile (ti, tj) is scaled by
//         2^-(exps[ti] + exps[tj]) in the epilogue (power-of-two tile scales).
// Both step 32 bytes along the swizzled row per instruction.
template <int KIND>
__global__ void __launch_bounds__(PTHREADS, 1)
    k_syrk_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              float* __restrict__ C, int ldc, int m, int ncols, int kext, int ab_fmt,
              int ntiles, int TJ, const signed char* __restrict__ exps, int lde, int cstages,
              int* __restrict__ err, unsigned long long wait_ns, int hold_producer) {
  extern __shared__ __align__(1024) unsigned char sm_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(sm_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + PSTAGES * STAGE_BYTES);
  uint64_t* empty = full + PSTAGES;
  uint64_t* acc_full = empty + PSTAGES;
  uint64_t* acc_empty = acc_full + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);
  __shared__ int s_fail;

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int nk = kext / (KIND == 0 ? BK : 2 * BK);  // stage = 128 bytes of K per row

  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int s = 0; s < PSTAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&acc_full[a], 1);
      mbar_init(&acc_empty[a], EPI_WARPS);
    }
    fence_mbar_init();
    prefetch_tmap(&tmA);
    prefetch_tmap(&tmB);
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, PTMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  long long issued = 0;  // producer: stage loads issued (global k-iteration count)
  if (warp == 0) {
    // hold_producer (a test hook) keeps the producer idle: nothing ever completes
    // the first stage, so the MMA issuer's bounded wait runs out and the kernel
    // takes its abort path
    if (lane == 0 && !hold_producer) {
      long long g = 0;
      for (int b = blockIdx.x; b < ntiles; b += gridDim.x) {
        int ti, tj;
        trap_index(b, TJ, ti, tj);
        for (int kb = 0; kb < nk; ++kb, ++g) {
          const int s = (int)(g % PSTAGES);
          if (g >= PSTAGES && !mbar_wait(&empty[s], (uint32_t)((g / PSTAGES) - 1) & 1, wait_ns)) {
            atomicExch(&s_fail, 1);
            break;
          }
          if (ld_shared_volatile(&s_fail)) break;
          unsigned char* sa = smem + s * STAGE_BYTES;
          mbar_expect_tx(&full[s], STAGE_BYTES);
          const int kx = kb * (KIND == 0 ? BK : 2 * BK);  // element coordinate of the stage
          tma_load_2d(sa, &tmA, kx, ti * BM, &full[s]);
          tma_load_2d(sa + TILE_BYTES, &tmB, kx, tj * BN, &full[s]);
          ++issued;
        }
        if (ld_shared_volatile(&s_fail)) break;
      }
    }
  } else if (warp == 1) {
    // MMA issuer: every chunk of `cstages` stages goes to an accumulator of its
    // own (two, alternating), so the epilogue adds the chunks in registers with
    // FP32 rounding (a long K summed inside one accumulator loses accuracy) and,
    // for FP8, applies each chunk's own tile scales
    if (lane == 0) {
      const uint32_t idesc = idesc_f16(BM, BN, ab_fmt);
      const int nch = nk / cstages;
      long long g = 0, ci = 0;
      bool ok = true;
      for (int b = blockIdx.x; b < ntiles && ok; b += gridDim.x) {
        for (int c = 0; c < nch && ok; ++c, ++ci) {
          const int a = (int)(ci & 1);
          if (ci >= 2 && !mbar_wait(&acc_empty[a], (uint32_t)((ci / 2) - 1) & 1, wait_ns)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t dacc = tmem + (uint32_t)(a * BN);
          for (int kb = 0; kb < cstages; ++kb, ++g) {
            const int s = (int)(g % PSTAGES);
            if (!mbar_wait(&full[s], (uint32_t)(g / PSTAGES) & 1, wait_ns)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t sa = smem_u32(smem + s * STAGE_BYTES);
            const uint32_t sb = sa + TILE_BYTES;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {  // 4 x 32 bytes of K per stage
              if (KIND == 0)
                tc_mma_f16(dacc, sdesc_sw128(sa + kk * 32), sdesc_sw128(sb + kk * 32), idesc,
                           (kb > 0 || kk > 0) ? 1u : 0u);
              else
                tc_mma_f8(dacc, sdesc_sw128(sa + kk * 32), sdesc_sw128(sb + kk * 32), idesc,
                          (kb > 0 || kk > 0) ? 1u : 0u);
            }
            tc_commit(&empty[s]);
          }
          // on failure the flag goes first, so that the epilogue, released by the
          // arrival below, leaves C alone
          if (!ok) atomicExch(&s_fail, 1);
          tc_commit(&acc_full[a]);
        }
      }
      if (!ok) atomicExch(&s_fail, 1);
    }
  } else {
    // epilogue warps 2..9
    const int q = warp & 3;                    // TMEM lane group of this warp
    const int ch = ((warp - 2) / 4) * (BN / 2);  // its half of the columns
    const int e = (warp - 2) * 32 + lane;      // 0..255: prefetch duty
    // L2 prefetch of the C tile (ti, tj): column e % 128, two 32-row lines
    auto prefetch_c = [&](int b) {
      if (b >= ntiles) return;
      int pi, pj;
      trap_index(b, TJ, pi, pj);
      const int c = pj * BN + (e % BN);
      if (c >= ncols) return;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = pi * BM + ((e / BN) * 2 + h) * 32;
        if (r < m) asm volatile("prefetch.global.L2 [%0];" ::"l"(C + (size_t)c * ldc + r));
      }
    };
    prefetch_c(blockIdx.x);
    // the chunks of a tile add up in registers (this warp's 32 rows x 64
    // columns), then one read-modify-write of C per tile
    const int nch = nk / cstages;
    long long ci = 0;
    bool ok = true;
    for (int b = blockIdx.x; b < ntiles && ok; b += gridDim.x) {
      int ti, tj;
      trap_index(b, TJ, ti, tj);
      prefetch_c(b + gridDim.x);
      float acc[2][32];
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[h][j] = 0.0f;
      for (int c = 0; c < nch; ++c, ++ci) {
        const int a = (int)(ci & 1);
        ok = mbar_wait(&acc_full[a], (uint32_t)(ci / 2) & 1, wait_ns);
        tc_fence_after();
        if (!ok || ld_shared_volatile(&s_fail)) {
          ok = false;
          break;
        }
        float scale = 1.0f;
        if (KIND == 1) {
          const signed char* ek = exps + (size_t)c * lde;
          scale = exp2f(-(float)((int)ek[ti] + (int)ek[tj]));
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          uint32_t v[32];
          tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(a * BN + ch + 32 * h), v);
          tmem_ld_wait();
#pragma unroll
          for (int j = 0; j < 32; ++j) acc[h][j] = fmaf(scale, __uint_as_float(v[j]), acc[h][j]);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[a]);
      }
      if (!ok) {
        atomicExch(&s_fail, 1);
        break;
      }
      const int r = ti * BM + q * 32 + lane;
      const bool diag = (ti == tj);
      if (r < m) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int cb = tj * BN + ch + 32 * h;
          float* cp = C + (size_t)cb * ldc + r;
          // columns j < jn of this chunk are in range (and on or below the diagonal)
          const int jn = min(32, min(ncols - cb, diag ? r - cb + 1 : 32));
          // all 32 loads first (independent, coalesced across the warp), then the stores
          float old[32];
#pragma unroll
          for (int j = 0; j < 32; ++j) old[j] = j < jn ? cp[j * ldc] : 0.0f;
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (j < jn) cp[j * ldc] = old[j] - acc[h][j];
        }
      }
    }
  }
  __syncwarp();

  // ---- teardown
  __syncthreads();
  if (ld_shared_volatile(&s_fail)) {
    if (warp == 0 && lane == 0) {
      // let every copy this CTA issued land before the CTA exits
      for (long long g = (issued > PSTAGES ? issued - PSTAGES : 0); g < issued; ++g)
        (void)mbar_wait(&full[g % PSTAGES], (uint32_t)(g / PSTAGES) & 1, wait_ns);
      atomicExch(err, 1);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, PTMEM_COLS);
}

}  // namespace tc

// ---------------------------------------------------------------- host side

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

int make_tmap_2d(CUtensorMap* map, const void* base, unsigned long long inner,
                 unsigned long long outer, unsigned long long ld_bytes, unsigned box_inner,
                 unsigned box_outer, CUtensorMapDataType dt, CUtensorMapSwizzle sw) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return JMG_ERR_CUDA;
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  cuuint64_t strides[1] = {(cuuint64_t)ld_bytes};
  cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_outer};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? JMG_OK : JMG_ERR_CUDA;
}

// 2D map over a row-major rows x cols matrix (element size esize bytes), box
// of 128 bytes x 128 rows, 128-byte swizzle.
static int make_map(CUtensorMap* map, const void* base, int rows, int cols, int ld, int esize,
                    CUtensorMapDataType dt) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return JMG_ERR_CUDA;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * esize};
  cuuint32_t box[2] = {(cuuint32_t)(128 / esize), (cuuint32_t)tc::BM};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? JMG_OK : JMG_ERR_CUDA;
}

template <int KIND>
static int syrk_persistent(int m, int ncols, int kext, int kchunk, const CUtensorMap& ma,
                           const CUtensorMap& mb, int ab_fmt, const signed char* exps, int lde,
                           float* C, int ldc, int* err, cudaStream_t s, int max_ctas,
                           int hold = 0) {
  const int stage_k = KIND == 0 ? tc::BK : 2 * tc::BK;  // K elements per stage
  if (kchunk <= 0 || kchunk > kext) kchunk = kext;
  if (kchunk % stage_k || kext % kchunk) return JMG_ERR_ALIGN;
  const int cstages = kchunk / stage_k;
  int dev = 0, nsm = 0;
  JMG_CUDA(cudaGetDevice(&dev));
  JMG_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  JMG_TRY(ensure_smem(tc::k_syrk_tc<KIND>, tc::PSMEM_BYTES));
  const int TI = cdiv(m, tc::BM), TJ = cdiv(ncols, tc::BN);
  const long long ntiles = (long long)TJ * (TJ + 1) / 2 + (long long)(TI - TJ) * TJ;
  const int grid = (int)std::min<long long>(ntiles, max_ctas > 0 ? std::min(max_ctas, nsm) : nsm);
  tc::k_syrk_tc<KIND><<<grid, tc::PTHREADS, tc::PSMEM_BYTES, s>>>(
      ma, mb, C, ldc, m, ncols, kext, ab_fmt, (int)ntiles, TJ, exps, lde, cstages, err, g_wait_ns,
      hold);
  return launched();
}

int launch_syrk_tc(int m, int ncols, int kext, const void* PA, const void* PB, int ldp, int prec,
                   float* C, int ldc, int* err, cudaStream_t s, int max_ctas, int hold,
                   int kchunk) {
  if (m <= 0 || ncols <= 0 || kext <= 0) return JMG_OK;
  if (ncols > m) return JMG_ERR_UNSUPPORTED;
  if (kext % tc::BK || ldp % 64 || ldp < kext) return JMG_ERR_ALIGN;
  if ((reinterpret_cast<uintptr_t>(PA) | reinterpret_cast<uintptr_t>(PB)) & 15) return JMG_ERR_ALIGN;
  if (prec != JMG_PREC_BF16 && prec != JMG_PREC_FP16) return JMG_ERR_UNSUPPORTED;
  CUtensorMapDataType dt =
      prec == JMG_PREC_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  CUtensorMap ma, mb;
  JMG_TRY(make_map(&ma, PA, m, kext, ldp, 2, dt));
  JMG_TRY(make_map(&mb, PB, m, kext, ldp, 2, dt));
  return syrk_persistent<0>(m, ncols, kext, kchunk, ma, mb, prec == JMG_PREC_BF16 ? 1 : 0, nullptr,
                            0, C, ldc, err, s, max_ctas, hold);
}

int launch_syrk_fp8(int m, int ncols, int kext, const void* Q, int ldq, const signed char* e,
                    int lde, float* C, int ldc, int* err, cudaStream_t s, int max_ctas) {
  if (m <= 0 || ncols <= 0 || kext <= 0) return JMG_OK;
  if (ncols > m) return JMG_ERR_UNSUPPORTED;
  if (kext % 128 || ldq % 128 || ldq < kext) return JMG_ERR_ALIGN;
  if (reinterpret_cast<uintptr_t>(Q) & 15) return JMG_ERR_ALIGN;
  if (!e) return JMG_ERR_UNSUPPORTED;
  CUtensorMap mq;
  JMG_TRY(make_map(&mq, Q, m, kext, ldq, 1, CU_TENSOR_MAP_DATA_TYPE_UINT8));
  return syrk_persistent<1>(m, ncols, kext, 128, mq, mq, 0, e, lde, C, ldc, err, s, max_ctas);
}

}  // namespace jmg
