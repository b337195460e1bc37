// k_ozaki.cu -- FP64-accurate product A X (and residual R = B - A X) on the
// BF16 tensor cores by error-free splitting (Ozaki, Ogita, Oishi and Rump
// 2012, "Error-free transformations of matrix multiplication by using fast
// routines of matrix multiplication and its applications").
//
// Every row i of the symmetric A (both triangles materialised from lower(A))
// is scaled by 2^-eA[i] so that |a_ij| 2^-eA[i] < 1, and every column c of X
// by 2^-eX[c]; each scaled value v is then cut into S = 8 slices of 7 bits,
//     v = sum_s k_s 2^-7(s+1) + r,   k_s integer, |k_0| <= 128, |k_s| <= 64,
// |r| <= 2^-57, as the balanced base-128 digits of the integer rint(v 2^56).
// The integers are exact in BF16, a product of two slices is an
// integer of at most 2^14, and
//     (A X)_ic = 2^(eA[i] + eX[c] - 14) sum_d 2^-7d  sum_{a+b=d} sum_k A_a[i,k] X_b[k,c].
// Pairs with a + b <= 7 are kept (the rest lie below 2^-56 of the row scale).
// For each d the inner sums are accumulated on the tensor cores in FP32 in a
// TMEM accumulator of its own; over a window of 256 values of k every partial
// sum is an integer below 2^24 (at most 2.5 * 2^14 * 256), so it is exact.
// After each window the epilogue converts the 8 accumulators to integers and
// adds them, exactly, into two 64-bit sums per output (d = 0..3 and d = 4..7,
// each weighted by its power of 2^7); at the end the two sums become one FP64
// value (one rounding), scaled by the powers of two, and one FP64 partial sum
// per K split is stored.  R = B - sum of partials is formed by the same
// reduction kernel as the CUDA-core residual.
//
// tcgen05 kernel, 576 threads: warp 0 issues TMA loads (8 X-slice tiles per
// 64-wide K block, then 8 A-slice tiles through a 6-stage ring), warp 1 issues
// the MMAs (M = 128, K = 16, N = up to 256: consecutive X slices of one A
// slice in one instruction), warps 2-17 drain
// TMEM (up to four per TMEM lane quarter, 16 columns each).  With 32 or fewer
// right-hand sides per tile the eight accumulators fit twice in TMEM and
// alternate by window, so the MMAs of a window overlap the drain of the last
// one.  All waits are bounded.
#include <algorithm>

#include "kernels.h"
#include "tc_ptx.cuh"

namespace jmg {
namespace oz {
constexpr int S = 8;        // slices per operand
constexpr int BM = 128;     // rows per tile
constexpr int BK = 64;      // K per block: 64 BF16 = one 128-byte swizzle row
constexpr int WIN = 4;      // K blocks per exact accumulation window (256 values)
constexpr int ASTAGES = 6;  // ring of A-slice tiles
constexpr int THREADS = 576;  // warps 0-1 producer / MMA, 2-17 epilogue (16 columns each)
constexpr int A_TILE = BM * BK * 2;  // 16 KiB

// rint(x 2^(56-e)) for |x| < 2^e, formed from the bits of x with integer
// operations only (FP64 runs at 1/64 of the FP32 rate on this GPU): x is
// M 2^(ex-1075) with the 53-bit significand M, so the value is M 2^sh with
// sh = ex - 1019 - e <= 3, a left shift, or a right shift rounded to nearest
// with ties to even.  Non-finite x gives 0 (those rows carry no valid slices).
JMG_DEV long long scaled_int(double x, int e) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  if (ex == 0x7FF) return 0;
  unsigned long long M = b & ((1ull << 52) - 1);
  int ee = ex;
  if (ex)
    M |= 1ull << 52;
  else
    ee = 1;  // subnormal
  const int sh = ee - 1019 - e;
  unsigned long long V;
  if (sh >= 0) {
    V = (sh > 62 || (M >> (62 - sh)) != 0) ? 0ull : M << sh;  // (no overflow when |x| < 2^e)
  } else {
    const int k = -sh;
    if (k >= 64) {
      V = 0;
    } else {
      V = M >> k;
      const unsigned long long rem = M & ((1ull << k) - 1), half = 1ull << (k - 1);
      if (rem > half || (rem == half && (V & 1))) ++V;
    }
  }
  return (b >> 63) ? -(long long)V : (long long)V;
}

// Slices of x 2^-e (|x 2^-e| < 1): V = rint(x 2^(56-e)) is an integer with
// |V| < 2^56, cut into balanced base-128 digits from the bottom, k_s in
// [-64, 63] for s = 7..1, and the top digit k_0 = the rest, |k_0| <= 128; then
// x 2^-e = sum_s k_s 2^-7(s+1) + r with |r| <= 2^-57.  Integer arithmetic only.
JMG_DEV void slice8(double x, int e, __nv_bfloat16 (&out)[S]) {
  long long V = scaled_int(x, e);
#pragma unroll
  for (int s = S - 1; s >= 1; --s) {
    const long long k = ((V + 64) & 127) - 64;
    out[s] = __int2bfloat16_rn((int)k);  // |k| <= 64: exact
    V = (V - k) >> 7;                    // exact
  }
  out[0] = __int2bfloat16_rn((int)V);    // |V| <= 128: exact
}

// exponent e with |x| 2^-e < 1 for every |x| <= m (0 for m == 0)
JMG_DEV int scale_exp(double m) {
  if (!(m > 0.0) || !isfinite(m)) return 0;
  int e;
  (void)frexp(m, &e);  // m = f 2^e, f in [0.5, 1)
  return e;
}
}  // namespace oz

// A slices: SA[s * sstride + i * lds + k] for every (i, k) of the symmetric
// matrix.  One CTA per lower 64 x 64 tile writes the tile and its mirror; each
// thread cuts 4 consecutive values of a row and stores 8 bytes per slice.
__global__ void __launch_bounds__(256) k_oz_slice_a(int n, const double* __restrict__ A, int lda,
                                                    const double* __restrict__ rowmax,
                                                    __nv_bfloat16* __restrict__ SA, int lds,
                                                    size_t sstride) {
  int ti, tj;
  tri_index(blockIdx.x, ti, tj);
  const int i0 = ti * 64, j0 = tj * 64;
  __shared__ double T[64][65];  // T[c][r] = a(i0 + r, j0 + c)
  __shared__ int er[64], ec[64];
  const int t = threadIdx.x;
  {
    double v[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {  // all loads first
      const int idx = t + 256 * q;
      const int r = idx % 64, c = idx / 64;
      const int i = i0 + r, j = j0 + c;
      v[q] = (i < n && j < n && i >= j) ? A[(size_t)j * lda + i] : 0.0;
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int idx = t + 256 * q;
      T[idx / 64][idx % 64] = v[q];
    }
  }
  if (t < 64) er[t] = (i0 + t < n) ? oz::scale_exp(rowmax[i0 + t]) : 0;
  else if (t < 128) ec[t - 64] = (j0 + t - 64 < n) ? oz::scale_exp(rowmax[j0 + t - 64]) : 0;
  __syncthreads();
  const bool diag = ti == tj;
  // the row of the padded slice ends at lds (a multiple of 64): 4-wide groups
  // never straddle it; values past n or above the diagonal are zero
  auto put4 = [&](int row, int k, const double (&x)[4], int e) {
    __nv_bfloat16 w[4][oz::S];
#pragma unroll
    for (int u = 0; u < 4; ++u) oz::slice8(x[u], e, w[u]);
#pragma unroll
    for (int s = 0; s < oz::S; ++s) {
      __nv_bfloat162 lo, hi;
      lo.x = w[0][s], lo.y = w[1][s], hi.x = w[2][s], hi.y = w[3][s];
      uint2 pk;
      pk.x = *reinterpret_cast<uint32_t*>(&lo);
      pk.y = *reinterpret_cast<uint32_t*>(&hi);
      *reinterpret_cast<uint2*>(&SA[s * sstride + (size_t)row * lds + k]) = pk;
    }
  };
  // direct: row i = i0 + r, columns k = j0 + c .. c+3 (threads run along k).
  // On a diagonal tile the whole row segment is written here, the entries
  // above the diagonal from their mirrors (a_rk = a_kr).
#pragma unroll 1
  for (int q = 0; q < 4; ++q) {
    const int idx = t + 256 * q;
    const int c = 4 * (idx % 16), r = idx / 16;
    const int i = i0 + r, k = j0 + c;
    if (i >= n || k >= n) continue;
    double x[4];  // (zero past n)
#pragma unroll
    for (int u = 0; u < 4; ++u) x[u] = (!diag || c + u <= r) ? T[c + u][r] : T[r][c + u];
    put4(i, k, x, er[r]);
  }
  if (diag) return;
  // mirror: row j0 + c, columns k = i0 + r .. r+3 (the tile is strictly below
  // the diagonal, so its transpose is strictly above it)
#pragma unroll 1
  for (int q = 0; q < 4; ++q) {
    const int idx = t + 256 * q;
    const int r = 4 * (idx % 16), c = idx / 16;
    const int row = j0 + c, k = i0 + r;
    if (row >= n || k >= n) continue;
    double x[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) x[u] = T[c][r + u];
    put4(row, k, x, ec[c]);
  }
}

// X slices: SX[s * sstride + c * ldsx + k]; one CTA per (padded) column.
// Padded columns c >= nrhs are zero.
__global__ void __launch_bounds__(256) k_oz_slice_x(int n, int nrhs, const double* __restrict__ X,
                                                    int ldx, int* __restrict__ ex,
                                                    __nv_bfloat16* __restrict__ SX, int ldsx,
                                                    size_t sstride) {
  __shared__ double red[8];
  const int c = blockIdx.x, t = threadIdx.x;
  const bool live = c < nrhs;
  double m = 0.0;
  if (live)
    for (int k = t; k < n; k += 256) m = fmax(m, fabs(X[(size_t)c * ldx + k]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((t & 31) == 0) red[t / 32] = m;
  __syncthreads();
  if (t == 0) {
    double mm = red[0];
    for (int w = 1; w < 8; ++w) mm = fmax(mm, red[w]);
    red[0] = mm;
  }
  __syncthreads();
  const int e = live ? oz::scale_exp(red[0]) : 0;
  if (t == 0) ex[c] = e;
  for (int k = t; k < n; k += 256) {
    __nv_bfloat16 w[oz::S];
    oz::slice8(live ? X[(size_t)c * ldx + k] : 0.0, e, w);
#pragma unroll
    for (int s = 0; s < oz::S; ++s) SX[s * sstride + (size_t)c * ldsx + k] = w[s];
  }
}

// ---------------------------------------------------------------------------
// The split product.  grid = (row tiles, column tiles, K splits).
template <int N>
__global__ void __launch_bounds__(oz::THREADS, 1)
    k_oz_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmX,
              int n, int nrhs, int nrhs_pad, const double* __restrict__ rowmax,
              const int* __restrict__ ex, double* __restrict__ part, int win_per_split,
              int* __restrict__ err, unsigned long long wait_ns) {
  using namespace oz;
  using namespace tc;
  constexpr int X_TILE = N * BK * 2;  // one slice: N rows x 128 bytes
  constexpr int X_BUF = S * X_TILE;
  // two accumulator sets where TMEM holds them (N <= 32): the MMAs of window
  // w+1 run while the epilogue drains window w
  constexpr int NBUF = (16 * N <= 512) ? 2 : 1;
  constexpr uint32_t TCOLS = (NBUF * 8 * N < 32) ? 32 : NBUF * 8 * N;
  extern __shared__ __align__(1024) unsigned char sm_raw_oz[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(sm_raw_oz) + 1023) & ~uintptr_t(1023));
  unsigned char* xbuf = smem;                  // [2][S][X_TILE]
  unsigned char* abuf = smem + 2 * X_BUF;      // [ASTAGES][A_TILE]
  uint64_t* bars = reinterpret_cast<uint64_t*>(abuf + ASTAGES * A_TILE);
  uint64_t* xfull = bars;           // 2
  uint64_t* xempty = bars + 2;      // 2
  uint64_t* afull = bars + 4;       // ASTAGES
  uint64_t* aempty = afull + ASTAGES;
  uint64_t* accf = aempty + ASTAGES;  // NBUF
  uint64_t* acce = accf + NBUF;       // NBUF
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acce + NBUF);
  __shared__ int s_fail;

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int rt = blockIdx.x, ct = blockIdx.y, z = blockIdx.z;
  const int nkb = (n + BK - 1) / BK;
  const int nwin_total = (nkb + WIN - 1) / WIN;
  const int w0 = z * win_per_split;
  const int w1 = min(nwin_total, w0 + win_per_split);
  const int kb0 = w0 * WIN, kb1 = min(nkb, w1 * WIN);

  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int i = 0; i < 2; ++i) {
      mbar_init(&xfull[i], 1);
      mbar_init(&xempty[i], 1);
    }
    for (int i = 0; i < ASTAGES; ++i) {
      mbar_init(&afull[i], 1);
      mbar_init(&aempty[i], 1);
    }
    for (int i = 0; i < NBUF; ++i) {
      mbar_init(&accf[i], 1);
      mbar_init(&acce[i], N * 4 / 16);
    }
    fence_mbar_init();
    prefetch_tmap(&tmA);
    prefetch_tmap(&tmX);
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, TCOLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  long long x_issued = 0, a_issued = 0;
  if (warp == 0) {
    if (lane == 0) {
      long long g = 0;
      for (int kb = kb0; kb < kb1; ++kb) {
        const int u = kb - kb0, xs = u & 1;
        if (u >= 2 && !mbar_wait(&xempty[xs], (uint32_t)((u >> 1) - 1) & 1, wait_ns)) {
          atomicExch(&s_fail, 1);
          break;
        }
        if (ld_shared_volatile(&s_fail)) break;
        mbar_expect_tx(&xfull[xs], S * X_TILE);
        for (int b = 0; b < S; ++b)
          tma_load_2d(xbuf + xs * X_BUF + b * X_TILE, &tmX, kb * BK, b * nrhs_pad + ct * N,
                      &xfull[xs]);
        ++x_issued;
        bool ok = true;
        for (int a = 0; a < S; ++a, ++g) {
          const int st = (int)(g % ASTAGES);
          if (g >= ASTAGES && !mbar_wait(&aempty[st], (uint32_t)((g / ASTAGES) - 1) & 1, wait_ns)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&afull[st], A_TILE);
          tma_load_2d(abuf + st * A_TILE, &tmA, kb * BK, a * n + rt * BM, &afull[st]);
          ++a_issued;
        }
        if (!ok) {
          atomicExch(&s_fail, 1);
          break;
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr int GMAX = (256 / N) < S ? (256 / N) : S;  // X slices per MMA
      long long g = 0;
      bool ok = true;
      for (int w = w0; w < w1 && ok; ++w) {
        const int use = w - w0, bw = use % NBUF;  // accumulator set of this window
        if (use >= NBUF &&
            !mbar_wait(&acce[bw], (uint32_t)((use / NBUF - 1) & 1), wait_ns)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t tacc = tmem + (uint32_t)(bw * 8 * N);
        const int kbw0 = max(kb0, w * WIN), kbw1 = min(kb1, (w + 1) * WIN);
        for (int kb = kbw0; kb < kbw1 && ok; ++kb) {
          const int u = kb - kb0, xs = u & 1;
          if (!mbar_wait(&xfull[xs], (uint32_t)(u >> 1) & 1, wait_ns)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t xb = smem_u32(xbuf + xs * X_BUF);
          for (int a = 0; a < S; ++a, ++g) {
            const int st = (int)(g % ASTAGES);
            if (!mbar_wait(&afull[st], (uint32_t)(g / ASTAGES) & 1, wait_ns)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t ab = smem_u32(abuf + st * A_TILE);
            // X slices b = 0 .. S-1-a feed levels d = a .. S-1.  The slices sit
            // one after another in shared memory and the levels' accumulators
            // one after another in TMEM, so GMAX consecutive slices make one
            // MMA of N * GMAX columns (<= 256) that reads the A tile once.
            for (int b0 = 0; b0 < S - a; b0 += GMAX) {
              const int cnt = min(GMAX, S - a - b0);
              const uint32_t idesc_g = idesc_f16(BM, N * cnt, 1);
              const uint32_t dacc = tacc + (uint32_t)((a + b0) * N);
#pragma unroll
              for (int kk = 0; kk < 4; ++kk) {
                const bool first = (kb == kbw0) && (a == 0) && (kk == 0);
                tc_mma_f16(dacc, sdesc_sw128(ab + kk * 32),
                           sdesc_sw128(xb + b0 * X_TILE + kk * 32), idesc_g, first ? 0u : 1u);
              }
            }
            tc_commit(&aempty[st]);
          }
          tc_commit(&xempty[xs]);
        }
        tc_commit(&accf[bw]);
      }
      if (!ok) atomicExch(&s_fail, 1);
    }
  } else {
    // epilogue: warp w reads TMEM lane group q = w % 4 (rows rt*128 + 32q + lane)
    // and CW columns of the accumulators.  Every window's accumulators are exact
    // integers (below 2^24); they are converted to integers and summed exactly
    // in 64 bits, d = 0..3 as hs = sum acc_d 2^(21-7d) and d = 4..7 as
    // ls = sum acc_d 2^(49-7d) (each window adds less than 2^45 to either, and
    // a CTA takes at most 256 windows, so both stay below 2^53).  Only the end
    // converts to FP64: sum_d acc_d 2^-7d = 2^-21 (hs + ls 2^-28), one rounding.
    constexpr int CW = 16;         // columns per epilogue warp
    constexpr int EW = N * 4 / CW;  // epilogue warps with columns (4 per 64 columns)
    const int ew = warp - 2;
    const int q = warp & 3;
    const int ch = (ew >> 2) * CW;
    if (ew < EW) {
      unsigned long long hs[CW], ls[CW];  // (unsigned: garbage rows past n wrap, never trap)
#pragma unroll
      for (int c = 0; c < CW; ++c) hs[c] = ls[c] = 0ull;
      bool ok = true;
      for (int w = w0; w < w1; ++w) {
        const int use = w - w0, bw = use % NBUF;
        if (!mbar_wait(&accf[bw], (uint32_t)((use / NBUF) & 1), wait_ns) ||
            ld_shared_volatile(&s_fail)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t tacc = tmem + (uint32_t)(bw * 8 * N);
#pragma unroll
        for (int d = 0; d < S; ++d) {
          const long long sc = 1ll << (d <= 3 ? 21 - 7 * d : 49 - 7 * d);
#pragma unroll
          for (int c0 = 0; c0 < CW; c0 += 16) {
            uint32_t v[16];
            tmem_ld16(tacc + ((uint32_t)(q * 32) << 16) + (uint32_t)(d * N + ch + c0), v);
            tmem_ld_wait();
#pragma unroll
            for (int c = 0; c < 16; ++c) {
              const long long t = (long long)__float2int_rn(__uint_as_float(v[c])) * sc;
              if (d <= 3)
                hs[c0 + c] += (unsigned long long)t;
              else
                ls[c0 + c] += (unsigned long long)t;
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acce[bw]);
      }
      if (ok) {
        const int row = rt * BM + q * 32 + lane;
        if (row < n) {
          const int er = oz::scale_exp(rowmax[row]);
#pragma unroll
          for (int c = 0; c < CW; ++c) {
            const int col = ct * N + ch + c;
            if (col < nrhs) {
              const double tot = fma((double)(long long)ls[c], 0x1p-28, (double)(long long)hs[c]);
              part[(size_t)z * n * nrhs + (size_t)col * n + row] =
                  ldexp(tot, er + ex[col] - 14 - 21);
            }
          }
        }
      } else {
        atomicExch(&s_fail, 1);
      }
    }
  }
  __syncwarp();
  __syncthreads();
  if (ld_shared_volatile(&s_fail)) {
    if (warp == 0 && lane == 0) {
      for (long long u = (x_issued > 2 ? x_issued - 2 : 0); u < x_issued; ++u)
        (void)mbar_wait(&xfull[u & 1], (uint32_t)(u >> 1) & 1, wait_ns);
      for (long long g = (a_issued > ASTAGES ? a_issued - ASTAGES : 0); g < a_issued; ++g)
        (void)mbar_wait(&afull[g % ASTAGES], (uint32_t)(g / ASTAGES) & 1, wait_ns);
      atomicExch(err, 1);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, TCOLS);
}

// ---------------------------------------------------------------------------
// host side

size_t oz_a_bytes(int n) {
  const size_t lds = round_up((size_t)std::max(n, 1), 64);
  return sizeof(__nv_bfloat16) * oz::S * lds * (size_t)std::max(n, 1);
}
static int oz_n_tile(int nrhs) { return nrhs > 32 ? 64 : (nrhs > 16 ? 32 : 16); }
size_t oz_x_bytes(int n, int nrhs) {
  const int N = oz_n_tile(nrhs);
  const size_t pad = round_up((size_t)std::max(nrhs, 1), (size_t)N);
  const size_t ldsx = round_up((size_t)std::max(n, 1), 64);
  return sizeof(__nv_bfloat16) * oz::S * pad * ldsx + sizeof(int) * round_up(pad, 64);
}
int oz_splits(int n, int nrhs) {
  // K splits: minimise (waves of CTAs over the SMs) x (windows per CTA), one
  // CTA per SM (the kernel takes ~195 KB of shared memory)
  const int N = oz_n_tile(nrhs);
  const int ctas = cdiv(n, oz::BM) * cdiv(nrhs, N);
  const int nwin = cdiv(cdiv(n, oz::BK), oz::WIN);
  int best = cdiv(nwin, 256);
  long long best_cost = -1;
  for (int ks = cdiv(nwin, 256); ks <= nwin; ++ks) {  // at most 256 windows per CTA
    const int wps = cdiv(nwin, ks);
    const int used = cdiv(nwin, wps);
    const long long cost = (long long)cdiv(ctas * used, 152) * (wps + 1);  // +1: fixed per-CTA cost
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = ks;
    }
  }
  return best;
}

int oz_prepare_a(int n, const double* A, int lda, double* rowmax, void* SA, cudaStream_t s) {
  JMG_TRY(launch_row_stats(n, A, lda, nullptr, rowmax, s));
  return oz_slice_a(n, A, lda, rowmax, SA, s);
}

int oz_slice_a(int n, const double* A, int lda, const double* rowmax, void* SA, cudaStream_t s) {
  if (n <= 0) return JMG_OK;
  const unsigned tiles = (unsigned)tri_tiles(cdiv(n, 64));
  const int lds = (int)round_up((size_t)n, 64);
  k_oz_slice_a<<<tiles, 256, 0, s>>>(n, A, lda, rowmax, (__nv_bfloat16*)SA, lds,
                                     (size_t)lds * n);
  return launched();
}

typedef CUresult (*EncodeTiledFnOz)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                    const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                    const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                    CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static int map_bf16(CUtensorMap* map, const void* base, int rows, int cols, int ld, int box_rows) {
  static EncodeTiledFnOz enc = nullptr;
  if (!enc) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult qr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &qr) != cudaSuccess ||
        qr != cudaDriverEntryPointSuccess)
      return JMG_ERR_CUDA;
    enc = reinterpret_cast<EncodeTiledFnOz>(p);
  }
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)oz::BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims,
                   strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? JMG_OK : JMG_ERR_CUDA;
}

template <int N>
static int oz_gemm_launch(int n, int nrhs, const void* SA, const void* SX, int nrhs_pad,
                          const double* rowmax, const int* ex, double* part, int ks, int* err,
                          cudaStream_t s) {
  const int lds = (int)round_up((size_t)n, 64);
  CUtensorMap ma, mx;
  JMG_TRY(map_bf16(&ma, SA, oz::S * n, n, lds, oz::BM));
  JMG_TRY(map_bf16(&mx, SX, oz::S * nrhs_pad, n, lds, N));
  constexpr int SMEM = 2 * oz::S * N * oz::BK * 2 + oz::ASTAGES * oz::A_TILE + 1024 + 256;
  JMG_TRY(ensure_smem(k_oz_gemm<N>, SMEM));
  const int nwin = cdiv(cdiv(n, oz::BK), oz::WIN);
  const int wps = cdiv(nwin, ks);
  dim3 grid(cdiv(n, oz::BM), nrhs_pad / N, cdiv(nwin, wps));
  k_oz_gemm<N><<<grid, oz::THREADS, SMEM, s>>>(ma, mx, n, nrhs, nrhs_pad, rowmax, ex, part, wps,
                                               err, g_wait_ns);
  return launched();
}

int oz_splits_used(int n, int nrhs) {
  const int ks = oz_splits(n, nrhs);
  const int nwin = cdiv(cdiv(n, oz::BK), oz::WIN);
  return cdiv(nwin, cdiv(nwin, ks));
}

// part = A X (split K) for the prepared A slices; X slices built here.
int oz_product(int n, int nrhs, const void* SA, const double* rowmax, const double* X, int ldx,
               void* xwork, double* part, int* err, cudaStream_t s) {
  if (n <= 0 || nrhs <= 0) return JMG_OK;
  const int N = oz_n_tile(nrhs);
  const int pad = (int)round_up((size_t)nrhs, (size_t)N);
  const int lds = (int)round_up((size_t)n, 64);
  __nv_bfloat16* SX = static_cast<__nv_bfloat16*>(xwork);
  int* ex = reinterpret_cast<int*>(SX + (size_t)oz::S * pad * lds);
  k_oz_slice_x<<<pad, 256, 0, s>>>(n, nrhs, X, ldx, ex, SX, lds, (size_t)pad * lds);
  JMG_TRY(launched());
  const int ks = oz_splits(n, nrhs);
  if (N == 64) return oz_gemm_launch<64>(n, nrhs, SA, SX, pad, rowmax, ex, part, ks, err, s);
  if (N == 32) return oz_gemm_launch<32>(n, nrhs, SA, SX, pad, rowmax, ex, part, ks, err, s);
  return oz_gemm_launch<16>(n, nrhs, SA, SX, pad, rowmax, ex, part, ks, err, s);
}

}  // namespace jmg
