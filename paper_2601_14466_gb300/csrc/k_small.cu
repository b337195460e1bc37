// k_small.cu -- the whole mixed-precision posv for small systems (n <= 2048)
// in ONE persistent cooperative kernel (paper: "Software design", potrs as one
// call on the framework's stream, and the refinement of Section 3 with its
// stopping rule).  For small n the tensor-core path is bound by launches and by
// the host reading the backward error after every residual; here every step,
// including the decision to stop, runs on the device:
//
//   1. Cholesky of fp32(A) (+ a diagonal shift after a breakdown) over 64 x 64
//      tiles of the lower triangle, as a dataflow over per-tile ready flags
//      instead of grid barriers: the owner of tile (i, j) starts from A_ij,
//      subtracts L_ik L_jk^T for k = 0, 1, ... as soon as both tiles are
//      published, then factors (i == j) or solves against L_jj (i > j) and
//      publishes its tile;
//   2. the inverse of L in the same dataflow: the owner of a diagonal tile
//      inverts L_jj right after publishing it, and the owner of the inverse
//      tile (i, j), i > j, forms  Linv_ij = -Linv_ii sum_{k=j..i-1} L_ik Linv_kj.
//      Factor tiles are numbered column by column, the inverse tiles after
//      them in the same order, and every CTA takes its tiles in increasing
//      number; a tile depends only on tiles with smaller numbers, so the
//      smallest unfinished tile can always proceed;
//   3. every solve M^{-1} d with M = L L^T is then two block products spread
//      over the CTAs, y = Linv d (row blocks) and x = Linv^T y (column blocks),
//      in FP32 on the right-hand side scaled column by column into range;
//   4. refinement: R = B - A X in FP64 over the tiles of lower(A) (tile (I, J)
//      adds A_IJ X_J to rows I and A_IJ^T X_I to rows J; the partial sums are
//      added in a fixed order, so the result does not depend on scheduling),
//      eta_j = ||r_j||_inf / (||A||_inf ||x_j||_inf + ||b_j||_inf), and
//      X += M^{-1} R until max_j eta_j <= tol, maxit steps, a NaN, or three
//      consecutive steps that fail to halve eta (the IR rule of the host path).
//      Every CTA evaluates the rule itself on the same reduced maxima, so no
//      broadcast is needed.
//
// Grid barriers are a monotone arrival counter; every wait (barrier or tile
// flag) is bounded by the runtime limit, and on expiry the kernel records
// JMG_ERR_TIMEOUT and every CTA leaves.  Launched cooperatively, so all CTAs are
// co-resident (which the flag waits rely on).
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "kernels.h"

namespace jmg {
namespace sm {
constexpr int NB = 64;      // tile size
constexpr int TH = 256;     // threads per CTA
constexpr int NMAX = 2048;  // largest order of the small path
constexpr int RMAX = 64;    // most right-hand sides of the small path
constexpr int CR = 8;       // right-hand sides per pass of the residual
constexpr int SCR = 4;      // right-hand sides per pass of the solve
constexpr int NTMAX = NMAX / NB;
constexpr int TILES_MAX = NTMAX * (NTMAX + 1) / 2;
constexpr int LDS = NB + 1;  // leading dimension of a shared tile read by rows
constexpr int MAX_TRIES = 6; // factorisations (1 + shifted retries)
}  // namespace sm

// Control block at the front of the workspace (cleared by the host before the
// launch).
struct SmallCtl {
  unsigned int arrive;  // grid-barrier arrivals (monotone)
  int status;           // 0 / JMG_ERR_TIMEOUT / JMG_ERR_NOT_SPD / JMG_ERR_NOT_CONVERGED
  int info;             // potrf info of the last factorisation (0 if SPD)
  int iters;            // refinement steps
  int converged;        // max_j eta_j <= tol reached
  int tries;            // factorisations performed
  int n_hist;           // residuals evaluated
  int pad0;
  unsigned long long anorm_bits;  // ||A||_inf (bits of a non-negative double)
  unsigned long long dmax_bits;   // max_i |a_ii|
  double eta;                     // max_j eta_j of the last residual
  double shift;                   // diagonal shift of the factor
  int fail[8];                    // per factorisation: first failing pivot (1-based)
  double eta_hist[32];
  unsigned long long bmax_bits[sm::RMAX];           // ||b_q||_inf
  unsigned long long colmax_bits[2][3 * sm::RMAX];  // |r|, |x|, |b| maxima, by parity
  int ready[sm::TILES_MAX];                         // factor tiles (factorisation number)
  int inv[sm::TILES_MAX];                           // inverse tiles (factorisation number)
};

// Workspace of the small path (256-byte aligned regions).
struct SmallPlan {
  size_t ctl, W, Li, Lv, Y, X, R, part, rs, total;
  int ldw, nt, ntiles, dcols;
};

static inline size_t take_al(size_t& off, size_t bytes) {
  const size_t at = off;
  off = round_up(off + bytes, 256);
  return at;
}

SmallPlan small_plan(int n, int nrhs) {
  SmallPlan p;
  size_t off = 0;
  const size_t N = (size_t)std::max(n, 1), R = (size_t)std::max(nrhs, 1);
  p.nt = cdiv(std::max(n, 1), sm::NB);
  p.ldw = p.nt * sm::NB;
  p.ntiles = p.nt * (p.nt + 1) / 2;
  p.dcols = round_up(std::max(nrhs, 1), sm::SCR);
  p.ctl = take_al(off, sizeof(SmallCtl));
  p.W = take_al(off, sizeof(float) * (size_t)p.ldw * p.ldw);                 // L, column-major
  p.Li = take_al(off, sizeof(float) * (size_t)p.nt * sm::NB * sm::NB);       // L_jj^{-1}, col-major
  p.Lv = take_al(off, sizeof(float) * (size_t)p.ntiles * sm::NB * sm::NB);   // Linv tiles, row-major
  p.Y = take_al(off, sizeof(float) * (size_t)p.ldw * p.dcols);
  p.X = take_al(off, sizeof(double) * N * R);
  p.R = take_al(off, sizeof(double) * N * R);
  p.part = take_al(off, sizeof(double) * (size_t)p.ntiles * 2 * sm::NB * R);
  p.rs = take_al(off, sizeof(double) * (size_t)p.ntiles * 2 * sm::NB);
  p.total = off;
  return p;
}

struct SmallArgs {
  int n, nrhs, lda, ldb, ldw, nt, ntiles, maxit, shift_retry;
  double tol;
  unsigned long long wait_ns;
  const double* A;
  double* B;
  int* info;
  float* W;
  float* Li;
  float* Lv;
  float* Y;
  double* X;
  double* R;
  double* part;
  double* rs;
  SmallCtl* ctl;
};

namespace sm {

// ------------------------------------------------------------------ sync

JMG_DEV int ld_acq(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
JMG_DEV unsigned ld_acq_u(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
JMG_DEV void st_rel(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
JMG_DEV int ld_vol(const int* p) { return *(const volatile int*)p; }

JMG_DEV void amax_bits(unsigned long long* p, double v) {
  const unsigned long long b =
      isnan(v) ? 0x7FFFFFFFFFFFFFFFull : (unsigned long long)__double_as_longlong(fabs(v));
  atomicMax(p, b);
}
JMG_DEV double from_bits(const unsigned long long* p) {
  return __longlong_as_double((long long)*(const volatile unsigned long long*)p);
}

// Grid barrier number ++k (complete at k * G arrivals).  Bounded; gives up
// when another CTA has recorded a timeout.  Returns false (in every thread)
// when the kernel must leave.
JMG_DEV bool grid_sync(SmallCtl* c, unsigned G, unsigned& k, uint64_t limit, int* s_bc) {
  __syncthreads();
  ++k;
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(&c->arrive, 1u);
    const unsigned target = k * G;
    int ok = 1;
    const uint64_t t0 = globaltimer_ns();
    while (ld_acq_u(&c->arrive) < target) {
      if (ld_vol(&c->status) == JMG_ERR_TIMEOUT) {
        ok = 0;
        break;
      }
      if (globaltimer_ns() - t0 > limit) {
        atomicCAS(&c->status, 0, JMG_ERR_TIMEOUT);
        ok = 0;
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
    s_bc[0] = ok && ld_vol(&c->status) != JMG_ERR_TIMEOUT;
  }
  __syncthreads();
  const bool ok = s_bc[0] != 0;
  __syncthreads();  // s_bc is reused by the next broadcast
  return ok;
}

// Wait until the flags f0 and f1 (nullptr: none) reach `epoch` (thread 0,
// bounded), then the CTA reads the tiles behind them.  False when the
// factorisation `tr` has failed or a wait ran out.
JMG_DEV bool wait_flags(SmallCtl* c, const int* f0, const int* f1, int epoch, int tr,
                        uint64_t limit, int* s_bc) {
  if (threadIdx.x == 0) {
    int ok = 1;
    for (int q = 0; q < 2 && ok; ++q) {
      const int* f = q == 0 ? f0 : f1;
      if (!f || ld_acq(f) >= epoch) continue;
      const uint64_t t0 = globaltimer_ns();
      while (ld_acq(f) < epoch) {
        if (ld_vol(&c->fail[tr]) != 0 || ld_vol(&c->status) == JMG_ERR_TIMEOUT) {
          ok = 0;
          break;
        }
        if (globaltimer_ns() - t0 > limit) {
          atomicCAS(&c->status, 0, JMG_ERR_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    s_bc[1] = ok;
  }
  __syncthreads();
  const bool ok = s_bc[1] != 0;
  __syncthreads();  // s_bc is reused by the next broadcast
  return ok;
}

// Every thread's stores of the tile are issued; thread 0 makes them visible
// at GPU scope and raises the flag.
JMG_DEV void publish(int* flag, int epoch) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    st_rel(flag, epoch);
  }
}

// tile number, column by column over the lower triangle: (i, j), i >= j
JMG_DEV int cm(int nt, int i, int j) { return j * nt - j * (j - 1) / 2 + (i - j); }
JMG_DEV void cm_inv(int nt, int t, int& i, int& j) {
  j = 0;
  while (t >= nt - j) {
    t -= nt - j;
    ++j;
  }
  i = j + t;
}

}  // namespace sm
}  // namespace jmg


namespace jmg {
namespace sm {

// inverse tiles below the diagonal, numbered column by column: (i, j), i > j
JMG_DEV void cmo_inv(int nt, int u, int& i, int& j) {
  j = 0;
  while (u >= nt - 1 - j) {
    u -= nt - 1 - j;
    ++j;
  }
  i = j + 1 + u;
}

// ------------------------------------------------------------------ tiles
//
// Operand tiles in shared memory are 64 x 64 with leading dimension 64 and
// the contraction index outermost: T[k * 64 + x].  gemm_sub takes two of them
// and updates the register tile of a thread (rows 4tx.., columns 4ty..).

// Ts[k * 64 + r] = L(I*64 + r, K*64 + k) from W (published tiles: read through
// L2), entries past n zero
JMG_DEV void load_L(float* Ts, const float* W, int ldw, int n, int I, int K) {
#pragma unroll
  for (int p = 0; p < NB * NB / 4 / TH; ++p) {  // all loads in flight at once
    const int e = threadIdx.x + p * TH;
    const int c = e >> 4, r4 = (e & 15) * 4, gr = I * NB + r4, gc = K * NB + c;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (gc < n) {
      const float* src = W + (size_t)gc * ldw + gr;
      if (gr + 3 < n) {
        v = __ldcg(reinterpret_cast<const float4*>(src));
      } else {
        if (gr < n) v.x = __ldcg(src);
        if (gr + 1 < n) v.y = __ldcg(src + 1);
        if (gr + 2 < n) v.z = __ldcg(src + 2);
      }
    }
    *reinterpret_cast<float4*>(&Ts[c * NB + r4]) = v;
  }
}

// a dense 64 x 64 tile copied as it is (4096 floats, 16-byte aligned)
JMG_DEV void load_dense(float* Ts, const float* src) {
  float4 v[NB * NB / 4 / TH];
#pragma unroll
  for (int p = 0; p < NB * NB / 4 / TH; ++p)
    v[p] = __ldcg(reinterpret_cast<const float4*>(src) + threadIdx.x + p * TH);
#pragma unroll
  for (int p = 0; p < NB * NB / 4 / TH; ++p)
    reinterpret_cast<float4*>(Ts)[threadIdx.x + p * TH] = v[p];
}

// acc -= As Bs^T over k < 64: acc(r, c) -= sum_k As[k*64 + r] Bs[k*64 + c]
JMG_DEV void gemm_sub(float (&acc)[4][4], const float* As, const float* Bs) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll 8
  for (int k = 0; k < NB; ++k) {
    const float4 a = *reinterpret_cast<const float4*>(&As[k * NB + 4 * tx]);
    const float4 b = *reinterpret_cast<const float4*>(&Bs[k * NB + 4 * ty]);
    const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(-av[i], bv[j], acc[i][j]);
  }
}

// acc = fp32(A_IJ + shift I) (rows 4tx.., columns 4ty.. of the tile); entries
// past n: identity on diagonal tiles, zero elsewhere; zero above the diagonal
JMG_DEV void init_acc(float (&acc)[4][4], const double* A, int lda, int n, int I, int J,
                      double shift) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int c = 4 * ty + j, gc = J * NB + c;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = 4 * tx + i, gr = I * NB + r;
      float v;
      if (gr < n && gc < n) {
        if (I == J && r < c) {
          v = 0.0f;
        } else {
          double d = A[(size_t)gc * lda + gr];
          if (I == J && r == c) d += shift;
          v = (float)d;
        }
      } else {
        v = (I == J && r == c) ? 1.0f : 0.0f;
      }
      acc[i][j] = v;
    }
  }
}

// S[c * LDS + r] = acc(r, c) (scale: 1 or -1)
JMG_DEV void acc_to_S(float* S, const float (&acc)[4][4], float scale) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int i = 0; i < 4; ++i) S[(4 * ty + j) * LDS + 4 * tx + i] = scale * acc[i][j];
}

// Cholesky of the 64 x 64 tile S (LDS, lower) in FP32, in place, over four
// 16-wide panels: (a) the 16 x 16 diagonal block by one warp in registers
// (lane r holds row r; the unscaled right-looking update shares each column
// through shared memory), (b) the rows below it by substitution, one thread per
// row,
// (c) the rank-16 update of the trailing lower triangle in 4 x 4 tiles.  Returns 0 or the
// 1-based index of the first pivot that is not > 0 and lies within the valid
// order `rows` (the rest of the tile is the identity); every thread returns
// the same value.
JMG_DEV int potf2_64(float* S, int rows, float* rinv, int* s_bc) {
  const int t = threadIdx.x, lane = t & 31;
  for (int c0 = 0; c0 < NB; c0 += 16) {
    if (t < 32) {
      // lane (r, h) holds row r, columns 8h .. 8h+7 of the 16 x 16 block
      const int r = lane & 15, h = lane >> 4;
      float a[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) a[j] = S[(c0 + 8 * h + j) * LDS + c0 + r];
      int fail = 0;
      // unscaled right-looking: a_rm -= a_rk a_mk / d_k.  Each step the half
      // holding column k puts it in shared memory (double-buffered by step);
      // every lane reads the pivot, its own a_rk and the a_mk of its columns
      // back as broadcasts (15 shuffles per step by one half-warp measured
      // ~3x slower)
      __shared__ float colb[2][16];
      __shared__ float piv[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        if (h == (k >> 3)) colb[k & 1][r] = a[k & 7];
        __syncwarp();
        float d = colb[k & 1][k];
        if (lane == 0) piv[k] = d;
        if (!(d > 0.0f) && !fail) fail = c0 + k + 1;
        if (fail) d = 1.0f;  // keep going on harmless numbers; the tile is dropped
        float rd;  // 1/d to within an ulp (an FP32 preconditioner; IEEE division would sit on the chain)
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rd) : "f"(d));
        const float akw = colb[k & 1][r] * rd;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int m = 8 * h + j;
          if (m > k && r >= m) a[j] = fmaf(-akw, colb[k & 1][m], a[j]);
        }
      }
      __syncwarp();
      // l_kk = sqrt(d_k), l_rk = a_rk / sqrt(d_k)
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int k = 8 * h + j;
        const float dk = piv[k];
        const float il = rsqrtf(fail ? 1.0f : dk);
        a[j] = r > k ? a[j] * il : (r == k ? dk * il : a[j]);
        if (r == k) rinv[c0 + k] = il;
      }
      if (!fail) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int k = 8 * h + j;
          const float v = a[j];
          if (k <= r) S[(c0 + k) * LDS + c0 + r] = v;
        }
      }
      if (lane == 0) s_bc[2] = fail;
    }
    __syncthreads();
    const int fail = s_bc[2];
    if (fail) return fail <= rows ? fail : 0;
    const int m = NB - 16 - c0;  // rows below the block
    if (t < m) {
      const int R = c0 + 16 + t;
      float x[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) x[k] = S[(c0 + k) * LDS + R];
#pragma unroll
      for (int k = 0; k < 16; ++k) {
#pragma unroll
        for (int q = 0; q < k; ++q) x[k] = fmaf(-x[q], S[(c0 + q) * LDS + c0 + k], x[k]);
        x[k] *= rinv[c0 + k];
      }
#pragma unroll
      for (int k = 0; k < 16; ++k) S[(c0 + k) * LDS + R] = x[k];
    }
    __syncthreads();
    // rank-16 update of the trailing lower triangle, one 4 x 4 tile per thread
    const int nt4 = m / 4;
    if (t < nt4 * (nt4 + 1) / 2) {
      int I = 0, J = t;  // tile (I, J), J <= I, numbered row by row
      while (J > I) {
        J -= I + 1;
        ++I;
      }
      const int r0 = c0 + 16 + 4 * I, q0 = c0 + 16 + 4 * J;
      float acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        float xr[4], xc[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          xr[i] = S[(c0 + k) * LDS + r0 + i];
          xc[i] = S[(c0 + k) * LDS + q0 + i];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(xr[i], xc[j], acc[i][j]);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (r0 + i >= q0 + j) S[(q0 + j) * LDS + r0 + i] -= acc[i][j];
    }
    __syncthreads();
  }
  return 0;
}

// X L^T = S for the tile S (LDS), in place; L (64 x 64, leading dimension 64,
// L(c', c) at L[c * 64 + c']) lower with rinv[c] = 1 / L(c, c).  Four threads
// per row (lanes of one warp), thread g holding the columns c = g (mod 4) in
// registers:  x_c = s_c / L(c, c), then s_c' -= x_c L(c', c) for c' > c.
JMG_DEV void trsm_rows(float* S, const float* L, const float* rinv) {
  const int t = threadIdx.x, lane = t & 31;
  const int r = (t >> 5) * 8 + (lane >> 2), g = lane & 3, base = lane & ~3;
  float s[16];
#pragma unroll
  for (int m = 0; m < 16; ++m) s[m] = S[(4 * m + g) * LDS + r];
#pragma unroll
  for (int c = 0; c < NB; ++c) {
    const float xo = s[c >> 2] * rinv[c];
    const float x = __shfl_sync(0xffffffffu, xo, base + (c & 3));
    if (g == (c & 3)) s[c >> 2] = x;
#pragma unroll
    for (int m = c >> 2; m < 16; ++m)
      if (4 * m + g > c) s[m] = fmaf(-x, L[c * NB + 4 * m + g], s[m]);
  }
#pragma unroll
  for (int m = 0; m < 16; ++m) S[(4 * m + g) * LDS + r] = s[m];
}

// store the tile S (LDS) to W: rows and columns below n; diagonal tiles only
// their lower triangle
JMG_DEV void store_tile(const float* S, float* W, int ldw, int n, int I, int J) {
  for (int e = threadIdx.x; e < NB * NB; e += TH) {
    const int r = e % NB, c = e / NB, gr = I * NB + r, gc = J * NB + c;
    if (gr < n && gc < n && (I != J || r >= c)) W[(size_t)gc * ldw + gr] = S[c * LDS + r];
  }
}

// FP64 tile of the symmetric A (from its lower triangle) into Ad (LDS):
// Ad[c * LDS + r] = A(I*64 + r, J*64 + c), zero past n; |.| if ABS
template <bool ABS>
JMG_DEV void load_Ad(double* Ad, const double* A, int lda, int n, int I, int J) {
#pragma unroll 8
  for (int p = 0; p < NB * NB / TH; ++p) {
    const int e = threadIdx.x + p * TH;
    const int r = e % NB, c = e / NB, gr = I * NB + r, gc = J * NB + c;
    double v = 0.0;
    if (gr < n && gc < n) v = gr >= gc ? A[(size_t)gc * lda + gr] : A[(size_t)gr * lda + gc];
    Ad[c * LDS + r] = ABS ? fabs(v) : v;
  }
}

}  // namespace sm
}  // namespace jmg

namespace jmg {
namespace sm {

// shared-memory map (bytes): factor T0 [64 x 65 f32] | As [64 x 64 f32] |
// Bs [64 x 64 f32]; residual Ad [64 x 65 f64] | XJ | XI [64 x CR f64]; solve
// passes: staged right-hand side [ldw x SCR f32] | partial sums
// [16 x 64 x SCR f32]; then the misc words.
constexpr int OFF_AS = NB * LDS * 4;
constexpr int OFF_BS = OFF_AS + NB * NB * 4;
constexpr int OFF_MISC = OFF_BS + NB * NB * 4;
constexpr int OFF_RED = NMAX * SCR * 4;
constexpr int SMEM_BYTES = OFF_MISC + NB * 4 + 3 * RMAX * 8 + 16;
static_assert(NB * LDS * 8 + 2 * NB * CR * 8 <= OFF_MISC, "residual tiles overlap misc");
static_assert(OFF_RED + 16 * NB * SCR * 4 <= OFF_MISC, "solve staging overlaps misc");

struct Smem {
  unsigned char* raw;
  float *T0, *As, *Bs, *rinv;
  double *sc, *isc, *etas;  // scales of the solve (powers of two), their inverses
  int* bc;
  __device__ explicit Smem(unsigned char* r)
      : raw(r),
        T0(reinterpret_cast<float*>(r)),
        As(reinterpret_cast<float*>(r + OFF_AS)),
        Bs(reinterpret_cast<float*>(r + OFF_BS)),
        rinv(reinterpret_cast<float*>(r + OFF_MISC)),
        sc(reinterpret_cast<double*>(r + OFF_MISC + NB * 4)),
        isc(reinterpret_cast<double*>(r + OFF_MISC + NB * 4 + RMAX * 8)),
        etas(reinterpret_cast<double*>(r + OFF_MISC + NB * 4 + 2 * RMAX * 8)),
        bc(reinterpret_cast<int*>(r + OFF_MISC + NB * 4 + 3 * RMAX * 8)) {}
};

JMG_DEV float* lv_tile(const SmallArgs& a, int I, int J) {
  return a.Lv + (size_t)cm(a.nt, I, J) * NB * NB;
}

// Pieces of the factorisation (see the header); each returns false when the
// tile loop must be left (a failed factorisation or a wait that ran out).

// T0 holds the updated tile (i, j), i > j: solve X L_jj^T = T0 in place,
// store and publish it (T0 keeps L_ij)
JMG_DEV bool sub_finish(const SmallArgs& a, const Smem& S, int i, int j, int tr) {
  SmallCtl* C = a.ctl;
  const int epoch = tr + 1;
  if (!wait_flags(C, &C->ready[cm(a.nt, j, j)], nullptr, epoch, tr, a.wait_ns, S.bc))
    return false;
  load_L(S.As, a.W, a.ldw, a.n, j, j);
  __syncthreads();
  if (threadIdx.x < NB) S.rinv[threadIdx.x] = 1.0f / S.As[threadIdx.x * NB + threadIdx.x];
  __syncthreads();
  trsm_rows(S.T0, S.As, S.rinv);
  __syncthreads();
  store_tile(S.T0, a.W, a.ldw, a.n, i, j);
  publish(&C->ready[cm(a.nt, i, j)], epoch);
  return true;
}

// T0 holds the updated diagonal tile (j, j): factor, store, publish; then
// invert it (Y L^T = I by the same substitution as the panel solve, so
// Y = L^{-T}) into Li (column-major) and its row-major Lv tile
JMG_DEV bool diag_finish(const SmallArgs& a, const Smem& S, int j, int tr) {
  SmallCtl* C = a.ctl;
  const int nt = a.nt, epoch = tr + 1;
  const int f = potf2_64(S.T0, min(NB, a.n - j * NB), S.rinv, S.bc);
  if (f) {
    if (threadIdx.x == 0) atomicCAS(&C->fail[tr], 0, j * NB + f);
    return false;
  }
  store_tile(S.T0, a.W, a.ldw, a.n, j, j);
  publish(&C->ready[cm(nt, j, j)], epoch);
  for (int e = threadIdx.x; e < NB * NB; e += TH) {
    const int r = e % NB, c = e / NB;
    S.As[c * NB + r] = S.T0[c * LDS + r];
    S.T0[c * LDS + r] = r == c ? 1.0f : 0.0f;
  }
  __syncthreads();
  trsm_rows(S.T0, S.As, S.rinv);  // T0(r, c) = Linv(c, r)
  __syncthreads();
  float* li = a.Li + (size_t)j * NB * NB;
  float* lv = lv_tile(a, j, j);
  for (int e = threadIdx.x; e < NB * NB; e += TH) {
    const int x = e / NB, y = e % NB;  // li: column x, row y;  lv: row x, column y
    li[e] = S.T0[y * LDS + x];         // Linv(y, x) = T0(x, y)
    lv[e] = S.T0[x * LDS + y];         // Linv(x, y) = T0(y, x)
  }
  publish(&C->inv[cm(nt, j, j)], epoch);
  return true;
}

// Work items of the factorisation, column by column; the item of the tile
// (j + 1, j) also does the diagonal tile (j + 1, j + 1), so the last product
// of a diagonal tile and its panel solve need no flag between them:
//   column 0: (0, 0), (1, 0)+(1, 1), (2, 0), ..., (nt-1, 0);
//   column j >= 1: (j+1, j)+(j+1, j+1), (j+2, j), ..., (nt-1, j).
// An item depends only on items with smaller numbers.
JMG_DEV int n_items(int nt) { return nt + (nt - 1) * (nt - 2) / 2; }
JMG_DEV void item_inv(int nt, int u, int& i, int& j) {
  j = 0;
  for (;;) {
    const int cnt = j == 0 ? nt : nt - 1 - j;
    if (u < cnt) break;
    u -= cnt;
    ++j;
  }
  i = j == 0 ? u : j + 1 + u;
}

JMG_DEV bool factor_item(const SmallArgs& a, const Smem& S, int i, int j, int tr, double shift) {
  __syncthreads();  // the previous item's shared data is dead
  const bool merged = i == j + 1;
  float acc[4][4], dacc[4][4];
  init_acc(acc, a.A, a.lda, a.n, i, j, shift);
  if (merged) init_acc(dacc, a.A, a.lda, a.n, i, i, shift);
  for (int k = 0; k < j; ++k) {  // acc -= L_ik L_jk^T (and dacc -= L_ik L_ik^T)
    SmallCtl* C = a.ctl;
    if (!wait_flags(C, &C->ready[cm(a.nt, i, k)], i != j ? &C->ready[cm(a.nt, j, k)] : nullptr,
                    tr + 1, tr, a.wait_ns, S.bc))
      return false;
    load_L(S.As, a.W, a.ldw, a.n, i, k);
    if (i != j) load_L(S.Bs, a.W, a.ldw, a.n, j, k);
    __syncthreads();
    gemm_sub(acc, S.As, i != j ? S.Bs : S.As);
    if (merged) gemm_sub(dacc, S.As, S.As);
    __syncthreads();
  }
  acc_to_S(S.T0, acc, 1.0f);
  __syncthreads();
  if (i == j) return diag_finish(a, S, j, tr);
  if (i != j + 1) return sub_finish(a, S, i, j, tr);
  // (j + 1, j), then the diagonal tile (i, i): its products with k < j came
  // with those of (i, j) (same tiles L_ik), then the panel solve, then the last
  // product with the tile just solved, from shared memory
  if (!sub_finish(a, S, i, j, tr)) return false;
  for (int e = threadIdx.x; e < NB * NB; e += TH) {
    const int r = e % NB, k = e / NB;
    S.As[k * NB + r] = S.T0[k * LDS + r];
  }
  __syncthreads();
  gemm_sub(dacc, S.As, S.As);
  __syncthreads();
  acc_to_S(S.T0, dacc, 1.0f);
  __syncthreads();
  return diag_finish(a, S, i, tr);
}

// One inverse tile below the diagonal:
//   Linv_ij = -Linv_ii sum_{k=j..i-1} L_ik Linv_kj,
// row-major into Lv.
JMG_DEV bool inverse_tile(const SmallArgs& a, const Smem& S, int i, int j, int tr) {
  const int nt = a.nt, n = a.n, epoch = tr + 1;
  SmallCtl* C = a.ctl;
  __syncthreads();
  float acc[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[p][q] = 0.0f;
  for (int k = j; k < i; ++k) {  // acc = -sum_k L_ik Linv_kj
    if (!wait_flags(C, &C->ready[cm(nt, i, k)], &C->inv[cm(nt, k, j)], epoch, tr, a.wait_ns,
                    S.bc))
      return false;
    load_L(S.As, a.W, a.ldw, n, i, k);
    load_dense(S.Bs, lv_tile(a, k, j));
    __syncthreads();
    gemm_sub(acc, S.As, S.Bs);
    __syncthreads();
  }
  if (!wait_flags(C, &C->inv[cm(nt, i, i)], nullptr, epoch, tr, a.wait_ns, S.bc)) return false;
  load_dense(S.As, a.Li + (size_t)i * NB * NB);  // As[k*64 + r] = Linv_ii(r, k)
  {
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int p = 0; p < 4; ++p)  // Bs[k*64 + c] = acc(k, c)
      *reinterpret_cast<float4*>(&S.Bs[(4 * tx + p) * NB + 4 * ty]) =
          make_float4(acc[p][0], acc[p][1], acc[p][2], acc[p][3]);
  }
  __syncthreads();
  float out[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) out[p][q] = 0.0f;
  gemm_sub(out, S.As, S.Bs);  // out = -Linv_ii acc = Linv_ii sum_k L_ik Linv_kj
  {
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float* lv = lv_tile(a, i, j);
#pragma unroll
    for (int p = 0; p < 4; ++p)
      *reinterpret_cast<float4*>(&lv[(4 * tx + p) * NB + 4 * ty]) =
          make_float4(-out[p][0], -out[p][1], -out[p][2], -out[p][3]);
  }
  publish(&C->inv[cm(nt, i, j)], epoch);
  return true;
}

// |A| row sums of this CTA's tiles: slot 0 rows I (the whole symmetric tile on
// the diagonal), slot 1 rows J (column sums of an off-diagonal tile)
JMG_DEV void row_sums(const SmallArgs& a, unsigned char* raw) {
  double* Ad = reinterpret_cast<double*>(raw);
  for (int tl = blockIdx.x; tl < a.ntiles; tl += gridDim.x) {
    int I, J;
    cm_inv(a.nt, tl, I, J);
    __syncthreads();
    load_Ad<true>(Ad, a.A, a.lda, a.n, I, J);
    __syncthreads();
    const int t = threadIdx.x;
    if (t < NB) {
      double s = 0.0;
      for (int c = 0; c < NB; ++c) s += Ad[c * LDS + t];
      a.rs[((size_t)tl * 2 + 0) * NB + t] = s;
    } else if (t < 2 * NB && I != J) {
      const int c = t - NB;
      double s = 0.0;
      for (int r = 0; r < NB; ++r) s += Ad[c * LDS + r];
      a.rs[((size_t)tl * 2 + 1) * NB + c] = s;
    }
  }
  __syncthreads();
}

// Partial products of the residual: tile (I, J) of lower(A) gives A_IJ X_J
// (slot 0, rows I) and, off the diagonal, A_IJ^T X_I (slot 1, rows J), FP64.
JMG_DEV void resid_tiles(const SmallArgs& a, unsigned char* raw) {
  double* Ad = reinterpret_cast<double*>(raw);
  double* XJ = Ad + NB * LDS;
  double* XI = XJ + NB * CR;
  const int t = threadIdx.x, n = a.n, nrhs = a.nrhs;
  for (int tl = blockIdx.x; tl < a.ntiles; tl += gridDim.x) {
    int I, J;
    cm_inv(a.nt, tl, I, J);
    __syncthreads();
    load_Ad<false>(Ad, a.A, a.lda, n, I, J);
    for (int q0 = 0; q0 < nrhs; q0 += CR) {
      for (int e = t; e < NB * CR; e += TH) {
        const int c = e / CR, q = q0 + e % CR;
        const int gj = J * NB + c, gi = I * NB + c;
        XJ[e] = (gj < n && q < nrhs) ? __ldcg(a.X + (size_t)q * n + gj) : 0.0;
        XI[e] = (gi < n && q < nrhs) ? __ldcg(a.X + (size_t)q * n + gi) : 0.0;
      }
      __syncthreads();
      const int r = t & (NB - 1), qg = t >> 6;
#pragma unroll
      for (int h = 0; h < CR / 4; ++h) {
        const int q = qg + 4 * h;
        if (q0 + q >= nrhs) continue;
        double s0 = 0.0;
        for (int c = 0; c < NB; ++c) s0 = fma(Ad[c * LDS + r], XJ[c * CR + q], s0);
        a.part[(((size_t)tl * 2 + 0) * nrhs + q0 + q) * NB + r] = s0;
        if (I != J) {
          double s1 = 0.0;  // here r plays the column of the tile
          for (int k = 0; k < NB; ++k) s1 = fma(Ad[r * LDS + k], XI[k * CR + q], s1);
          a.part[(((size_t)tl * 2 + 1) * nrhs + q0 + q) * NB + r] = s1;
        }
      }
      __syncthreads();
    }
  }
}

JMG_DEV unsigned long long abs_bits(double v) {
  return isnan(v) ? 0x7FFFFFFFFFFFFFFFull : (unsigned long long)__double_as_longlong(fabs(v));
}
JMG_DEV unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

// R = B - (sum of the partial products, tiles in a fixed order) for the row
// tiles of this CTA, with the column maxima of |R|, |X|, |B| into cmx; with
// `first`, also ||A||_inf from the row sums.
JMG_DEV void reduce_rows(const SmallArgs& a, unsigned long long* cmx, bool first) {
  const int t = threadIdx.x, n = a.n, nrhs = a.nrhs, nt = a.nt, lane = t & 31;
  SmallCtl* C = a.ctl;
  for (int I = blockIdx.x; I < nt; I += gridDim.x) {
    for (int base = 0; base < NB * nrhs; base += TH) {
      const int e = base + t, r = e & (NB - 1), q = e >> 6, gr = I * NB + r;
      unsigned long long br = 0, bx = 0, bb = 0;
      if (e < NB * nrhs && gr < n) {
        double s = 0.0;  // fixed order; the loads are issued ahead
#pragma unroll 8
        for (int J = 0; J <= I; ++J)
          s += __ldcg(a.part + (((size_t)cm(nt, I, J) * 2 + 0) * nrhs + q) * NB + r);
#pragma unroll 8
        for (int J = I + 1; J < nt; ++J)
          s += __ldcg(a.part + (((size_t)cm(nt, J, I) * 2 + 1) * nrhs + q) * NB + r);
        const double b = a.B[(size_t)q * a.ldb + gr], x = __ldcg(a.X + (size_t)q * n + gr);
        const double rr = b - s;
        a.R[(size_t)q * n + gr] = rr;
        br = abs_bits(rr), bx = abs_bits(x), bb = abs_bits(b);
      }
      br = warp_max_u64(br), bx = warp_max_u64(bx), bb = warp_max_u64(bb);
      if (lane == 0 && base + t < NB * nrhs) {  // one column per warp (64 | NB * nrhs)
        atomicMax(&cmx[q], br);
        atomicMax(&cmx[RMAX + q], bx);
        atomicMax(&cmx[2 * RMAX + q], bb);
      }
    }
    if (first && t < NB) {
      const int gr = I * NB + t;
      unsigned long long bs = 0;
      if (gr < n) {
        double s = 0.0;
#pragma unroll 8
        for (int J = 0; J <= I; ++J) s += __ldcg(a.rs + ((size_t)cm(nt, I, J) * 2 + 0) * NB + t);
#pragma unroll 8
        for (int J = I + 1; J < nt; ++J)
          s += __ldcg(a.rs + ((size_t)cm(nt, J, I) * 2 + 1) * NB + t);
        bs = abs_bits(s);
      }
      bs = warp_max_u64(bs);
      if (lane == 0) atomicMax(&C->anorm_bits, bs);
    }
  }
}

}  // namespace sm
}  // namespace jmg

namespace jmg {
namespace sm {

// ------------------------------------------------------------------ solve
//
// Both passes read the row-major inverse tiles with 16 lanes across a tile row
// (float4 each: 256 contiguous bytes) and 16 row groups; thread (cg, rg) takes
// the columns 4cg..4cg+3 and the rows rg + 16m (m < 4) of every tile.

// y_I = sum_{J<=I} Linv_IJ d_J for the row blocks I of this CTA, with
// d = fp32(src / sc) (SCR columns at a time), into Y.
JMG_DEV void ypass(const SmallArgs& a, const Smem& S, const double* src, int lds) {
  float* dst = reinterpret_cast<float*>(S.raw);            // d: [row][SCR]
  float* red = reinterpret_cast<float*>(S.raw + OFF_RED);  // [cg][row][SCR]
  const int t = threadIdx.x, n = a.n, nrhs = a.nrhs, ldw = a.ldw;
  const int cg = t & 15, rg = t >> 4;
  for (int I = blockIdx.x; I < a.nt; I += gridDim.x) {
    const int rows = (I + 1) * NB;
    for (int q0 = 0; q0 < nrhs; q0 += SCR) {
      __syncthreads();
#pragma unroll 8
      for (int e = t; e < rows * SCR; e += TH) {
        const int rr = e / SCR, q = q0 + e % SCR;
        float v = 0.0f;
        if (rr < n && q < nrhs) v = (float)(__ldcg(src + (size_t)q * lds + rr) * S.isc[q]);
        dst[e] = v;
      }
      __syncthreads();
      float acc[4][SCR];
#pragma unroll
      for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int q = 0; q < SCR; ++q) acc[m][q] = 0.0f;
#pragma unroll 2
      for (int J = 0; J <= I; ++J) {
        const float* lv = lv_tile(a, I, J);
        float4 l[4];
#pragma unroll
        for (int m = 0; m < 4; ++m)
          l[m] = __ldcg(reinterpret_cast<const float4*>(lv + (rg + 16 * m) * NB + 4 * cg));
        const float4* d4 = reinterpret_cast<const float4*>(dst) + J * NB + 4 * cg;
        const float4 d0 = d4[0], d1 = d4[1], d2 = d4[2], d3 = d4[3];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          acc[m][0] = fmaf(l[m].x, d0.x, fmaf(l[m].y, d1.x, fmaf(l[m].z, d2.x, fmaf(l[m].w, d3.x, acc[m][0]))));
          acc[m][1] = fmaf(l[m].x, d0.y, fmaf(l[m].y, d1.y, fmaf(l[m].z, d2.y, fmaf(l[m].w, d3.y, acc[m][1]))));
          acc[m][2] = fmaf(l[m].x, d0.z, fmaf(l[m].y, d1.z, fmaf(l[m].z, d2.z, fmaf(l[m].w, d3.z, acc[m][2]))));
          acc[m][3] = fmaf(l[m].x, d0.w, fmaf(l[m].y, d1.w, fmaf(l[m].z, d2.w, fmaf(l[m].w, d3.w, acc[m][3]))));
        }
      }
#pragma unroll
      for (int m = 0; m < 4; ++m)
        *reinterpret_cast<float4*>(&red[(cg * NB + rg + 16 * m) * SCR]) =
            make_float4(acc[m][0], acc[m][1], acc[m][2], acc[m][3]);
      __syncthreads();
      for (int e = t; e < NB * SCR; e += TH) {
        const int r = e / SCR, q = e % SCR;
        float v = 0.0f;
        for (int g = 0; g < 16; ++g) v += red[(g * NB + r) * SCR + q];
        a.Y[(size_t)(q0 + q) * ldw + I * NB + r] = v;
      }
    }
  }
}

// x_J = sum_{I>=J} Linv_IJ^T y_I for the column blocks J of this CTA, then
// X (first: =, else +=) sc * x.
JMG_DEV void xpass(const SmallArgs& a, const Smem& S, bool first) {
  float* ys = reinterpret_cast<float*>(S.raw);             // y rows J*64..: [row][SCR]
  float* red = reinterpret_cast<float*>(S.raw + OFF_RED);  // [rg][col][SCR]
  const int t = threadIdx.x, n = a.n, nrhs = a.nrhs, ldw = a.ldw, nt = a.nt;
  const int cg = t & 15, rg = t >> 4;
  for (int J = blockIdx.x; J < nt; J += gridDim.x) {
    const int rows = (nt - J) * NB;
    for (int q0 = 0; q0 < nrhs; q0 += SCR) {
      __syncthreads();
#pragma unroll 8
      for (int e = t; e < rows * SCR; e += TH) {
        const int rr = e / SCR, q = e % SCR;
        ys[e] = __ldcg(a.Y + (size_t)(q0 + q) * ldw + J * NB + rr);
      }
      __syncthreads();
      float acc[4][SCR];  // [column c4 + i][q]
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < SCR; ++q) acc[i][q] = 0.0f;
#pragma unroll 2
      for (int I = J; I < nt; ++I) {
        const float* lv = lv_tile(a, I, J);
        float4 l[4];
#pragma unroll
        for (int m = 0; m < 4; ++m)
          l[m] = __ldcg(reinterpret_cast<const float4*>(lv + (rg + 16 * m) * NB + 4 * cg));
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const float4 y = reinterpret_cast<const float4*>(ys)[(I - J) * NB + rg + 16 * m];
          const float lm[4] = {l[m].x, l[m].y, l[m].z, l[m].w};
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            acc[i][0] = fmaf(lm[i], y.x, acc[i][0]);
            acc[i][1] = fmaf(lm[i], y.y, acc[i][1]);
            acc[i][2] = fmaf(lm[i], y.z, acc[i][2]);
            acc[i][3] = fmaf(lm[i], y.w, acc[i][3]);
          }
        }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
        *reinterpret_cast<float4*>(&red[(rg * NB + 4 * cg + i) * SCR]) =
            make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
      __syncthreads();
      for (int e = t; e < NB * SCR; e += TH) {
        const int c = e / SCR, q = q0 + e % SCR, gc = J * NB + c;
        if (gc >= n || q >= nrhs) continue;
        float v = 0.0f;
        for (int g = 0; g < 16; ++g) v += red[(g * NB + c) * SCR + e % SCR];
        const double x = S.sc[q] * (double)v;
        double* dx = a.X + (size_t)q * n + gc;
        *dx = first ? x : *dx + x;
      }
    }
  }
}

}  // namespace sm
}  // namespace jmg

namespace jmg {
namespace sm {

// Scale of a right-hand-side column for the FP32 solve: the power of two at
// or above its largest magnitude (1 for a zero, infinite or NaN column), so
// that scaling and unscaling are exact.
JMG_DEV double pow2_scale(double m) {
  if (!(m > 0.0) || !isfinite(m)) return 1.0;
  int e;
  frexp(m, &e);  // m = f 2^e, 0.5 <= f < 1
  return ldexp(1.0, e);
}

// The stopping rule on the reduced column maxima (every CTA evaluates it on the
// same numbers in the same order, so every CTA takes the same decision).
// Sets S.sc to the scales of the next correction.  Returns stop (0/1); CTA 0
// records the history.
JMG_DEV int decide(const SmallArgs& a, const Smem& S, const unsigned long long* cmx, double& prev,
                   int& stall, int& iters) {
  SmallCtl* C = a.ctl;
  const int t = threadIdx.x, nrhs = a.nrhs;
  const double an = from_bits(&C->anorm_bits);
  if (t < nrhs) {
    const double rm = from_bits(&cmx[t]), xm = from_bits(&cmx[RMAX + t]),
                 bm = from_bits(&cmx[2 * RMAX + t]);
    const double den = an * xm + bm;
    double e;
    if (isnan(rm) || isnan(den)) e = NAN;
    else if (den > 0.0) e = rm / den;
    else e = rm > 0.0 ? INFINITY : 0.0;
    S.etas[t] = e;
    S.sc[t] = pow2_scale(rm);
    S.isc[t] = 1.0 / S.sc[t];  // exact
  }
  __syncthreads();
  if (t == 0) {
    double e = 0.0;
    bool nan = false;
    for (int q = 0; q < nrhs; ++q) {
      if (isnan(S.etas[q])) nan = true;
      else e = fmax(e, S.etas[q]);
    }
    if (nan) e = NAN;
    int stp = 0, conv = 0;
    if (e <= a.tol) {
      stp = conv = 1;
    } else if (iters >= a.maxit || isnan(e)) {
      stp = 1;
    } else {
      stall = e > 0.5 * prev ? stall + 1 : 0;
      if (stall >= 3) stp = 1;
    }
    prev = e;
    if (blockIdx.x == 0) {
      const int h = C->n_hist;
      if (h < 32) C->eta_hist[h] = e;
      C->n_hist = h + 1;
      C->eta = e;
      C->converged = conv;
      C->iters = stp ? iters : iters + 1;
    }
    if (!stp) ++iters;
    S.bc[3] = stp;
  }
  __syncthreads();
  const int stp = S.bc[3];
  __syncthreads();
  return stp;
}

__global__ void __launch_bounds__(TH, 2) k_small_posv(SmallArgs a) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const Smem S(sm_raw);
  SmallCtl* C = a.ctl;
  const unsigned G = gridDim.x;
  unsigned kb = 0;  // grid barriers passed
  const int t = threadIdx.x, bid = blockIdx.x, n = a.n, nrhs = a.nrhs, nt = a.nt;
  const uint64_t lim = a.wait_ns;

  // max |a_ii| (the shift of a retry) and ||b_q||_inf (the first scaling);
  // read only after a grid barrier
  for (int i = bid * TH + t; i < n; i += (int)G * TH)
    amax_bits(&C->dmax_bits, a.A[(size_t)i * a.lda + i]);
  for (int r0 = bid * TH; r0 < n; r0 += (int)G * TH) {  // rows r0 + t, every column
    const int rr = r0 + t;
    for (int q = 0; q < nrhs; ++q) {
      const unsigned long long m =
          warp_max_u64(rr < n ? abs_bits(a.B[(size_t)q * a.ldb + rr]) : 0ull);
      if ((t & 31) == 0 && m) atomicMax(&C->bmax_bits[q], m);
    }
  }

  // 1-2: factorisation and inverse (with shifted retries)
  const int nfac = n_items(nt), ninv = a.ntiles - nt;
  double shift = 0.0;
  int tr = 0;
  for (;;) {
    for (int u = bid; u < nfac + ninv; u += (int)G) {
      int i, j;
      bool ok;
      if (u < nfac) {
        item_inv(nt, u, i, j);
        ok = factor_item(a, S, i, j, tr, shift);
      } else {
        cmo_inv(nt, u - nfac, i, j);
        ok = inverse_tile(a, S, i, j, tr);
      }
      if (!ok) break;
    }
    if (tr == 0) row_sums(a, sm_raw);
    if (!grid_sync(C, G, kb, lim, S.bc)) return;
    if (t == 0) S.bc[2] = ld_vol(&C->fail[tr]);
    __syncthreads();
    const int f = S.bc[2];
    __syncthreads();
    if (!f) break;
    if (!a.shift_retry || tr + 1 >= MAX_TRIES) {
      if (bid == 0 && t == 0) {
        C->info = f;
        C->tries = tr + 1;
        C->shift = shift;
        *a.info = f;
        atomicCAS(&C->status, 0, JMG_ERR_NOT_SPD);
      }
      return;
    }
    const double dmax = from_bits(&C->dmax_bits);
    shift = shift == 0.0 ? 4.0 * 0x1p-24 * dmax : 16.0 * shift;
    ++tr;
  }
  if (bid == 0 && t == 0) {
    C->tries = tr + 1;
    C->shift = shift;
  }

  // 3: X = M^{-1} B
  if (t < nrhs) {
    S.sc[t] = pow2_scale(from_bits(&C->bmax_bits[t]));
    S.isc[t] = 1.0 / S.sc[t];  // exact
  }
  __syncthreads();
  ypass(a, S, a.B, a.ldb);
  if (!grid_sync(C, G, kb, lim, S.bc)) return;
  xpass(a, S, true);

  // 4: refinement
  double prev = INFINITY;
  int stall = 0, iters = 0;
  for (int it = 0;; ++it) {
    unsigned long long* cmx = C->colmax_bits[it & 1];
    if (!grid_sync(C, G, kb, lim, S.bc)) return;
    resid_tiles(a, sm_raw);
    if (!grid_sync(C, G, kb, lim, S.bc)) return;
    reduce_rows(a, cmx, it == 0);
    if (!grid_sync(C, G, kb, lim, S.bc)) return;
    const int stop = decide(a, S, cmx, prev, stall, iters);
    if (bid == 0 && t < 3 * RMAX) C->colmax_bits[(it + 1) & 1][t] = 0ull;
    if (stop) break;
    ypass(a, S, a.R, n);
    if (!grid_sync(C, G, kb, lim, S.bc)) return;
    xpass(a, S, false);
  }

  // X -> B (X was last written before the barrier that preceded the decision)
  for (long long e = (long long)bid * TH + t; e < (long long)n * nrhs; e += (long long)G * TH) {
    const int rr = (int)(e % n), q = (int)(e / n);
    a.B[(size_t)q * a.ldb + rr] = __ldcg(a.X + e);
  }
  if (bid == 0 && t == 0) {
    *a.info = 0;
    if (!C->converged) atomicCAS(&C->status, 0, JMG_ERR_NOT_CONVERGED);
  }
}

}  // namespace sm

// ------------------------------------------------------------------ host

bool small_path_fits(int n, int nrhs) { return n >= 1 && n <= sm::NMAX && nrhs <= sm::RMAX; }

size_t small_workspace(int n, int nrhs) { return small_plan(n, nrhs).total; }

namespace {
struct SmallLaunch {
  int nsm = 0, per_sm = 0;
};
std::mutex g_small_mu;
std::vector<SmallLaunch> g_small;
}  // namespace

static int small_launch_shape(SmallLaunch* out) {
  int dev = 0;
  JMG_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_small_mu);
  if ((int)g_small.size() <= dev) g_small.resize(dev + 1);
  SmallLaunch& L = g_small[dev];
  if (L.nsm == 0) {
    JMG_TRY(ensure_smem(sm::k_small_posv, sm::SMEM_BYTES));
    JMG_CUDA(cudaDeviceGetAttribute(&L.nsm, cudaDevAttrMultiProcessorCount, dev));
    JMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&L.per_sm, sm::k_small_posv, sm::TH,
                                                           sm::SMEM_BYTES));
    if (L.per_sm < 1) {
      L.nsm = 0;
      return JMG_ERR_UNSUPPORTED;
    }
  }
  *out = L;
  return JMG_OK;
}

int small_posv(int n, int nrhs, const double* A, int lda, double* B, int ldb, int* info,
               const jmg_options& o, jmg_stats* st, void* work, cudaStream_t s) {
  const SmallPlan p = small_plan(n, nrhs);
  char* w = static_cast<char*>(work);
  SmallArgs a;
  a.n = n, a.nrhs = nrhs, a.lda = lda, a.ldb = ldb, a.ldw = p.ldw, a.nt = p.nt;
  a.ntiles = p.ntiles, a.maxit = o.maxit, a.shift_retry = o.shift_retry, a.tol = o.tol;
  a.wait_ns = g_wait_ns;
  a.A = A, a.B = B, a.info = info;
  a.W = reinterpret_cast<float*>(w + p.W);
  a.Li = reinterpret_cast<float*>(w + p.Li);
  a.Lv = reinterpret_cast<float*>(w + p.Lv);
  a.Y = reinterpret_cast<float*>(w + p.Y);
  a.X = reinterpret_cast<double*>(w + p.X);
  a.R = reinterpret_cast<double*>(w + p.R);
  a.part = reinterpret_cast<double*>(w + p.part);
  a.rs = reinterpret_cast<double*>(w + p.rs);
  a.ctl = reinterpret_cast<SmallCtl*>(w + p.ctl);
  SmallLaunch L;
  JMG_TRY(small_launch_shape(&L));
  // every item of the dataflow gets its own CTA when the GPU holds that many
  const int items = p.nt + (p.nt - 1) * (p.nt - 2) / 2 + (p.ntiles - p.nt);
  const int G = std::max(1, std::min(items, L.per_sm * L.nsm));
  JMG_CUDA(cudaMemsetAsync(a.ctl, 0, sizeof(SmallCtl), s));
  void* args[] = {&a};
  JMG_CUDA(cudaLaunchCooperativeKernel((const void*)sm::k_small_posv, dim3(G), dim3(sm::TH), args,
                                       (size_t)sm::SMEM_BYTES, s));
  JMG_TRY(launched());
  // the outcome (status, counters, history): one small read
  SmallCtl h;
  JMG_CUDA(cudaMemcpyAsync(&h, a.ctl, offsetof(SmallCtl, bmax_bits), cudaMemcpyDeviceToHost, s));
  JMG_CUDA(cudaStreamSynchronize(s));
  if (st) {
    st->status = h.status;
    st->info = h.info;
    st->iters = h.iters;
    st->refine_used = JMG_REFINE_IR;
    st->words_used = 1;
    st->factor_tries = h.tries;
    st->bwd_err = h.eta;
    st->shift = h.shift;
    st->anorm = __builtin_bit_cast(double, h.anorm_bits);
    st->n_resid = h.n_hist;
    st->n_hist = h.n_hist;
    for (int k = 0; k < 32; ++k) st->eta_hist[k] = h.eta_hist[k];
    st->n_solve = h.status == JMG_ERR_NOT_SPD ? 0 : 1 + h.iters;  // first solve + one per step
  }
  return h.status;
}

}  // namespace jmg
