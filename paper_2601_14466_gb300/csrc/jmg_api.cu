// jmg_api.cu -- C ABI and host-side drivers of the SPD solver.
//
// Paper: "Software design" -- the potrs workflow (Cholesky potrf followed by
// potrs, optional log det) issued as one call on the framework's stream.
//
// Plain path (prec NATIVE, FP64): right-looking blocked Cholesky in place
//   for each diagonal block k:  potf2 (FP64)  ->  panel TRSM (FP64)
//                               ->  trailing SYRK update (FP64 CUDA cores)
//   then blocked forward / back substitution.
// Mixed path (prec BF16 / FP16): the same loop on an FP32 working copy W of
//   lower(A) with FP64 diagonal blocks, an FP32 panel TRSM and tensor-core
//   trailing updates on 16-bit split words; the FP32 factor then
//   preconditions an FP64 refinement loop (residual in FP64 against the
//   untouched A) until the normwise backward error reaches `tol`.
#include <chrono>
#include <cmath>
#include <mutex>
#include <vector>

#include "../../include/jmg_dev.h"
#include "kernels.h"

namespace jmg {

// ---------------------------------------------------------------- workspace plan
struct Plan {
  size_t off_W = 0, off_PA = 0, off_PB = 0, off_X = 0, off_R = 0, off_D = 0, off_part = 0,
         off_colmax = 0, off_eta = 0, off_anorm = 0, off_rowsum = 0, off_ints = 0, off_Z = 0,
         off_P = 0, off_Q = 0, off_scal = 0, off_sync = 0, off_exp = 0, off_ozrow = 0,
         off_ozA = 0, off_ozX = 0, off_SV = 0, total = 0;
  bool split = false;
  int ldw = 0, ldp = 0, kext = 0, splits = 1, ldd = 0, NB = 0, lde = 0;
};

static void opts_or_default(const jmg_options* in, jmg_options* out) {
  if (in)
    *out = *in;
  else
    jmg_default_options(out);
  if (out->nb <= 0) out->nb = 128;
  if (out->NB <= 0) out->NB = out->nb;
  if (out->words <= 0) out->words = 1;
  if (out->words > 3) out->words = 3;
  if (out->tol <= 0) out->tol = 1e-13;
  if (out->maxit <= 0) out->maxit = 30;
}

static Plan plan_posv_mixed(int n, int nrhs, const jmg_options& o) {
  Plan p;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t at = off;
    off = round_up(off + bytes, 256);
    return at;
  };
  const size_t N = (size_t)n, R = (size_t)(nrhs > 0 ? nrhs : 1);
  p.ldw = (int)round_up(N > 0 ? N : 1, 32);
  p.ldd = p.ldw;  // the FP32 right-hand sides of the preconditioner solves
  p.kext = o.prec == JMG_PREC_FP8 ? o.nb : o.nb * split_pairs(o.words);  // one panel
  // outer block width: a multiple of the panel width, at most n rounded up
  p.NB = std::max(o.nb, std::min(o.NB / o.nb, cdiv(std::max(n, 1), o.nb)) * o.nb);
  p.ldp = (int)round_up((size_t)p.kext * (p.NB / o.nb), o.prec == JMG_PREC_FP8 ? 128 : 64);
  p.lde = n / 128 + 2;  // FP8 exponents per panel
  p.splits = residual_splits(n, nrhs > 0 ? nrhs : 1);
  // the factor and what a refine-only call (reuse_factor) needs come first, at
  // offsets that do not depend on nrhs
  p.off_W = take(sizeof(float) * (size_t)p.ldw * N);
  p.off_SV = take(sv_image_bytes(n));  // inverses and coupling blocks of the solves
  p.off_anorm = take(sizeof(double) * 2);  // [0] ||A||_inf, [1] shift of the factor
  p.off_ints = take(sizeof(int) * 8);
  p.split = o.resid != 1;  // tensor-core split products (auto or explicit)
  if (p.split) {
    p.off_ozrow = take(sizeof(double) * (N > 0 ? N : 1));
    p.off_ozA = take(oz_a_bytes(n));
  }
  p.off_PA = take(2 * N * p.ldp);  // 16-bit words, or e4m3 bytes for FP8
  p.off_exp = take((size_t)p.lde * (p.NB / o.nb));
  p.off_PB = take(2 * N * p.ldp);
  p.off_X = take(sizeof(double) * N * R);
  p.off_R = take(sizeof(double) * N * R);
  p.off_D = take(sizeof(float) * (size_t)p.ldd * R);
  if (p.split) {
    p.off_ozX = take(oz_x_bytes(n, nrhs > 0 ? nrhs : 1));
    p.splits = std::max(p.splits, oz_splits_used(n, nrhs > 0 ? nrhs : 1));
  }
  p.off_part = take(sizeof(double) * N * R * p.splits);
  p.off_colmax = take(sizeof(double) * 3 * R);
  p.off_eta = take(sizeof(double) * (1 + R));
  p.off_rowsum = take(sizeof(double) * (N > 0 ? N : 1));
  p.off_Z = take(sizeof(double) * N * R);
  p.off_P = take(sizeof(double) * N * R);
  p.off_Q = take(sizeof(double) * N * R);
  p.off_scal = take(sizeof(double) * 8 * R);
  p.off_sync = take(sizeof(int) * std::max(trsv_sync_ints(n, nrhs > 0 ? nrhs : 1),
                                            sv_sync_ints(n, nrhs > 0 ? nrhs : 1)));
  p.total = off;
  return p;
}

// scratch of the plain potrs / posv: the solve's tickets and flags only
static size_t plain_solve_bytes(int n, int nrhs) {
  if (n <= 0 || nrhs <= 0) return 0;
  return round_up(sizeof(int) * trsv_sync_ints(n, nrhs), 256);
}

// Side streams and events of the mixed path, created once per device on first
// use and kept for the life of the process (a call made on another thread
// shares them: events are re-recorded, which can only add dependencies).
struct DevAux {
  cudaStream_t hi = nullptr, lo = nullptr;  // high / low priority, non-blocking
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
};
static int dev_aux(DevAux** out) {
  static std::mutex mu;
  static DevAux aux[64];
  int dev = 0;
  JMG_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return JMG_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(mu);
  DevAux& a = aux[dev];
  if (!a.hi) {
    int prio_lo = 0, prio_hi = 0;
    JMG_CUDA(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
    JMG_CUDA(cudaStreamCreateWithPriority(&a.lo, cudaStreamNonBlocking, prio_lo));
    for (auto& e : a.ev) JMG_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    JMG_CUDA(cudaStreamCreateWithPriority(&a.hi, cudaStreamNonBlocking, prio_hi));
  }
  *out = &a;
  return JMG_OK;
}

template <typename T>
static T* at(void* work, size_t off) {
  return reinterpret_cast<T*>(reinterpret_cast<char*>(work) + off);
}

// ---------------------------------------------------------------- FP64 factor
// Plain factorisation in the storage type T (double: FP64 throughout; float:
// FP32 panel solves and trailing updates on the CUDA cores, the diagonal blocks
// in FP64 arithmetic).
template <typename T>
static int potrf_plain(int n, T* A, int lda, int nb, int* info, cudaStream_t s) {
  for (int k = 0; k < n; k += nb) {
    const int kb = std::min(nb, n - k);
    T* Akk = A + (size_t)k * lda + k;
    JMG_TRY(launch_potf2(Akk, lda, kb, k, info, s));
    const int m = n - k - kb;
    if (m <= 0) break;
    T* L21 = Akk + kb;
    JMG_TRY(launch_trsm(L21, lda, m, kb, Akk, info, s));
    JMG_TRY(launch_gemm<T>(m, m, kb, L21, lda, MODE_N, L21, lda, MODE_T,
                           A + (size_t)(k + kb) * lda + (k + kb), lda, OUT_SUB_LOWER, 1, info, s));
  }
  return JMG_OK;
}

// ---------------------------------------------------------------- mixed factor
// Factor the FP32 working matrix W (lower) in place; info_f and err are device
// ints of the workspace.  Two-level right-looking blocking:
//  * outer blocks of NB columns (a multiple of the panel width nb);
//  * inside a block, panel by panel: the panel solve below the diagonal block,
//    the panel's split words (or FP8 codes) into column slot p of the block's
//    operand, and the update of the block's remaining columns only (a narrow
//    trapezoid, depth one panel);
//  * after the block's last panel, ONE update of the whole trailing matrix with
//    the block's operand (depth NB words per pair): the read-modify-write of the
//    trailing matrix happens once per NB columns instead of once per panel.
// Every update is split in two: the next panel's columns first, then the rest
// on one SM fewer, while the next diagonal block (one CTA, bound by its serial
// chain) is factored on a second stream on the free SM.
static int factor_mixed(int n, float* W, int ldw, const jmg_options& o, const Plan& p,
                        void* work, int* info_f, int* err, cudaStream_t s) {
  const int nb = o.nb, NB = p.NB;
  const bool fp8 = o.prec == JMG_PREC_FP8;
  const int kp = fp8 ? nb : nb * split_pairs(o.words);  // operand columns of one panel
  char* PA = at<char>(work, p.off_PA);
  char* PB = split_pairs(o.words) > 1 ? at<char>(work, p.off_PB) : PA;
  signed char* ex = fp8 ? at<signed char>(work, p.off_exp) : nullptr;
  const int lde = p.lde;           // exponents: ex[panel * lde + 128-row tile of the operand]
  const size_t esz = fp8 ? 1 : 2;  // bytes per operand element
  // operand row r of the current block <-> row k0 + r of W
  auto opA = [&](size_t row, int col) { return PA + (row * p.ldp + col) * esz; };
  auto opB = [&](size_t row, int col) { return PB + (row * p.ldp + col) * esz; };
  // the high-priority side stream and its events (made once per device)
  DevAux* aux = nullptr;
  JMG_TRY(dev_aux(&aux));
  struct {
    cudaStream_t s2;
    cudaEvent_t panel, diag;
  } side{aux->hi, aux->ev[0], aux->ev[1]};
  int dev = 0, nsm = 152;
  JMG_CUDA(cudaGetDevice(&dev));
  JMG_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));

  // C (rows x cols trapezoid at W[r0, r0]) -= operand rows [orow, orow + rows) x K columns
  // [kc, kc + kext); FP8 exponents from panel kc / nb on (one chunk per panel)
  auto update = [&](int r0, int rows, int cols, size_t orow, int kc, int kext, int ctas) -> int {
    float* Cp = W + (size_t)r0 * ldw + r0;
    if (fp8)
      return launch_syrk_fp8(rows, cols, kext, opA(orow, kc), p.ldp,
                             ex + (size_t)(kc / nb) * lde + orow / 128, lde, Cp, ldw, err, s, ctas);
    return launch_syrk_tc(rows, cols, kext, opA(orow, kc), opB(orow, kc), p.ldp, o.prec, Cp, ldw,
                          err, s, ctas, 0, kp);
  };
  // the update of a trapezoid whose first nb columns hold the next diagonal
  // block: those columns first, the block on the side stream, then the rest
  auto update_lookahead = [&](int r0, int rows, int cols, size_t orow, int kc, int kext) -> int {
    const int pc = std::min(nb, cols);
    JMG_TRY(update(r0, rows, pc, orow, kc, kext, 0));
    JMG_CUDA(cudaEventRecord(side.panel, s));
    JMG_CUDA(cudaStreamWaitEvent(side.s2, side.panel, 0));
    JMG_TRY(launch_potf2(W + (size_t)r0 * ldw + r0, ldw, std::min(nb, rows), r0, info_f, side.s2));
    JMG_CUDA(cudaEventRecord(side.diag, side.s2));
    if (cols > pc && rows > pc)
      JMG_TRY(update(r0 + pc, rows - pc, cols - pc, orow + pc, kc, kext, nsm - 1));
    JMG_CUDA(cudaStreamWaitEvent(s, side.diag, 0));
    return JMG_OK;
  };

  JMG_TRY(launch_potf2(W, ldw, std::min(nb, n), 0, info_f, s));
  for (int k0 = 0; k0 < n; k0 += NB) {
    const int NBk = std::min(NB, n - k0);
    const int q = cdiv(NBk, nb);
    for (int pp = 0; pp < q; ++pp) {
      const int k = k0 + pp * nb, kb = std::min(nb, n - k), m = n - k - kb;
      if (m <= 0) break;
      float* Wkk = W + (size_t)k * ldw + k;
      float* L21 = Wkk + kb;
      JMG_TRY(launch_trsm(L21, ldw, m, kb, Wkk, info_f, s));
      const size_t orow = (size_t)(k + kb - k0);  // operand row of L21's first row
      if (fp8)
        JMG_TRY(launch_quant_fp8(m, kb, L21, ldw, opA(orow, pp * kp), p.ldp,
                                 ex + (size_t)pp * lde + orow / 128, s));
      else
        JMG_TRY(launch_split_words(m, kb, L21, ldw, o.prec, o.words, opA(orow, pp * kp),
                                   opB(orow, pp * kp), p.ldp, s));
      const int ncb = k0 + NBk - (k + kb);  // columns of this block right of the panel
      if (ncb > 0) {
        // the block's remaining columns, with this panel's words only
        JMG_TRY(update_lookahead(k + kb, m, ncb, orow, pp * kp, kp));
      } else {
        // the block is factored: the whole trailing matrix, with every panel of it
        JMG_TRY(update_lookahead(k + kb, m, m, orow, 0, q * kp));
      }
    }
  }
  // the solves' images: inverses of the diagonal blocks, coupling blocks, and
  // L mirrored into the upper triangle of W
  return sv_prepare(n, W, ldw, at<float>(work, p.off_SV), s);
}

// column max of |B| into colmax_r and R = B (start of refinement from X = 0)
__global__ void k_copy_colmax(int n, const double* __restrict__ B, int ldb, double* __restrict__ R,
                              double* __restrict__ colmax) {
  const int c = blockIdx.y;
  double m = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double v = B[(size_t)c * ldb + i];
    R[(size_t)c * n + i] = v;
    m = (isnan(v) || isnan(m)) ? NAN : fmax(m, fabs(v));
  }
  for (int o = 16; o > 0; o >>= 1) {
    double a = __shfl_xor_sync(0xffffffffu, m, o);
    m = (isnan(a) || isnan(m)) ? NAN : fmax(m, a);
  }
  if ((threadIdx.x & 31) == 0) atomic_max_nonneg(&colmax[c], m);
}

static double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

static int sync_read(void* host, const void* dev, size_t bytes, cudaStream_t s) {
  JMG_CUDA(cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, s));
  JMG_CUDA(cudaStreamSynchronize(s));
  return JMG_OK;
}

// M^{-1} R in FP32 with per-column scaling, added to X (FP64): X += s * (L L^T)^{-1} (R / s)
// `status` is a device int set to -1 if a device-side wait of the solve ran out.
static int precond_update(int n, int nrhs, const float* W, int ldw, const float* SV,
                          const double* R, const double* colmax_r, float* D, int ldd, double* X,
                          int* sync, int* status, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1) {
  JMG_TRY(launch_scale_to_f32(n, nrhs, R, n, colmax_r, D, ldd, s));
  if (e0) JMG_CUDA(cudaEventRecord(e0, s));
  JMG_TRY(sv_solve_llt(n, nrhs, W, ldw, SV, D, ldd, sync, status, s));
  if (e1) JMG_CUDA(cudaEventRecord(e1, s));
  JMG_TRY(launch_axpy_f32(n, nrhs, D, ldd, colmax_r, X, n, s));
  return JMG_OK;
}

// Refinement state of one mixed solve (device buffers carved from `work`).
struct MixedCtx {
  int n, nrhs, lda, ldb;
  const double* A;
  double* B;
  const Plan* p;
  const jmg_options* o;
  void* work;
  cudaStream_t s;
  float* W;
  double *X, *R, *Z, *P, *Q, *part, *colmax, *eta, *dsc, *rowsum, *rz, *rz_new, *pq;
  float* D;
  int* ints;  // [0] factor info, [1] factor err, [2] solve status, [3] PCG breakdown
  int* sync;
  cudaEvent_t ev[6];  // timing: [0,1] residual product, [2,3] solve, [4,5] factor
  bool solve_pending = false;
  jmg_stats* S;
  std::vector<double> eh;
};

static void hist(MixedCtx& c, double e) {
  if (c.S->n_hist < 32) c.S->eta_hist[c.S->n_hist] = e;
  c.S->n_hist++;
}

// Rout = Bin - A Xin (Bin == nullptr: Rout = A Xin) with column norms: the
// FP64 CUDA-core GEMM or the split tensor-core product.  The product kernel is
// timed with c.ev when timing is on.
static int product(MixedCtx& c, const double* Xin, const double* Bin, int ldbin, double* Rout) {
  if (!c.p->split)
    return launch_residual(c.n, c.nrhs, c.A, c.lda, Xin, c.n, Bin, ldbin, Rout, c.n, c.colmax,
                           c.part, c.p->splits, c.s, c.ev[0], c.ev[1]);
  JMG_CUDA(cudaMemsetAsync(c.colmax, 0, sizeof(double) * 3 * c.nrhs, c.s));
  if (c.ev[0]) JMG_CUDA(cudaEventRecord(c.ev[0], c.s));
  JMG_TRY(oz_product(c.n, c.nrhs, at<char>(c.work, c.p->off_ozA), at<double>(c.work, c.p->off_ozrow),
                     Xin, c.n, at<char>(c.work, c.p->off_ozX), c.part, &c.ints[1], c.s));
  if (c.ev[1]) JMG_CUDA(cudaEventRecord(c.ev[1], c.s));
  return launch_resid_reduce(c.n, c.nrhs, oz_splits_used(c.n, c.nrhs), c.part, Xin, c.n, Bin,
                             ldbin, Rout, c.n, c.colmax, c.s);
}

// after a stream synchronisation: add the timed solve (if one is pending)
static int collect_solve(MixedCtx& c) {
  if (!c.solve_pending) return JMG_OK;
  float ms = 0.f;
  JMG_CUDA(cudaEventElapsedTime(&ms, c.ev[2], c.ev[3]));
  c.S->t_solve_gpu_ms += ms;
  c.S->n_solve++;
  c.solve_pending = false;
  return JMG_OK;
}

// R = B - A X (true residual), eta -> host; returns max eta in c.eh[0]
static int true_residual(MixedCtx& c) {
  JMG_TRY(product(c, c.X, c.B, c.ldb, c.R));
  JMG_TRY(launch_eta(c.nrhs, c.colmax, c.dsc, c.eta, c.s));
  JMG_TRY(sync_read(c.eh.data(), c.eta, sizeof(double) * (1 + c.nrhs), c.s));
  c.S->n_resid++;
  if (c.o->timing) {
    float ms = 0.f;
    JMG_CUDA(cudaEventElapsedTime(&ms, c.ev[0], c.ev[1]));
    c.S->t_resid_gpu_ms += ms;
    JMG_TRY(collect_solve(c));
  }
  return JMG_OK;
}

// Z = M^{-1} R with the FP32 factor (per-column scaling by ||r_c||)
static int precond_to(MixedCtx& c, double* Zout) {
  JMG_TRY(launch_scale_to_f32(c.n, c.nrhs, c.R, c.n, c.colmax, c.D, c.p->ldd, c.s));
  if (c.ev[2]) JMG_CUDA(cudaEventRecord(c.ev[2], c.s));
  JMG_TRY(sv_solve_llt(c.n, c.nrhs, c.W, c.p->ldw, at<float>(c.work, c.p->off_SV), c.D, c.p->ldd,
                       c.sync, &c.ints[2], c.s));
  if (c.ev[3]) {
    JMG_CUDA(cudaEventRecord(c.ev[3], c.s));
    c.solve_pending = true;
  }
  return launch_scale_from_f32(c.n, c.nrhs, c.D, c.p->ldd, c.colmax, Zout, c.s);
}

// Preconditioned CG on A X = B from the current X and its true residual R,
// FP64 vectors, M = L L^T (the low-precision factor).  Stops when the
// recursively updated residual suggests eta <= tol / 2 (the caller then checks
// the true residual), at maxit, or on a breakdown (p^T A p <= 0).
static int pcg(MixedCtx& c, bool* breakdown) {
  const int n = c.n, nrhs = c.nrhs;
  *breakdown = false;
  JMG_TRY(precond_to(c, c.Z));
  JMG_CUDA(cudaMemcpyAsync(c.P, c.Z, sizeof(double) * (size_t)n * nrhs, cudaMemcpyDeviceToDevice,
                           c.s));
  JMG_TRY(launch_dot_cols(n, nrhs, c.R, n, c.Z, n, c.rz, c.s));
  while (c.S->iters < c.o->maxit) {
    // Q = A P (same FP64 kernel as the residual, without B)
    JMG_TRY(product(c, c.P, nullptr, n, c.Q));
    JMG_TRY(launch_dot_cols(n, nrhs, c.P, n, c.Q, n, c.pq, c.s));
    JMG_TRY(launch_pcg_step(n, nrhs, c.P, c.Q, c.rz, c.pq, c.X, c.R, c.colmax, &c.ints[3], c.s));
    JMG_TRY(launch_eta(nrhs, c.colmax, c.dsc, c.eta, c.s));
    int bad = 0;
    JMG_TRY(sync_read(c.eh.data(), c.eta, sizeof(double) * (1 + nrhs), c.s));
    JMG_TRY(sync_read(&bad, &c.ints[3], sizeof(int), c.s));
    if (c.o->timing) {
      float ms = 0.f;
      JMG_CUDA(cudaEventElapsedTime(&ms, c.ev[0], c.ev[1]));
      c.S->t_resid_gpu_ms += ms;
      JMG_TRY(collect_solve(c));
    }
    c.S->n_resid++;
    c.S->iters++;
    hist(c, c.eh[0]);
    if (bad || std::isnan(c.eh[0])) {
      *breakdown = true;
      return JMG_OK;
    }
    if (c.eh[0] <= 0.5 * c.o->tol) return JMG_OK;
    JMG_TRY(precond_to(c, c.Z));
    JMG_TRY(launch_dot_cols(n, nrhs, c.R, n, c.Z, n, c.rz_new, c.s));
    JMG_TRY(launch_pcg_dir(n, nrhs, c.Z, c.P, c.rz_new, c.rz, c.s));
    JMG_CUDA(cudaMemcpyAsync(c.rz, c.rz_new, sizeof(double) * nrhs, cudaMemcpyDeviceToDevice, c.s));
  }
  return JMG_OK;
}

static int posv_mixed(int n, int nrhs, const double* A, int lda, double* B, int ldb, int* info,
                      const jmg_options& o, jmg_stats* st, void* work, cudaStream_t s) {
  const Plan p = plan_posv_mixed(n, nrhs, o);
  jmg_stats local{};
  MixedCtx c;
  c.n = n, c.nrhs = nrhs, c.lda = lda, c.ldb = ldb, c.A = A, c.B = B, c.p = &p, c.o = &o;
  c.work = work, c.s = s;
  c.W = at<float>(work, p.off_W);
  c.X = at<double>(work, p.off_X);
  c.R = at<double>(work, p.off_R);
  c.Z = at<double>(work, p.off_Z);
  c.P = at<double>(work, p.off_P);
  c.Q = at<double>(work, p.off_Q);
  c.D = at<float>(work, p.off_D);
  c.part = at<double>(work, p.off_part);
  c.colmax = at<double>(work, p.off_colmax);
  c.eta = at<double>(work, p.off_eta);
  c.dsc = at<double>(work, p.off_anorm);  // [0] ||A||_inf, [1] shift, [2] max_i a_ii
  c.rowsum = at<double>(work, p.off_rowsum);
  c.rz = at<double>(work, p.off_scal);
  c.rz_new = c.rz + nrhs;
  c.pq = c.rz + 2 * nrhs;
  c.ints = at<int>(work, p.off_ints);
  c.sync = at<int>(work, p.off_sync);
  for (auto& e : c.ev) e = nullptr;
  c.S = st ? st : &local;
  c.eh.assign(1 + nrhs, 0.0);
  jmg_stats& S = *c.S;
  S = jmg_stats{};
  S.words_used = o.words;
  S.refine_used = JMG_REFINE_IR;
  if (o.timing) {
    for (auto& e : c.ev) JMG_CUDA(cudaEventCreate(&e));
  }
  struct EvGuard {
    cudaEvent_t* e;
    ~EvGuard() {
      for (int i = 0; i < 6; ++i)
        if (e[i]) cudaEventDestroy(e[i]);
    }
  } guard{c.ev};

  const double t0 = now_ms();
  // The prologue of the refinement -- ||A||_inf, and the row maxima and slices
  // of A for the split residual -- only feeds the first residual: it runs on a
  // low-priority side stream beside the factorisation and the initial solve.
  // Every return path leaves `s` waiting for it (stream order keeps the
  // workspace alive for it).
  struct Prologue {
    cudaStream_t main = nullptr, s3 = nullptr;
    cudaEvent_t start = nullptr, done = nullptr;
    bool pending = false;
    int wait() {
      if (pending) JMG_CUDA(cudaStreamWaitEvent(main, done, 0));
      pending = false;
      return JMG_OK;
    }
    ~Prologue() { (void)wait(); }
  } pro;
  pro.main = s;
  if (!o.reuse_factor) {
    DevAux* aux = nullptr;
    JMG_TRY(dev_aux(&aux));
    pro.s3 = aux->lo;  // the low-priority side stream and its events (made once per device)
    pro.start = aux->ev[2];
    pro.done = aux->ev[3];
    JMG_CUDA(cudaEventRecord(pro.start, s));  // A and the workspace are ready here
    JMG_CUDA(cudaStreamWaitEvent(pro.s3, pro.start, 0));
    if (p.split) {  // one pass for the row sums (||A||_inf) and row maxima (slice scales)
      double* rowmax = at<double>(work, p.off_ozrow);
      JMG_TRY(launch_row_stats(n, A, lda, c.rowsum, rowmax, pro.s3));
      JMG_TRY(launch_max_reduce(n, c.rowsum, &c.dsc[0], pro.s3));
      JMG_TRY(oz_slice_a(n, A, lda, rowmax, at<char>(work, p.off_ozA), pro.s3));
    } else {
      JMG_TRY(launch_norm_inf(n, A, lda, c.rowsum, &c.dsc[0], pro.s3));
    }
    JMG_CUDA(cudaEventRecord(pro.done, pro.s3));
    pro.pending = true;
    JMG_TRY(launch_diag_max(n, A, lda, &c.dsc[2], s));
    JMG_CUDA(cudaMemsetAsync(&c.dsc[1], 0, sizeof(double), s));
  }
  double h2[2] = {0, 0};  // shift, max_i a_ii
  JMG_TRY(sync_read(h2, &c.dsc[1], sizeof(h2), s));
  double shift = h2[0];
  const double dmax = h2[1];
  // unit roundoff of the factor: the split words, but never below FP32's
  const double u_f =
      o.prec == JMG_PREC_FP8
          ? std::ldexp(1.0, -4)
          : std::max(std::pow(o.prec == JMG_PREC_FP16 ? std::ldexp(1.0, -11) : std::ldexp(1.0, -8),
                              o.words),
                     std::ldexp(1.0, -24));
  // Diagonal shifts of the factor (a reading: the method is silent on
  // breakdown).  The first shift is u_f max_i a_ii / 4, then x4 per retry.  The
  // shift trades the perturbation of the low-precision factor (which breaks
  // it down when lambda_min(A) is below about u_f ||A||) against the distance
  // of M = L L^T from A; on the n = 65536, kappa ~ 1e4 FP8 system the refinement
  // needs 21 steps at this shift, 33 at a quarter of it and 59 at 16x it.  The
  // FP8 factor starts shifted: unshifted it breaks down on all but
  // near-identity matrices, and a failed factorisation costs a whole one.
  const double s_first = 0.25 * u_f * dmax;
  auto next_shift = [&](double sh) { return sh == 0.0 ? s_first : 4.0 * sh; };
  if (o.prec == JMG_PREC_FP8 && shift == 0.0) shift = s_first;

  bool converged = false;
  for (int attempt = 0;; ++attempt) {
    if (!o.reuse_factor || attempt > 0) {
      for (;;) {  // factor, shifting the diagonal while the low-precision factor breaks down
        JMG_CUDA(cudaMemsetAsync(c.ints, 0, sizeof(int) * 4, s));
        if (c.ev[4]) JMG_CUDA(cudaEventRecord(c.ev[4], s));
        JMG_TRY(launch_lower_to_f32(n, A, lda, c.W, p.ldw, shift, s));
        JMG_TRY(factor_mixed(n, c.W, p.ldw, o, p, work, &c.ints[0], &c.ints[1], s));
        if (c.ev[5]) JMG_CUDA(cudaEventRecord(c.ev[5], s));
        int hs[2] = {0, 0};
        JMG_TRY(sync_read(hs, c.ints, sizeof(hs), s));
        if (c.ev[5]) {
          float ms = 0.f;
          JMG_CUDA(cudaEventElapsedTime(&ms, c.ev[4], c.ev[5]));
          S.t_factor_gpu_ms += ms;
        }
        S.factor_tries++;
        if (hs[1]) return S.status = JMG_ERR_TIMEOUT;
        if (hs[0] == 0) break;
        if (!o.shift_retry || S.factor_tries >= 6) {
          JMG_CUDA(cudaMemcpyAsync(info, &c.ints[0], sizeof(int), cudaMemcpyDeviceToDevice, s));
          S.info = hs[0];
          return S.status = JMG_ERR_NOT_SPD;
        }
        shift = next_shift(shift);
      }
      JMG_CUDA(cudaMemcpyAsync(&c.dsc[1], &shift, sizeof(double), cudaMemcpyHostToDevice, s));
      JMG_CUDA(cudaStreamSynchronize(s));
    } else {
      JMG_CUDA(cudaMemsetAsync(&c.ints[2], 0, sizeof(int) * 2, s));
    }
    S.shift = shift;
    const double t1 = now_ms();
    S.t_factor_ms += t1 - t0;

    // initial solve X = M^{-1} B
    JMG_CUDA(cudaMemsetAsync(c.X, 0, sizeof(double) * (size_t)n * nrhs, s));
    JMG_CUDA(cudaMemsetAsync(c.colmax, 0, sizeof(double) * 3 * nrhs, s));
    {
      dim3 grid(std::min(cdiv(n, 256), 64), nrhs);
      k_copy_colmax<<<grid, 256, 0, s>>>(n, B, ldb, c.R, c.colmax);
      JMG_TRY(launched());
    }
    JMG_TRY(precond_update(n, nrhs, c.W, p.ldw, at<float>(work, p.off_SV), c.R, c.colmax, c.D,
                           p.ldd, c.X, c.sync, &c.ints[2], s, c.ev[2], c.ev[3]));
    c.solve_pending = c.ev[3] != nullptr;
    const double t2 = now_ms();
    S.t_solve_ms += t2 - t1;

    JMG_TRY(pro.wait());  // the residual needs ||A||_inf and the slices of A
    // refinement: classic IR, switching to PCG when IR is slow or diverges
    bool use_pcg = (o.refine == JMG_REFINE_PCG);
    double prev = INFINITY;
    int stall = 0;
    bool breakdown = false;
    for (;;) {
      JMG_TRY(true_residual(c));
      hist(c, c.eh[0]);
      S.bwd_err = c.eh[0];
      if (c.eh[0] <= o.tol) {
        converged = true;
        break;
      }
      if (S.iters >= o.maxit || std::isnan(c.eh[0])) break;
      if (!use_pcg) {
        const bool slow = S.iters >= 1 && c.eh[0] > 0.25 * prev;
        if (o.refine == JMG_REFINE_AUTO && slow) {
          use_pcg = true;
        } else if (o.refine == JMG_REFINE_IR) {
          stall = (c.eh[0] > 0.5 * prev) ? stall + 1 : 0;
          if (stall >= 3) break;
        }
      }
      prev = c.eh[0];
      if (!use_pcg) {
        JMG_TRY(precond_update(n, nrhs, c.W, p.ldw, at<float>(work, p.off_SV), c.R, c.colmax,
                               c.D, p.ldd, c.X, c.sync, &c.ints[2], s, c.ev[2], c.ev[3]));
        c.solve_pending = c.ev[3] != nullptr;
        S.iters++;
        continue;
      }
      S.refine_used = JMG_REFINE_PCG;
      JMG_TRY(pcg(c, &breakdown));
      if (breakdown) break;
    }
    S.t_refine_ms += now_ms() - t2;
    if (converged) break;
    // not converged: refactor with a (larger) diagonal shift
    if (!o.shift_retry || attempt >= 3 || S.iters >= o.maxit) break;
    shift = next_shift(shift);
  }
  {
    int hs3[3] = {0, 0, 0};
    JMG_TRY(sync_read(hs3, c.ints, sizeof(hs3), s));
    if (hs3[1] != 0 || hs3[2] != 0) return S.status = JMG_ERR_TIMEOUT;
  }
  JMG_CUDA(cudaMemsetAsync(info, 0, sizeof(int), s));
  JMG_TRY(launch_copy2d(n, nrhs, c.X, n, B, ldb, s));
  JMG_TRY(sync_read(&S.anorm, &c.dsc[0], sizeof(double), s));
  S.status = converged ? JMG_OK : JMG_ERR_NOT_CONVERGED;
  return S.status;
}

static int check_common(int n, int lda, int dtype) {
  if (n < 0) return -1;
  if (lda < std::max(1, n)) return -3;
  if (dtype != JMG_F64 && dtype != JMG_F32) return -4;
  return JMG_OK;
}

template <typename T>
__global__ void k_logdet(int n, const T* __restrict__ L, int lda, double* __restrict__ out) {
  // one CTA, fixed-order reduction (in FP64 for either storage type)
  __shared__ double part[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += log((double)L[(size_t)i * lda + i]);
  part[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = 2.0 * part[0];
}

// ---------------------------------------------------------------- host-buffer posv
// jmg_posv_host stages its operands at the front of `work`: the device copy of
// A (leading dimension n), then that of B (leading dimension n), then the
// device info word, then jmg_posv's own workspace.
struct HostStage {
  size_t off_B = 0, off_info = 0, off_posv = 0;
};

static HostStage host_stage(int n, int nrhs, size_t es) {
  HostStage h;
  h.off_B = round_up(es * (size_t)n * (size_t)n, 256);
  h.off_info = h.off_B + round_up(es * (size_t)n * (size_t)std::max(nrhs, 1), 256);
  h.off_posv = h.off_info + 256;
  return h;
}

// One rows x cols column-major block between host and device in one copy: a
// linear copy when the block is contiguous on both sides, else a 2-D copy.
// The whole block moves, so a symmetric A travels with its upper triangle: a
// copy that skips it needs one copy row per column, and on GB300 each row
// costs about 1 us of copy-engine time, more than the bytes it saves below
// n ~ 50000.  Adds the bytes to *bytes.
static int copy_block(void* dst, int ldd, const void* src, int lds, int rows, int cols, size_t es,
                      cudaMemcpyKind kind, long long* bytes, cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return JMG_OK;
  const size_t row_bytes = es * (size_t)rows;
  if (cols == 1 || (lds == rows && ldd == rows))
    JMG_CUDA(cudaMemcpyAsync(dst, src, row_bytes * (size_t)cols, kind, s));
  else
    JMG_CUDA(cudaMemcpy2DAsync(dst, es * (size_t)ldd, src, es * (size_t)lds, row_bytes,
                               (size_t)cols, kind, s));
  *bytes += (long long)(row_bytes * (size_t)cols);
  return JMG_OK;
}

}  // namespace jmg

using namespace jmg;

extern "C" {

void jmg_default_options(jmg_options* o) {
  if (!o) return;
  o->nb = 128;
  o->NB = 1024;
  o->prec = JMG_PREC_NATIVE;
  o->words = 1;
  o->tol = 1e-13;
  o->maxit = 300;
  o->refine = JMG_REFINE_AUTO;
  o->shift_retry = 1;
  o->timing = 0;
  o->reuse_factor = 0;
  o->resid = 0;
}

size_t jmg_workspace_size(int op, int n, int nrhs, int dtype, const jmg_options* opt) {
  jmg_options o;
  opts_or_default(opt, &o);
  if (op == JMG_OP_POSV_HOST) {
    if (n <= 0 || (dtype != JMG_F64 && dtype != JMG_F32)) return 0;
    const size_t es = dtype == JMG_F32 ? sizeof(float) : sizeof(double);
    return host_stage(n, nrhs, es).off_posv + jmg_workspace_size(JMG_OP_POSV, n, nrhs, dtype, &o);
  }
  if (op == JMG_OP_POSV && o.prec == JMG_PREC_FP32)
    return small_path_fits(n, nrhs) ? small_workspace(n, nrhs) : 0;
  if (op == JMG_OP_POSV && o.prec != JMG_PREC_NATIVE && n > 0)
    return plan_posv_mixed(n, nrhs, o).total;
  if (op == JMG_OP_POSV || op == JMG_OP_POTRS) return plain_solve_bytes(n, nrhs);
  return 0;
}

const char* jmg_status_string(int st) {
  switch (st) {
    case JMG_OK: return "ok";
    case JMG_ERR_CUDA: return "CUDA error";
    case JMG_ERR_WORKSPACE: return "workspace too small";
    case JMG_ERR_NOT_SPD: return "matrix is not positive definite";
    case JMG_ERR_NOT_CONVERGED: return "refinement did not reach the tolerance";
    case JMG_ERR_TIMEOUT: return "device-side wait timed out";
    case JMG_ERR_UNSUPPORTED: return "unsupported option combination";
    case JMG_ERR_ALIGN: return "alignment requirement not met";
    default: return st < 0 ? "illegal argument" : "unknown status";
  }
}

int jmg_potrf(int n, void* A, int lda, int dtype, int* info, const jmg_options* opt, void* work,
              size_t lwork, void* stream) {
  (void)work;
  (void)lwork;
  JMG_TRY(check_common(n, lda, dtype));
  if (!info) return -5;
  if (n > 0 && !A) return -2;
  jmg_options o;
  opts_or_default(opt, &o);
  if (o.nb != 64 && o.nb != 128) return -6;
  if (o.prec != JMG_PREC_NATIVE) return JMG_ERR_UNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  JMG_CUDA(cudaMemsetAsync(info, 0, sizeof(int), s));
  if (dtype == JMG_F32) return potrf_plain<float>(n, (float*)A, lda, o.nb, info, s);
  return potrf_plain<double>(n, (double*)A, lda, o.nb, info, s);
}

int jmg_potrs(int n, int nrhs, const void* L, int lda, void* B, int ldb, int dtype, void* work,
              size_t lwork, void* stream) {
  if (n < 0) return -1;
  if (nrhs < 0) return -2;
  if (lda < std::max(1, n)) return -4;
  if (ldb < std::max(1, n)) return -6;
  if (dtype != JMG_F64 && dtype != JMG_F32) return -7;
  if (n == 0 || nrhs == 0) return JMG_OK;
  if (!L) return -3;
  if (!B) return -5;
  if (!work || lwork < plain_solve_bytes(n, nrhs)) return JMG_ERR_WORKSPACE;
  if (reinterpret_cast<uintptr_t>(work) & 15) return JMG_ERR_ALIGN;
  if (dtype == JMG_F32)
    return solve_llt<float>(n, nrhs, (const float*)L, lda, (float*)B, ldb, (int*)work, nullptr,
                            (cudaStream_t)stream);
  return solve_llt<double>(n, nrhs, (const double*)L, lda, (double*)B, ldb, (int*)work, nullptr,
                           (cudaStream_t)stream);
}

int jmg_posv(int n, int nrhs, void* A, int lda, void* B, int ldb, int dtype, int* info,
             const jmg_options* opt, jmg_stats* stats, void* work, size_t lwork, void* stream) {
  if (n < 0) return -1;
  if (nrhs < 0) return -2;
  if (lda < std::max(1, n)) return -4;
  if (ldb < std::max(1, n)) return -6;
  if (dtype != JMG_F64 && dtype != JMG_F32) return -7;
  if (!info) return -8;
  jmg_options o;
  opts_or_default(opt, &o);
  if (o.nb != 64 && o.nb != 128) return -9;
  cudaStream_t s = (cudaStream_t)stream;
  if (stats) *stats = jmg_stats{};
  if (n == 0) {
    JMG_CUDA(cudaMemsetAsync(info, 0, sizeof(int), s));
    return JMG_OK;
  }
  if (!A) return -3;
  if (nrhs > 0 && !B) return -5;
  if (o.prec == JMG_PREC_NATIVE) {
    if (nrhs > 0 && (!work || lwork < plain_solve_bytes(n, nrhs))) return JMG_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(work) & 15) return JMG_ERR_ALIGN;
    JMG_CUDA(cudaMemsetAsync(info, 0, sizeof(int), s));
    if (dtype == JMG_F32) {
      JMG_TRY(potrf_plain<float>(n, (float*)A, lda, o.nb, info, s));
      if (nrhs > 0)
        JMG_TRY(solve_llt<float>(n, nrhs, (const float*)A, lda, (float*)B, ldb, (int*)work, info,
                                 s));
      return JMG_OK;
    }
    JMG_TRY(potrf_plain<double>(n, (double*)A, lda, o.nb, info, s));
    if (nrhs > 0)
      JMG_TRY(solve_llt<double>(n, nrhs, (const double*)A, lda, (double*)B, ldb, (int*)work, info,
                                s));
    return JMG_OK;
  }
  if (dtype == JMG_F32) return JMG_ERR_UNSUPPORTED;  // mixed modes refine FP64 data
  if (o.prec == JMG_PREC_FP32) {
    if (!small_path_fits(n, nrhs)) return JMG_ERR_UNSUPPORTED;
    if (nrhs == 0) {
      JMG_CUDA(cudaMemsetAsync(info, 0, sizeof(int), s));
      return JMG_OK;
    }
    if (!work || lwork < small_workspace(n, nrhs)) return JMG_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(work) & 255) return JMG_ERR_ALIGN;
    return small_posv(n, nrhs, (const double*)A, lda, (double*)B, ldb, info, o, stats, work, s);
  }
  if (o.prec != JMG_PREC_BF16 && o.prec != JMG_PREC_FP16 && o.prec != JMG_PREC_FP8)
    return JMG_ERR_UNSUPPORTED;
  if (o.prec == JMG_PREC_FP8 && o.nb != 128) return -9;
  if (nrhs == 0) {
    JMG_CUDA(cudaMemsetAsync(info, 0, sizeof(int), s));
    return JMG_OK;
  }
  size_t need = plan_posv_mixed(n, nrhs, o).total;
  if (!work || lwork < need) return JMG_ERR_WORKSPACE;
  if (reinterpret_cast<uintptr_t>(work) & 255) return JMG_ERR_ALIGN;
  return posv_mixed(n, nrhs, (const double*)A, lda, (double*)B, ldb, info, o, stats, work, s);
}

int jmg_posv_host(int n, int nrhs, const void* A, int lda, const void* B, int ldb, void* X,
                  int ldx, int dtype, int* info, const jmg_options* opt, jmg_stats* stats,
                  void* work, size_t lwork, void* stream) {
  if (n < 0) return -1;
  if (nrhs < 0) return -2;
  if (lda < std::max(1, n)) return -4;
  if (ldb < std::max(1, n)) return -6;
  if (ldx < std::max(1, n)) return -8;
  if (dtype != JMG_F64 && dtype != JMG_F32) return -9;
  if (!info) return -10;
  jmg_options o;
  opts_or_default(opt, &o);
  if (o.nb != 64 && o.nb != 128) return -11;
  if (o.prec == JMG_PREC_FP8 && o.nb != 128) return -11;
  if (stats) *stats = jmg_stats{};
  *info = 0;
  if (n == 0) return JMG_OK;
  if (!A) return -3;
  if (nrhs > 0 && !B) return -5;
  if (nrhs > 0 && !X) return -7;
  if (o.prec != JMG_PREC_NATIVE && dtype == JMG_F32) return JMG_ERR_UNSUPPORTED;
  if (o.prec != JMG_PREC_NATIVE && o.prec != JMG_PREC_BF16 && o.prec != JMG_PREC_FP16 &&
      o.prec != JMG_PREC_FP8 && o.prec != JMG_PREC_FP32)
    return JMG_ERR_UNSUPPORTED;
  if (o.prec == JMG_PREC_FP32 && !small_path_fits(n, nrhs)) return JMG_ERR_UNSUPPORTED;
  const size_t es = dtype == JMG_F32 ? sizeof(float) : sizeof(double);
  const HostStage h = host_stage(n, nrhs, es);
  const size_t need = jmg_workspace_size(JMG_OP_POSV_HOST, n, nrhs, dtype, &o);
  if (!work || lwork < need) return JMG_ERR_WORKSPACE;
  if (reinterpret_cast<uintptr_t>(work) & 255) return JMG_ERR_ALIGN;
  char* w = static_cast<char*>(work);
  char* Ad = w;
  char* Bd = w + h.off_B;
  int* info_d = reinterpret_cast<int*>(w + h.off_info);
  cudaStream_t s = (cudaStream_t)stream;
  long long h2d = 0, d2h = 0;
  // From the first queued copy on, every path synchronises before it returns:
  // the copies read and write the caller's host buffers.
  int st = copy_block(Ad, n, A, lda, n, n, es, cudaMemcpyHostToDevice, &h2d, s);
  if (st == JMG_OK) st = copy_block(Bd, n, B, ldb, n, nrhs, es, cudaMemcpyHostToDevice, &h2d, s);
  if (st == JMG_OK)
    st = jmg_posv(n, nrhs, Ad, n, Bd, n, dtype, info_d, &o, stats, w + h.off_posv,
                  lwork - h.off_posv, stream);
  int hinfo = 0;
  if (st == JMG_OK || st == JMG_ERR_NOT_CONVERGED || st == JMG_ERR_NOT_SPD) {
    if (copy_block(X, ldx, Bd, n, n, nrhs, es, cudaMemcpyDeviceToHost, &d2h, s) != JMG_OK)
      st = JMG_ERR_CUDA;
    if (cudaMemcpyAsync(&hinfo, info_d, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
      st = JMG_ERR_CUDA;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess && st == JMG_OK) st = JMG_ERR_CUDA;
  if (st < 0) st = JMG_ERR_CUDA;  // the arguments were checked above: cannot happen
  *info = hinfo;
  if (st == JMG_OK && hinfo > 0) st = JMG_ERR_NOT_SPD;
  if (st == JMG_OK && hinfo < 0) st = JMG_ERR_TIMEOUT;
  if (stats) {
    stats->status = st;
    stats->info = hinfo;
    stats->h2d_bytes = h2d;
    stats->d2h_bytes = d2h;
  }
  return st;
}

int jmg_posv_batched(int n, int nrhs, int batch, void* A, int lda, long long strideA, void* B,
                     int ldb, long long strideB, int dtype, int* info, void* stream) {
  if (n < 0) return -1;
  if (nrhs < 0) return -2;
  if (batch < 0) return -3;
  if (lda < std::max(1, n)) return -5;
  if (strideA < (long long)lda * n) return -6;
  if (ldb < std::max(1, n)) return -8;
  if (strideB < (long long)ldb * nrhs) return -9;
  if (dtype != JMG_F64 && dtype != JMG_F32) return -10;
  if (!info) return -11;
  if (n > 128) return JMG_ERR_UNSUPPORTED;
  if (batch > 0 && n > 0 && !A) return -4;
  if (batch > 0 && n > 0 && nrhs > 0 && !B) return -7;
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == JMG_F32)
    return posv_small_batched<float>(n, nrhs, batch, (float*)A, lda, strideA, (float*)B, ldb,
                                     strideB, info, s);
  return posv_small_batched<double>(n, nrhs, batch, (double*)A, lda, strideA, (double*)B, ldb,
                                    strideB, info, s);
}

int jmg_logdet(int n, const void* L, int lda, int dtype, double* out, void* stream) {
  if (n < 0) return -1;
  if (lda < std::max(1, n)) return -3;
  if (dtype != JMG_F64 && dtype != JMG_F32) return -4;
  if (!out) return -5;
  if (n > 0 && !L) return -2;
  if (dtype == JMG_F32)
    k_logdet<float><<<1, 256, 0, (cudaStream_t)stream>>>(n, (const float*)L, lda, out);
  else
    k_logdet<double><<<1, 256, 0, (cudaStream_t)stream>>>(n, (const double*)L, lda, out);
  return launched();
}

// ---------------------------------------------------------------- dev entry points
int jmg_sym_grad(int n, int nrhs, const double* Bbar, int ldb, const double* X, int ldx,
                 double* Abar, int ldab, void* stream) {
  if (n < 0) return -1;
  if (nrhs < 0) return -2;
  if (ldb < std::max(1, n)) return -4;
  if (ldx < std::max(1, n)) return -6;
  if (ldab < std::max(1, n)) return -8;
  if (n > 0 && !Abar) return -7;
  if (n > 0 && nrhs > 0 && (!Bbar || !X)) return !Bbar ? -3 : -5;
  return launch_sym_grad(n, nrhs, Bbar, ldb, X, ldx, Abar, ldab, (cudaStream_t)stream);
}

int jmg_dev_syrk_tc(int m, int ncols, int kext, const void* PA, const void* PB, int ldp,
                    int prec, float* C, int ldc, int* err, void* stream) {
  if (m < 0) return -1;
  if (ncols < 0 || ncols > m) return -2;
  if (ldc < std::max(1, m)) return -9;
  if (!err) return -10;
  return launch_syrk_tc(m, ncols, kext, PA, PB, ldp, prec, C, ldc, err, (cudaStream_t)stream);
}

int jmg_dev_syrk_fp8(int m, int ncols, int kext, const void* Q, int ldq, const signed char* e,
                     float* C, int ldc, int* err, void* stream) {
  if (m < 0) return -1;
  if (ncols < 0 || ncols > m) return -2;
  if (ldc < std::max(1, m)) return -8;
  if (!err) return -9;
  return launch_syrk_fp8(m, ncols, kext, Q, ldq, e, 0, C, ldc, err, (cudaStream_t)stream);
}

int jmg_dev_syrk_fp8_chunks(int m, int ncols, int kext, const void* Q, int ldq,
                            const signed char* e, int lde, float* C, int ldc, int* err,
                            void* stream) {
  if (m < 0) return -1;
  if (ncols < 0 || ncols > m) return -2;
  if (lde < 0) return -7;
  if (ldc < std::max(1, m)) return -9;
  if (!err) return -10;
  return launch_syrk_fp8(m, ncols, kext, Q, ldq, e, lde, C, ldc, err, (cudaStream_t)stream);
}

size_t jmg_dev_residual_workspace(int n, int nrhs) {
  if (n <= 0 || nrhs <= 0) return 0;
  return sizeof(double) * (size_t)n * nrhs * residual_splits(n, nrhs);
}

int jmg_dev_residual(int n, int nrhs, const double* A, int lda, const double* X, int ldx,
                     const double* B, int ldb, double* R, int ldr, double* colmax, void* work,
                     size_t lwork, void* stream) {
  if (n < 0) return -1;
  if (nrhs < 0) return -2;
  if (lwork < jmg_dev_residual_workspace(n, nrhs)) return JMG_ERR_WORKSPACE;
  return launch_residual(n, nrhs, A, lda, X, ldx, B, ldb, R, ldr, colmax, (double*)work,
                         residual_splits(n, nrhs), (cudaStream_t)stream);
}

struct SplitLayout {
  size_t rowmax, sa, sx, part, total;
};
static SplitLayout split_layout(int n, int nrhs) {
  SplitLayout L;
  size_t off = 0;
  auto take = [&](size_t b) {
    size_t at = off;
    off = round_up(off + b, 256);
    return at;
  };
  L.rowmax = take(sizeof(double) * (size_t)std::max(n, 1));
  L.sa = take(oz_a_bytes(n));
  L.sx = take(oz_x_bytes(n, nrhs));
  L.part = take(sizeof(double) * (size_t)n * nrhs * oz_splits_used(n, nrhs));
  L.total = off;
  return L;
}

size_t jmg_dev_residual_split_workspace(int n, int nrhs) {
  if (n <= 0 || nrhs <= 0) return 0;
  return split_layout(n, nrhs).total;
}

int jmg_dev_residual_split(int n, int nrhs, const double* A, int lda, const double* X, int ldx,
                           const double* B, int ldb, double* R, int ldr, double* colmax,
                           int* err, void* work, size_t lwork, void* stream) {
  if (n < 0) return -1;
  if (nrhs < 0) return -2;
  if (n == 0 || nrhs == 0) return JMG_OK;
  if (!err) return -12;
  const SplitLayout L = split_layout(n, nrhs);
  if (!work || lwork < L.total) return JMG_ERR_WORKSPACE;
  if (reinterpret_cast<uintptr_t>(work) & 255) return JMG_ERR_ALIGN;
  cudaStream_t s = (cudaStream_t)stream;
  char* w = static_cast<char*>(work);
  double* rowmax = reinterpret_cast<double*>(w + L.rowmax);
  double* part = reinterpret_cast<double*>(w + L.part);
  JMG_TRY(oz_prepare_a(n, A, lda, rowmax, w + L.sa, s));
  JMG_TRY(oz_product(n, nrhs, w + L.sa, rowmax, X, ldx, w + L.sx, part, err, s));
  JMG_CUDA(cudaMemsetAsync(colmax, 0, sizeof(double) * 3 * nrhs, s));
  return launch_resid_reduce(n, nrhs, oz_splits_used(n, nrhs), part, X, ldx, B, ldb, R, ldr,
                             colmax, s);
}

int jmg_dev_norm_inf(int n, const double* A, int lda, double* out, void* work, size_t lwork,
                     void* stream) {
  if (n < 0) return -1;
  if (lwork < sizeof(double) * (size_t)std::max(n, 1)) return JMG_ERR_WORKSPACE;
  return launch_norm_inf(n, A, lda, (double*)work, out, (cudaStream_t)stream);
}

long long jmg_dev_launch_count(void) { return g_launches; }

// layout of jmg_dev_sv_potrs's workspace: W (ldw x n), D (ldw x nrhs), images, sync
struct SvDevLayout {
  size_t W, D, SV, sync, total;
  int ldw;
};
static SvDevLayout sv_dev_layout(int n, int nrhs) {
  SvDevLayout L;
  size_t off = 0;
  auto take = [&](size_t b) {
    size_t at = off;
    off = round_up(off + b, 256);
    return at;
  };
  L.ldw = (int)round_up((size_t)std::max(n, 1), 32);
  L.W = take(sizeof(float) * (size_t)L.ldw * std::max(n, 1));
  L.D = take(sizeof(float) * (size_t)L.ldw * std::max(nrhs, 1));
  L.SV = take(sv_image_bytes(n));
  L.sync = take(sizeof(int) * sv_sync_ints(n, nrhs));
  L.total = off;
  return L;
}

size_t jmg_dev_sv_workspace(int n, int nrhs) {
  if (n <= 0 || nrhs <= 0) return 0;
  return sv_dev_layout(n, nrhs).total;
}

int jmg_dev_sv_potrs(int n, int nrhs, const float* L, int lda, float* B, int ldb, void* work,
                     size_t lwork, void* stream) {
  if (n < 0) return -1;
  if (nrhs < 0) return -2;
  if (lda < std::max(1, n)) return -4;
  if (ldb < std::max(1, n)) return -6;
  if (n == 0 || nrhs == 0) return JMG_OK;
  if (!L) return -3;
  if (!B) return -5;
  const SvDevLayout Lo = sv_dev_layout(n, nrhs);
  if (!work || lwork < Lo.total) return JMG_ERR_WORKSPACE;
  if (reinterpret_cast<uintptr_t>(work) & 255) return JMG_ERR_ALIGN;
  cudaStream_t s = (cudaStream_t)stream;
  char* w = static_cast<char*>(work);
  float* W = reinterpret_cast<float*>(w + Lo.W);
  float* D = reinterpret_cast<float*>(w + Lo.D);
  float* SV = reinterpret_cast<float*>(w + Lo.SV);
  int* sync = reinterpret_cast<int*>(w + Lo.sync);
  JMG_CUDA(cudaMemcpy2DAsync(W, sizeof(float) * Lo.ldw, L, sizeof(float) * lda, sizeof(float) * n,
                             n, cudaMemcpyDeviceToDevice, s));
  JMG_CUDA(cudaMemcpy2DAsync(D, sizeof(float) * Lo.ldw, B, sizeof(float) * ldb, sizeof(float) * n,
                             nrhs, cudaMemcpyDeviceToDevice, s));
  JMG_TRY(sv_prepare(n, W, Lo.ldw, SV, s));
  JMG_TRY(sv_solve_llt(n, nrhs, W, Lo.ldw, SV, D, Lo.ldw, sync, nullptr, s));
  JMG_CUDA(cudaMemcpy2DAsync(B, sizeof(float) * ldb, D, sizeof(float) * Lo.ldw, sizeof(float) * n,
                             nrhs, cudaMemcpyDeviceToDevice, s));
  return JMG_OK;
}

unsigned long long jmg_dev_set_wait_limit_ns(unsigned long long ns) {
  const unsigned long long old = g_wait_ns;
  if (ns > 0) g_wait_ns = ns;
  return old;
}

int jmg_dev_trsv_leaderless(int n, int nrhs, const void* L, int lda, void* B, int ldb, int dtype,
                            int* sync, int* info, void* stream) {
  if (n <= 0) return -1;
  if (nrhs <= 0) return -2;
  if (lda < n) return -4;
  if (ldb < n) return -6;
  if (!L) return -3;
  if (!B) return -5;
  if (!sync) return -8;
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == JMG_F32)
    return launch_trsv_persist<float>(n, nrhs, (const float*)L, lda, (float*)B, ldb, 0, sync, info,
                                      s, 1);
  if (dtype == JMG_F64)
    return launch_trsv_persist<double>(n, nrhs, (const double*)L, lda, (double*)B, ldb, 0, sync,
                                       info, s, 1);
  return -7;
}

int jmg_dev_syrk_tc_idle_producer(int m, int ncols, int kext, const void* PA, const void* PB,
                                  int ldp, int prec, float* C, int ldc, int* err, void* stream) {
  if (m <= 0) return -1;
  if (ncols <= 0 || ncols > m) return -2;
  if (ldc < m) return -9;
  if (!err) return -10;
  return launch_syrk_tc(m, ncols, kext, PA, PB, ldp, prec, C, ldc, err, (cudaStream_t)stream, 0,
                        1);
}

int jmg_dev_quant_fp8(int m, int kb, const float* L21, int ldw, void* Q, int ldq, signed char* e,
                      void* stream) {
  if (m < 0) return -1;
  if (kb <= 0) return -2;
  if (ldw < std::max(1, m)) return -4;
  if (ldq < kb) return -6;
  if (m > 0 && (!L21 || !Q || !e)) return !L21 ? -3 : (!Q ? -5 : -7);
  return launch_quant_fp8(m, kb, L21, ldw, Q, ldq, e, (cudaStream_t)stream);
}

}  // extern "C"
