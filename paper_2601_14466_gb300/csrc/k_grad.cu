// k_grad.cu -- adjoint of the SPD solve X = A^{-1} B with respect to A:
//
//     Abar = -(Bbar X^T + X Bbar^T) / 2          (full symmetric, FP64)
//
// where Bbar = A^{-1} Xbar comes from the solve with the stored factor.  The
// paper exposes potrs as a primitive that composes with the framework's
// transformations ("Summary"); reverse-mode differentiation is one of them, and
// this is its matrix-calculus form for a symmetric A read from one triangle.
//
// One CTA per 64 x 64 lower tile (ti >= tj); the rank-2 nrhs products run on
// the FP64 CUDA cores (4 x 4 register tile per thread).  The tile is written
// to (ti, tj) directly and to the mirror (tj, ti) through a shared-memory
// transpose so that both stores coalesce down columns; on diagonal tiles the
// upper half is the mirror of the lower half, so Abar is exactly symmetric.
#include "kernels.h"

namespace jmg {

namespace grad {
constexpr int TB = 64, KC = 16;
}

__global__ void __launch_bounds__(256) k_sym_grad(int n, int nrhs, const double* __restrict__ Bb,
                                                  int ldb, const double* __restrict__ X, int ldx,
                                                  double* __restrict__ G, int ldg) {
  using namespace grad;
  int ti, tj;
  tri_index(blockIdx.x, ti, tj);
  const int i0 = ti * TB, j0 = tj * TB;
  // the four K slices and, after the K loop, the output tile share one buffer
  // (4 * KC * (TB + 1) == TB * (TB + 1) doubles, 33 KB)
  __shared__ double sbuf[TB * (TB + 1)];
  double(*Bi)[TB + 1] = reinterpret_cast<double(*)[TB + 1]>(sbuf);
  double(*Xi)[TB + 1] = Bi + KC;
  double(*Bj)[TB + 1] = Bi + 2 * KC;
  double(*Xj)[TB + 1] = Bi + 3 * KC;
  double(*T)[TB + 1] = reinterpret_cast<double(*)[TB + 1]>(sbuf);
  static_assert(4 * KC == TB, "slices and tile share the buffer");
  const int t = threadIdx.x, tx = t % 16, ty = t / 16;  // rows tx + 16q, cols ty + 16p
  double acc[4][4];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int p = 0; p < 4; ++p) acc[q][p] = 0.0;
  for (int k0 = 0; k0 < nrhs; k0 += KC) {
    // 4 x (64 x 16) values: 4 per thread per slice
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int idx = t + 256 * q;
      const int r = idx % TB, k = idx / TB;
      const int gk = k0 + k;
      const bool kin = gk < nrhs;
      const int gi = i0 + r, gj = j0 + r;
      Bi[k][r] = (kin && gi < n) ? Bb[(size_t)gk * ldb + gi] : 0.0;
      Xi[k][r] = (kin && gi < n) ? X[(size_t)gk * ldx + gi] : 0.0;
      Bj[k][r] = (kin && gj < n) ? Bb[(size_t)gk * ldb + gj] : 0.0;
      Xj[k][r] = (kin && gj < n) ? X[(size_t)gk * ldx + gj] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < KC; ++k) {
      double bi[4], xi[4], bj[4], xj[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        bi[q] = Bi[k][tx + 16 * q];
        xi[q] = Xi[k][tx + 16 * q];
        bj[q] = Bj[k][ty + 16 * q];
        xj[q] = Xj[k][ty + 16 * q];
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int p = 0; p < 4; ++p) acc[q][p] = fma(bi[q], xj[p], fma(xi[q], bj[p], acc[q][p]));
    }
    __syncthreads();
  }
  // (the K loop ended with a barrier, so the slices are free)
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const double v = -0.5 * acc[q][p];
      const int r = tx + 16 * q, c = ty + 16 * p;
      T[r][c] = v;
      // diagonal tiles: lower half here, the upper half is its mirror (below), so
      // the result is symmetric bit for bit
      if (i0 + r < n && j0 + c < n && (ti != tj || r >= c)) G[(size_t)(j0 + c) * ldg + i0 + r] = v;
    }
  __syncthreads();
  // mirror: G[j0 + c', i0 + r'] = T[r'][c'], written down columns i0 + r'
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int idx = t + 256 * q;
    const int c = idx % TB, r = idx / TB;  // row j0 + c of G, column i0 + r
    if (j0 + c < n && i0 + r < n && (ti != tj || r > c)) G[(size_t)(i0 + r) * ldg + j0 + c] = T[r][c];
  }
}

int launch_sym_grad(int n, int nrhs, const double* Bb, int ldb, const double* X, int ldx, double* G,
                    int ldg, cudaStream_t s) {
  if (n <= 0) return JMG_OK;
  if (nrhs <= 0) {
    JMG_CUDA(cudaMemset2DAsync(G, sizeof(double) * ldg, 0, sizeof(double) * n, n, s));
    return JMG_OK;
  }
  k_sym_grad<<<(unsigned)tri_tiles(cdiv(n, grad::TB)), 256, 0, s>>>(n, nrhs, Bb, ldb, X, ldx, G,
                                                                      ldg);
  return launched();
}

}  // namespace jmg
