// k_layout.cu -- in-place conversion of a row-major matrix to column-major
// order (paper: "Local memory-layout conversion": the framework's arrays are
// row-major, the solver wants column-major, and a second full-sized copy is
// what the conversion must avoid).
//
// The m x n matrix M sits row-major in a buffer of m n elements: M(i, j) at
// i n + j.  Its column-major form puts M(i, j) at j m + i, i.e. the buffer
// becomes the row-major n x m matrix M^T.  As in the rectangular permutation
// decomposition of Catanzaro, Keller and Garland (2014), the move is written
// as three permutations, each of which stays inside one column or one row of
// the m x n view, so each can be done in place with scratch for one column or
// row at a time.  With c = gcd(m, n) and b = n / c:
//
//   1. columns (only when c > 1): column j is rotated by floor(j / b) rows:
//        new(p, j) = old((p + floor(j / b)) mod m, j);
//   2. rows: in row p the entry of column j moves to column
//        q = (j m + i) mod n,  i = (p + floor(j / b)) mod m
//      (i is the original row of that entry); for every p this is a
//      bijection of the columns, because j m mod n runs over the multiples of c
//      as j mod b does, while the rotation above makes i mod c distinct for the
//      c runs of b columns;
//   3. columns: the entry for final position (r, q), whose linear index
//      L = r n + q equals j m + i for its original (i, j) = (L mod m, L / m),
//      sits in row (i - floor(j / b)) mod m of column q after steps 1 and 2:
//        new(r, q) = cur((i - floor(j / b)) mod m, q).
//
// Columns go in batches of CB adjacent columns, one batch per CTA at a time,
// through a scratch slab of m x CB elements in `work`; the number of batches
// in flight is what the scratch holds.  Rows go one per CTA through shared
// memory (or a scratch row when they are longer than shared memory holds).
#include <algorithm>

#include "kernels.h"

namespace jmg {
namespace lay {
constexpr int CB = 32;  // columns per batch
constexpr int TH = 256;
}  // namespace lay

// Steps 1 and 3: gather each column batch into the CTA's scratch slab, then
// copy it back.  step 1: source row (p + floor(j/b)) mod m; step 3: the row
// given by the final linear index.
template <typename T, int STEP>
__global__ void __launch_bounds__(lay::TH) k_col_perm(long long m, long long n, long long b,
                                                     T* __restrict__ A, T* __restrict__ scratch) {
  const long long nbatch = (n + lay::CB - 1) / lay::CB;
  T* S = scratch + (size_t)blockIdx.x * (size_t)m * lay::CB;
  const int t = threadIdx.x, lane = t % lay::CB, grp = t / lay::CB;
  constexpr int NGRP = lay::TH / lay::CB;
  for (long long bt = blockIdx.x; bt < nbatch; bt += gridDim.x) {
    const long long j = bt * lay::CB + lane;  // this thread's column
    const bool live = j < n;
    for (long long r = grp; r < m; r += NGRP) {
      long long src = 0;
      if (live) {
        if (STEP == 1) {
          src = (r + j / b) % m;
        } else {
          const long long L = r * n + j;
          const long long i = L % m, jj = L / m;
          src = ((i - jj / b) % m + m) % m;
        }
      }
      S[(size_t)r * lay::CB + lane] = live ? A[(size_t)src * n + j] : T(0);
    }
    __syncthreads();
    for (long long r = grp; r < m; r += NGRP)
      if (live) A[(size_t)r * n + j] = S[(size_t)r * lay::CB + lane];
    __syncthreads();  // the slab is reused by the next batch
  }
}

// Step 2: row p scattered into shared memory (or the CTA's scratch row), then
// written back in order.
template <typename T, bool SMEM>
__global__ void __launch_bounds__(lay::TH) k_row_perm(long long m, long long n, long long b,
                                                     T* __restrict__ A, T* __restrict__ scratch) {
  extern __shared__ __align__(16) unsigned char sm_lay[];
  T* S = SMEM ? reinterpret_cast<T*>(sm_lay) : scratch + (size_t)blockIdx.x * (size_t)n;
  for (long long p = blockIdx.x; p < m; p += gridDim.x) {
    T* row = A + (size_t)p * n;
    for (long long j = threadIdx.x; j < n; j += blockDim.x) {
      const long long i = (p + j / b) % m;
      const long long q = (j * m + i) % n;
      S[q] = row[j];
    }
    __syncthreads();
    for (long long q = threadIdx.x; q < n; q += blockDim.x) row[q] = S[q];
    __syncthreads();
  }
}

static long long gcd_ll(long long a, long long b) {
  while (b) {
    const long long t = a % b;
    a = b;
    b = t;
  }
  return a;
}

size_t layout_min_scratch(long long m, long long n, size_t esize) {
  // one column slab, and one scratch row if a row does not fit in shared memory
  return esize * (size_t)std::max<long long>(m * lay::CB, n);
}

template <typename T>
static int r2c_impl(long long m, long long n, T* A, void* work, size_t lwork, cudaStream_t s) {
  if (m <= 1 || n <= 1) return JMG_OK;  // a vector: both orders coincide
  const long long c = gcd_ll(m, n), b = n / c;
  int dev = 0, nsm = 152;
  JMG_CUDA(cudaGetDevice(&dev));
  JMG_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  T* scratch = static_cast<T*>(work);
  const long long nbatch = (n + lay::CB - 1) / lay::CB;
  const size_t slab = sizeof(T) * (size_t)m * lay::CB;
  const int col_grid = (int)std::max<long long>(
      1, std::min<long long>({nbatch, (long long)(lwork / slab), 4LL * nsm}));
  if (c > 1) {
    k_col_perm<T, 1><<<col_grid, lay::TH, 0, s>>>(m, n, b, A, scratch);
    JMG_TRY(launched());
  }
  const size_t row_bytes = sizeof(T) * (size_t)n;
  if (row_bytes <= 160 * 1024) {
    JMG_TRY(ensure_smem(k_row_perm<T, true>, (int)row_bytes));
    const int grid = (int)std::min<long long>(m, 4LL * nsm);
    k_row_perm<T, true><<<grid, lay::TH, row_bytes, s>>>(m, n, b, A, scratch);
  } else {
    const int grid = (int)std::max<long long>(
        1, std::min<long long>({m, (long long)(lwork / row_bytes), 4LL * nsm}));
    k_row_perm<T, false><<<grid, lay::TH, 0, s>>>(m, n, b, A, scratch);
  }
  JMG_TRY(launched());
  k_col_perm<T, 3><<<col_grid, lay::TH, 0, s>>>(m, n, b, A, scratch);
  return launched();
}

int layout_r2c(long long m, long long n, void* A, int dtype, void* work, size_t lwork,
               cudaStream_t s) {
  if (dtype == JMG_F32) return r2c_impl<float>(m, n, static_cast<float*>(A), work, lwork, s);
  return r2c_impl<double>(m, n, static_cast<double*>(A), work, lwork, s);
}

}  // namespace jmg

using namespace jmg;

extern "C" size_t jmg_layout_workspace(long long m, long long n, int dtype) {
  if (m <= 1 || n <= 1) return 0;
  const size_t es = dtype == JMG_F32 ? sizeof(float) : sizeof(double);
  return round_up(layout_min_scratch(m, n, es), 256);
}

extern "C" int jmg_rowmajor_to_colmajor(long long m, long long n, void* A, int dtype, void* work,
                                        size_t lwork, void* stream) {
  if (m < 0) return -1;
  if (n < 0) return -2;
  if (dtype != JMG_F64 && dtype != JMG_F32) return -4;
  if (m <= 1 || n <= 1) return JMG_OK;
  if (!A) return -3;
  if (!work || lwork < jmg_layout_workspace(m, n, dtype)) return JMG_ERR_WORKSPACE;
  return layout_r2c(m, n, A, dtype, work, lwork, (cudaStream_t)stream);
}

extern "C" int jmg_colmajor_to_rowmajor(long long m, long long n, void* A, int dtype, void* work,
                                        size_t lwork, void* stream) {
  // the column-major m x n matrix is the row-major n x m matrix M^T: its
  // row-to-column conversion is the inverse move
  if (m < 0) return -1;
  if (n < 0) return -2;
  if (dtype != JMG_F64 && dtype != JMG_F32) return -4;
  if (m <= 1 || n <= 1) return JMG_OK;
  if (!A) return -3;
  if (!work || lwork < jmg_layout_workspace(n, m, dtype)) return JMG_ERR_WORKSPACE;
  return layout_r2c(n, m, A, dtype, work, lwork, (cudaStream_t)stream);
}
