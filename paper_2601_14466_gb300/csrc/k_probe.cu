// k_probe.cu -- arithmetic-throughput probes (FP64 FMA, FP64 mma.sync, FP32 FMA).
// They give the FP64 and FP32 peaks against which the solver's kernels are
// reported; the host times one launch with CUDA events.
#include "kernels.h"

namespace jmg {

// 8 independent FMA chains per thread; 2 flops per FMA.
template <typename T>
__global__ void __launch_bounds__(256) k_probe_fma(int iters, T* __restrict__ sink) {
  T a[8];
  const T m = T(0.999999), c = T(1e-7);
#pragma unroll
  for (int q = 0; q < 8; ++q) a[q] = T(threadIdx.x + q) * T(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int q = 0; q < 8; ++q) a[q] = fma(a[q], m, c);
    }
  }
  T s = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) s += a[q];
  if (s == T(-12345.0)) sink[blockIdx.x] = s;  // never true: keeps the chains live
}

// FP64 tensor-core path of mma.sync: m8n8k4, 4 independent accumulators per warp.
__global__ void __launch_bounds__(256) k_probe_dmma(int iters, double* __restrict__ sink) {
  double a = 1.0 + threadIdx.x * 1e-6, b = 1.0 - threadIdx.x * 1e-6;
  double d[4][2];
#pragma unroll
  for (int q = 0; q < 4; ++q) d[q][0] = d[q][1] = 0.0;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        asm volatile(
            "mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
            : "+d"(d[q][0]), "+d"(d[q][1])
            : "d"(a), "d"(b));
      }
    }
  }
  double s = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) s += d[q][0] + d[q][1];
  if (s == -12345.0) sink[blockIdx.x] = s;
}

}  // namespace jmg

extern "C" int jmg_dev_probe(int kind, int blocks, int iters, double* sink, double* flops,
                             void* stream) {
  using namespace jmg;
  cudaStream_t s = (cudaStream_t)stream;
  if (blocks <= 0 || iters <= 0) return -2;
  double f = 0;
  if (kind == 0) {
    k_probe_fma<double><<<blocks, 256, 0, s>>>(iters, sink);
    f = 2.0 * 8 * 16 * (double)iters * 256.0 * blocks;
  } else if (kind == 1) {
    k_probe_dmma<<<blocks, 256, 0, s>>>(iters, sink);
    f = 2.0 * 8 * 8 * 4 * (double)(4 * 8) * iters * (256 / 32) * blocks;
  } else if (kind == 2) {
    k_probe_fma<float><<<blocks, 256, 0, s>>>(iters, reinterpret_cast<float*>(sink));
    f = 2.0 * 8 * 16 * (double)iters * 256.0 * blocks;
  } else {
    return -1;
  }
  if (flops) *flops = f;
  return launched();
}
