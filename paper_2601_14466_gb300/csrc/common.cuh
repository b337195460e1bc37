// common.cuh -- shared helpers of the SPD solver's CUDA sources (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/jmg.h"

#define JMG_DEV __device__ __forceinline__

namespace jmg {

// ---------------------------------------------------------------- host side

extern long long g_launches;  // launches queued by this library (jmg_dev_launch_count)

// Time limit of every device-side wait (flag and mbarrier spins), passed to the
// kernels at launch.  2 s by default: far above any legal wait.  Process-wide;
// jmg_dev_set_wait_limit_ns changes it (tests shorten it to make a wait run out).
extern unsigned long long g_wait_ns;

// Raise a kernel's dynamic shared-memory limit to `bytes` on the current
// device, once per (kernel, device) pair; thread-safe.
int ensure_smem_raw(const void* func, int bytes);
template <typename F>
inline int ensure_smem(F* func, int bytes) {
  return ensure_smem_raw(reinterpret_cast<const void*>(func), bytes);
}

inline int cuda_status(cudaError_t e) { return e == cudaSuccess ? JMG_OK : JMG_ERR_CUDA; }

// After a launch: count it, and turn a launch error into JMG_ERR_CUDA.
inline int launched() {
  ++g_launches;
  return cuda_status(cudaGetLastError());
}

#define JMG_TRY(expr)              \
  do {                             \
    int _st = (expr);              \
    if (_st != JMG_OK) return _st; \
  } while (0)

#define JMG_CUDA(expr) JMG_TRY(::jmg::cuda_status(expr))

inline size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
inline int cdiv(int a, int b) { return (a + b - 1) / b; }

// Number of lower-triangle tiles (ti >= tj) of a t x t tile grid.
inline long long tri_tiles(int t) { return (long long)t * (t + 1) / 2; }

// ---------------------------------------------------------------- device side

// Lower-triangle tile index -> (ti, tj), ti >= tj, row-by-row enumeration.
JMG_DEV void tri_index(int b, int& ti, int& tj) {
  // FP32 estimate (FP64 is slow on this GPU), corrected to the exact integer
  int t = (int)((sqrtf(8.0f * (float)b + 1.0f) - 1.0f) * 0.5f);
  while ((long long)t * (t + 1) / 2 > b) --t;
  while ((long long)(t + 1) * (t + 2) / 2 <= b) ++t;
  ti = t;
  tj = b - t * (t + 1) / 2;
}

JMG_DEV int cdiv_dev(int a, int b) { return (a + b - 1) / b; }

JMG_DEV uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Volatile read of a flag in shared memory.  (A volatile access through a
// generic pointer is ordered behind the thread's outstanding global loads and
// stores, so a flag check written that way waits for them.)
JMG_DEV int ld_shared_volatile(const int* p) {
  int v;
  asm volatile("ld.volatile.shared.b32 %0, [%1];" : "=r"(v) : "r"(smem_u32(p)) : "memory");
  return v;
}

JMG_DEV uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Atomic max of a non-negative double held as its bit pattern (the ordering of
// non-negative IEEE doubles matches the ordering of their bits as integers).
// NaN (any sign) is stored as the largest pattern so that it wins.
JMG_DEV void atomic_max_nonneg(double* addr, double v) {
  unsigned long long bits = isnan(v) ? 0x7FFFFFFFFFFFFFFFull : (unsigned long long)__double_as_longlong(fabs(v));
  atomicMax(reinterpret_cast<unsigned long long*>(addr), bits);
}

}  // namespace jmg
