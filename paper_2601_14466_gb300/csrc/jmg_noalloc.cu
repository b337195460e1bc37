// jmg_noalloc.cu -- jmg_potrs_static: the FP64 solve with a Cholesky factor
// that needs no scratch from the caller and allocates nothing.
//
// jmg_potrs takes its scratch (the tickets, counters, flags and error
// word of the one-launch triangular solves) from a caller-provided `work` buffer.  Some
// callers cannot provide one: code that runs after device memory has been
// handed out once and for all (a fixed memory budget set at start-up, or a
// host framework that owns every device byte through its own pool), and plain
// C callers without a device allocator of their own.  For them this entry point
// keeps the scratch in a fixed array in device memory, declared at file scope,
// so a call allocates nothing (no cudaMalloc, no cudaFree, no allocating
// library routine).
#include <mutex>

#include "kernels.h"

namespace jmg {
namespace {

// Fixed scratch: 65536 ints (256 KiB), resident on every GPU that loads the
// library until the process exits.  Every call shares it and it keeps the last
// call's contents; the solve launcher clears the part it uses before each
// launch (word 0, the outcome, only before the forward solve, so that it
// carries a timeout of either direction to jmg_potrs_static_status).
constexpr int kStaticScratchInts = 65536;
static __device__ __align__(256) int g_solve_scratch[kStaticScratchInts];

// Host-side device address of g_solve_scratch, one per device, looked up on the
// first call made with that device current.  (In host code the symbol's name
// is only a stand-in and must not be passed to a kernel.)
constexpr int kMaxDevices = 64;
std::mutex g_mu;
int* g_scratch_dev[kMaxDevices] = {};

int scratch_for_current_device(int** out) {
  int dev = -1;
  JMG_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return JMG_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_solve_scratch);
    if (e != cudaSuccess || !p) return JMG_ERR_CUDA;
    g_scratch_dev[dev] = static_cast<int*>(p);
  }
  *out = g_scratch_dev[dev];
  return JMG_OK;
}

}  // namespace
}  // namespace jmg

extern "C" int jmg_potrs_static(int n, int nrhs, const void* L, int lda, void* B, int ldb,
                                int dtype, void* stream) {
  using namespace jmg;
  if (n < 0) return -1;
  if (nrhs < 0) return -2;
  if (lda < std::max(1, n)) return -4;
  if (ldb < std::max(1, n)) return -6;
  if (dtype != JMG_F64) return dtype == JMG_F32 ? JMG_ERR_UNSUPPORTED : -7;
  if (n == 0 || nrhs == 0) return JMG_OK;
  if (!L) return -3;
  if (!B) return -5;
  if (trsv_sync_ints(n, nrhs) > (size_t)kStaticScratchInts) return JMG_ERR_WORKSPACE;
  int* scratch = nullptr;
  JMG_TRY(scratch_for_current_device(&scratch));
  return solve_llt<double>(n, nrhs, static_cast<const double*>(L), lda, static_cast<double*>(B),
                           ldb, scratch, nullptr, static_cast<cudaStream_t>(stream));
}

// The solve writes its outcome into the first word of the fixed scratch (0, or
// JMG_ERR_TIMEOUT when a device-side wait ran out).  The word stays there until
// the next call on the same device clears it, so this reads the outcome of the
// last call queued on `stream`.
extern "C" int jmg_potrs_static_status(int* status, void* stream) {
  using namespace jmg;
  if (!status) return -1;
  int* scratch = nullptr;
  JMG_TRY(scratch_for_current_device(&scratch));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int word = 0;
  JMG_CUDA(cudaMemcpyAsync(&word, scratch, sizeof(int), cudaMemcpyDeviceToHost, s));
  JMG_CUDA(cudaStreamSynchronize(s));
  *status = word;
  return JMG_OK;
}
