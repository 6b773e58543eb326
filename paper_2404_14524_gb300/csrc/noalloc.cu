// The normal-equations operator for callers that cannot allocate device
// memory.
//
// Some callers of this library run where allocation is not an option: code
// inside a CUDA-graph capture or a memory-pool-managed region where a
// cudaMalloc would break the capture or the pool's accounting, embedded or
// real-time hosts that forbid allocation after start-up, and plugins that only
// receive pointers from their host application.  They cannot create a solver
// handle (nys_create allocates the workspace), so this entry point takes no
// handle: its scratch (the intermediate vector t = D .* (A^T v) and the
// split-reduction partial sums) lives in one fixed, file-scope device array
// that every GPU loading the library holds until the process exits.
//
// The array's host-side name is only a stand-in for the device symbol, so the
// first call on each device (with that device current) looks up the real
// device address with cudaGetSymbolAddress and caches it; make that first call
// before any stream capture.  All calls share the array: calls that can
// overlap on the GPU (different streams, or different host threads without
// ordering) race on it and must be serialised by the caller.  No part of the
// scratch needs to start at zero: every call writes all the scratch it reads.
#include <mutex>

#include "../../include/nys.h"
#include "internal.h"

namespace {

constexpr size_t kNoallocScratchDoubles = size_t(1) << 20;   // 8 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_noalloc_scratch[kNoallocScratchDoubles];

std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kMaxDevices] = {nullptr};

}  // namespace

extern "C" int nys_normal_matvec_noalloc(int m, int n, const double* A, long long lda, const double* D,
                                         double delta, const double* v, double* out, void* cuda_stream) {
  if (m <= 0 || n <= 0 || lda < n || !A || !D || !v || !out || out == v) return NYS_ERR_ARG;
  if ((size_t)n > kNoallocScratchDoubles) return NYS_ERR_NOMEM;   // t alone exceeds the fixed scratch
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return NYS_ERR_CUDA;
  double* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return NYS_ERR_CUDA;
      }
      g_noalloc_ptr[dev] = static_cast<double*>(p);
    }
    base = g_noalloc_ptr[dev];
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  // t takes the first n doubles (rounded up to keep 256-byte alignment); the
  // split-reduction partials use the rest (fewer splits when it is short).
  const size_t t_len = (static_cast<size_t>(n) + 31) / 32 * 32;
  double* t = base;
  double* split = base + t_len;
  const size_t split_cap = t_len < kNoallocScratchDoubles ? kNoallocScratchDoubles - t_len : 0;
  if (nys::gemv_t_f64(st, m, n, A, lda, v, D, t, split, split_cap) != cudaSuccess) return NYS_ERR_CUDA;
  if (nys::gemv_n_f64(st, m, n, A, lda, t, delta, v, out) != cudaSuccess) return NYS_ERR_CUDA;
  return NYS_OK;
}
