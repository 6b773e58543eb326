// Shared device helpers: deterministic block/grid reductions, error flags,
// and a bounded grid barrier for cooperative launches.
//
// Every grid-wide reduction in this library is deterministic: each block
// reduces its values in a fixed shuffle/shared-memory tree, writes one partial
// per block, and the last block to finish (found through an atomic ticket)
// sums the partials in a fixed order.  No spin-waits are involved.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <math.h>

namespace nys {

constexpr int kNT = 256;           // threads per block for vector kernels
constexpr int kWarps = kNT / 32;

// Device error word values (mirrors nys_status; 0 = ok).
constexpr int kErrNumeric = -3;
constexpr int kErrCoreBreakdown = -4;
constexpr int kErrTimeout = -5;

__device__ __forceinline__ void set_error(int* err, int code) {
  if (err) atomicCAS(err, 0, code);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Sum of K values over the block; the result is valid in every thread.
// `sh` must hold K * (NT/32) doubles.
template <int NT, int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = warp_sum(v[k]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) sh[k * (NT / 32) + wid] = v[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) s += sh[k * (NT / 32) + w];
    v[k] = s;
  }
  __syncthreads();
}

template <int NT>
__device__ __forceinline__ double block_min(double v, double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_min(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double s = sh[0];
#pragma unroll
  for (int w = 1; w < NT / 32; ++w) s = fmin(s, sh[w]);
  __syncthreads();
  return s;
}

// Grid-wide deterministic sum of K values.  Each block passes its own
// (not yet block-reduced) values.  Returns true in every thread of the last
// block, where `out` holds the grid totals; false elsewhere.
// partials: gridDim.x * K doubles; counter: zero on entry, left zero on exit.
template <int NT, int K>
__device__ bool grid_sum(double (&v)[K], double* partials, unsigned int* counter, double (&out)[K]) {
  __shared__ double sh[K * (NT / 32)];
  __shared__ bool last;
  block_sum<NT, K>(v, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) partials[(size_t)blockIdx.x * K + k] = v[k];
    __threadfence();
    unsigned t = atomicAdd(counter, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += NT) {
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] += __ldcg(partials + (size_t)b * K + k);
  }
  block_sum<NT, K>(acc, sh);
#pragma unroll
  for (int k = 0; k < K; ++k) out[k] = acc[k];
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

template <int NT>
__device__ bool grid_min(double v, double* partials, unsigned int* counter, double* out) {
  __shared__ double sh[NT / 32];
  __shared__ bool last;
  v = block_min<NT>(v, sh);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = v;
    __threadfence();
    unsigned t = atomicAdd(counter, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double acc = INFINITY;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += NT) acc = fmin(acc, __ldcg(partials + b));
  acc = block_min<NT>(acc, sh);
  *out = acc;
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

// Bounded grid barrier for cooperative launches (all blocks co-resident).
// `bar` is one word that must be zero when the launch starts; each barrier
// leaves its low 31 bits at zero again.  Block 0 adds 2^31 - (blocks - 1),
// every other block adds 1, so the top bit flips exactly when the last block
// arrives, whatever the arrival order; a waiting block watches for that flip.
// One atomic per block and one polled word: no reset step, no second round
// trip.  A block that waits longer than the spin limit records kErrTimeout in
// *err and returns false; so does every block once *err is non-zero.
__device__ __forceinline__ bool grid_barrier(unsigned int* bar, int* err) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int inc = blockIdx.x == 0 ? 0x80000000u - (gridDim.x - 1u) : 1u;
    volatile int* verr = err;
    __threadfence();                       // this block's writes before its arrival
    const unsigned int old = atomicAdd(bar, inc);
    unsigned long long spins = 0;
    while (true) {
      unsigned int cur;
      asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(cur) : "l"(bar) : "memory");
      if ((cur ^ old) & 0x80000000u) break;
      if ((++spins & 31u) == 0) {
        if (*verr != 0) break;
        if (spins > (1ull << 24)) { set_error(err, kErrTimeout); break; }
        __nanosleep(32);
      }
    }
    __threadfence();
    ok = (*verr == 0);
  }
  __syncthreads();
  return ok != 0;
}

}  // namespace nys
