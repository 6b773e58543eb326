// Whole Nystrom-PCG solve in one cooperative launch, for small QPs.
//
// For small problems (A of a few MB, L2-resident) a PCG iteration issued as
// separate kernels is bound by launch latency, not by A.  Here all CTAs stay
// resident and run the CG loop themselves.  CTA b owns a band of rows (for
// the m-vectors) and a band of columns (for t = D .* A^T p); every CTA keeps a
// full copy of the search direction p in shared memory and updates it
// redundantly, so p never round-trips through global memory.  Grid-wide sums
// are reduced by every CTA from per-CTA partials in the same fixed order, so
// all CTAs take identical (deterministic) decisions.  Four bounded grid
// barriers per iteration:
//
//   1. p = z + beta p (smem, all rows);  t = D .* (A^T p) over own columns
//      (warps split the rows, lanes the columns, a tree over the warps)
//   -- barrier (t complete)
//   2. w = A t + delta p over own rows; partial p^T w            -> alpha
//   3. x += alpha p; r -= alpha w over own rows; partials U^T r, r^T r
//   -- barrier (inside the U^T r reduction)                       -> stop?
//   4. z = r + U (wts .* s) over own rows; partial r^T z          -> beta
//
// Arithmetic and stopping rule are those of the multi-kernel path (pcg.cu):
// same CG recurrences, same eta test at the top of an iteration, FP64.
#include "common.cuh"
#include "internal.h"

namespace nys {

namespace {

constexpr int kPT = 256;
constexpr int kPW = kPT / 32;
constexpr int kMaxM = 4096;      // p lives in shared memory
constexpr int kMaxEll = 1024;
constexpr int kMaxSmemVec = 24576;   // m + n entries of p and t in shared memory

struct PState {
  double *x, *r, *z, *w, *t;
  double* part_ut;    // gridDim.x * (ell + 1): partials of U^T r and ||r||^2
  double* part_sum;   // gridDim.x: partials of single dot products
};

// Sum over the grid: block reduce, publish, barrier, then every CTA reduces
// the partials in block order.  Returns false on barrier timeout.
__device__ bool all_sum(double& v, double* part, unsigned* bar, int* err, double* sh) {
  double a[1] = {v};
  block_sum<kPT, 1>(a, sh);
  if (threadIdx.x == 0) __stcg(part + blockIdx.x, a[0]);
  __threadfence();
  if (!grid_barrier(bar, err)) return false;
  double acc[1] = {0.0};
  for (int b = threadIdx.x; b < (int)gridDim.x; b += kPT) acc[0] += __ldcg(part + b);
  block_sum<kPT, 1>(acc, sh);
  v = acc[0];
  return true;
}

// s = U^T r (into the CTA's shared s) and ||r||^2 over the grid; each CTA
// contributes its own row band [i0, i1), which it has written itself.
__device__ bool all_ut(int ell, const double* __restrict__ U, int ld, const double* r, int i0, int i1,
                       double* part2, double* s, double& rr, unsigned* bar, int* err, double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double* mine = part2 + (size_t)blockIdx.x * (ell + 1);
  __syncthreads();   // r of the band was written by other threads of this CTA
  for (int c = wid; c < ell; c += kPW) {
    const double* u = U + (size_t)c * ld;
    double acc = 0.0;
    for (int i = i0 + lane; i < i1; i += 32) acc = fma(__ldg(u + i), __ldcg(r + i), acc);
    acc = warp_sum(acc);
    if (lane == 0) __stcg(mine + c, acc);
  }
  double v[1] = {0.0};
  for (int i = i0 + threadIdx.x; i < i1; i += kPT) {
    const double ri = __ldcg(r + i);
    v[0] = fma(ri, ri, v[0]);
  }
  block_sum<kPT, 1>(v, sh);
  if (threadIdx.x == 0) __stcg(mine + ell, v[0]);
  __threadfence();
  if (!grid_barrier(bar, err)) return false;
  for (int e = threadIdx.x; e <= ell; e += kPT) {
    double acc = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) acc += __ldcg(part2 + (size_t)b * (ell + 1) + e);
    if (e < ell) s[e] = acc;
    else sh[kPW * 4] = acc;
  }
  __syncthreads();
  rr = sh[kPW * 4];
  __syncthreads();
  return true;
}

__global__ void __launch_bounds__(kPT) k_pcg_persistent(int m, int n, const double* __restrict__ A, long long lda,
                                                        const double* __restrict__ D, double delta, int ell,
                                                        const double* __restrict__ U, int ld,
                                                        const double* __restrict__ lam, const double* __restrict__ xi,
                                                        PState S, double eta2, int max_iter, int forced,
                                                        unsigned* bar, int* err, int* iters_out, double* sd) {
  extern __shared__ double ps[];            // p (m entries), then t (n entries)
  double* ts = ps + m;
  __shared__ double sh[kPW * 4 + 2];
  __shared__ double ws[kMaxEll];            // (lam_ell + delta) / (lam + delta) - 1
  __shared__ double ss[kMaxEll];            // s = U^T r
  __shared__ double red[kPW * 64];          // per-warp partials of A^T p
  const int tid = threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5;
  const int rb = (m + gridDim.x - 1) / gridDim.x;
  const int i0 = min(m, (int)blockIdx.x * rb), i1 = min(m, i0 + rb);
  const int cb = (n + gridDim.x - 1) / gridDim.x;
  const int j0 = min(n, (int)blockIdx.x * cb), j1 = min(n, j0 + cb);

  // setup (own rows): r = xi, x = 0
  for (int i = i0 + tid; i < i1; i += kPT) { __stcg(S.r + i, xi[i]); __stcg(S.x + i, 0.0); }
  const double lam_ell = lam[ell - 1];
  for (int c = tid; c < ell; c += kPT) ws[c] = (lam_ell + delta) / (lam[c] + delta) - 1.0;
  double rr = 0.0;
  if (!all_ut(ell, U, ld, S.r, i0, i1, S.part_ut, ss, rr, bar, err, sh)) return;
  const double bnorm2 = rr;
  const int limit = forced >= 0 ? forced : max_iter;
  int it = 0;
  bool done = (bnorm2 == 0.0) || (limit <= 0);
  // z = r + U (ws .* s) (own rows), rz
  double rz = 0.0;
  {
    double v = 0.0;
    for (int i = i0 + tid; i < i1; i += kPT) {
      double acc = 0.0;
      for (int c = 0; c < ell; ++c) acc = fma(__ldg(U + (size_t)c * ld + i), ws[c] * ss[c], acc);
      const double ri = __ldcg(S.r + i), zi = ri + acc;
      __stcg(S.z + i, zi);
      v = fma(ri, zi, v);
    }
    if (!all_sum(v, S.part_sum, bar, err, sh)) return;
    rz = v;
  }
  double beta = 0.0;              // first direction: p = z
  while (!done) {
    // 1. p = z + beta p in shared memory (every CTA, all rows); t over own columns
    for (int i = tid; i < m; i += kPT) ps[i] = fma(beta, it == 0 ? 0.0 : ps[i], __ldcg(S.z + i));
    __syncthreads();
    // warps over rows (two interleaved accumulators each), lanes over 64
    // columns, then a fixed tree over the warps: no thread walks a whole
    // column, so the FP64 latency chains stay short
    for (int c0 = j0; c0 < j1; c0 += 32) {
      // one 32-column block at a time (warp-uniform loop: no predicated-off
      // FP64 instructions for columns past the band)
      const int j = c0 + lane;
      double a = 0.0, b = 0.0;
      if (j < j1) {
        int i = wid;
        for (; i + kPW < m; i += 2 * kPW) {
          a = fma(__ldg(A + (long long)i * lda + j), ps[i], a);
          b = fma(__ldg(A + (long long)(i + kPW) * lda + j), ps[i + kPW], b);
        }
        if (i < m) a = fma(__ldg(A + (long long)i * lda + j), ps[i], a);
      }
      red[wid * 32 + lane] = a + b;
      __syncthreads();
      if (tid < 32 && c0 + tid < j1) {
        double w8[kPW];
#pragma unroll
        for (int w = 0; w < kPW; ++w) w8[w] = red[w * 32 + tid];
#pragma unroll
        for (int st = 1; st < kPW; st <<= 1)
#pragma unroll
          for (int w = 0; w + st < kPW; w += 2 * st) w8[w] += w8[w + st];
        __stcg(S.t + c0 + tid, D[c0 + tid] * w8[0]);
      }
      __syncthreads();
    }
    __threadfence();
    if (!grid_barrier(bar, err)) return;
    // 2. w = A t + delta p over own rows (warp per row); p^T w.  t is staged
    // in shared memory first (one coalesced pass instead of a chain of L2
    // round trips per row).
    for (int j = tid; j < n; j += kPT) ts[j] = __ldcg(S.t + j);
    __syncthreads();
    double v = 0.0;
    for (int i = i0 + wid; i < i1; i += kPW) {
      const double* a = A + (long long)i * lda;
      double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
      int j = lane;
      for (; j + 96 < n; j += 128) {
        a0 = fma(__ldg(a + j), ts[j], a0);
        a1 = fma(__ldg(a + j + 32), ts[j + 32], a1);
        a2 = fma(__ldg(a + j + 64), ts[j + 64], a2);
        a3 = fma(__ldg(a + j + 96), ts[j + 96], a3);
      }
      for (; j < n; j += 32) a0 = fma(__ldg(a + j), ts[j], a0);
      const double acc = warp_sum((a0 + a1) + (a2 + a3));
      if (lane == 0) {
        const double wi = fma(delta, ps[i], acc);
        __stcg(S.w + i, wi);
        v = fma(ps[i], wi, v);
      }
    }
    if (!all_sum(v, S.part_sum, bar, err, sh)) return;
    const double pw = v;
    if (!(pw > 0.0) || !isfinite(pw)) { set_error(err, kErrNumeric); break; }
    const double alpha = rz / pw;
    // 3. x += alpha p; r -= alpha w (own rows); then s = U^T r, ||r||^2
    for (int i = i0 + tid; i < i1; i += kPT) {
      __stcg(S.x + i, fma(alpha, ps[i], __ldcg(S.x + i)));
      __stcg(S.r + i, fma(-alpha, __ldcg(S.w + i), __ldcg(S.r + i)));
    }
    if (!all_ut(ell, U, ld, S.r, i0, i1, S.part_ut, ss, rr, bar, err, sh)) return;
    ++it;
    if (!isfinite(rr)) { set_error(err, kErrNumeric); break; }
    if (forced >= 0 ? (it >= forced) : (rr <= eta2 * bnorm2 || it >= max_iter)) break;
    // 4. z = r + U (ws .* s) (own rows); r^T z
    v = 0.0;
    for (int i = i0 + tid; i < i1; i += kPT) {
      double acc = 0.0;
      for (int c = 0; c < ell; ++c) acc = fma(__ldg(U + (size_t)c * ld + i), ws[c] * ss[c], acc);
      const double ri = __ldcg(S.r + i), zi = ri + acc;
      __stcg(S.z + i, zi);
      v = fma(ri, zi, v);
    }
    if (!all_sum(v, S.part_sum, bar, err, sh)) return;
    const double rz_new = v;
    if (!(rz_new > 0.0) || !isfinite(rz_new)) {
      if (rz_new != 0.0) set_error(err, kErrNumeric);
      break;
    }
    beta = rz_new / rz;
    rz = rz_new;
  }
  if (blockIdx.x == 0 && tid == 0) {
    *iters_out = it;
    sd[SD_RR] = rr;
    sd[SD_BNORM2] = bnorm2;
    sd[SD_ETA2] = eta2;
  }
}

}  // namespace

bool pcg_persistent_fits(int m, int n, int ell) {
  // p and t in shared memory next to the 16 KB of weights and U^T r
  return m <= kMaxM && m + n <= kMaxSmemVec && (long long)m * n <= (1ll << 23) && ell <= kMaxEll;
}

cudaError_t pcg_persistent_f64(cudaStream_t st, int m, int n, const double* A, long long lda, const double* D,
                               double delta, int ell, const double* U, int ld, const double* lam, const double* xi,
                               double eta, int max_iter, int forced, PcgWork w, double* part, size_t part_cap,
                               unsigned* bar, double* sd, int* si, int num_sms) {
  const size_t dsm = sizeof(double) * ((size_t)m + (size_t)n);
  // set to the kernel's maximum (p and t of the largest fitting system), never
  // lowered: handles on other host threads may be launching it concurrently
  cudaError_t e = cudaFuncSetAttribute(k_pcg_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(sizeof(double) * kMaxSmemVec));
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg_persistent, kPT, dsm);
  if (e != cudaSuccess) return e;
  // about 16K multiply-adds of the operator per CTA (the FP64 rate of an SM
  // bounds each phase), at least 2 CTAs, at most one CTA per SM
  long long g = ((long long)m * n + 16383) / 16384;
  if (g < 2) g = 2;
  if (g > num_sms) g = num_sms;
  if (g > (long long)per_sm * num_sms) g = (long long)per_sm * num_sms;
  const int grid = (int)g;
  if ((size_t)grid * (ell + 2) > part_cap) return cudaErrorInvalidValue;
  e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  PState S{w.x, w.r, w.z, w.w, w.t, part, part + (size_t)grid * (ell + 1)};
  int mm = m, nn = n, ee = ell, ldd = ld, mi = max_iter, fo = forced;
  long long la = lda;
  double dl = delta, e2 = eta * eta;
  int* err = si + SI_ERR;
  int* it = si + SI_ITERS;
  void* args[] = {&mm, &nn, &A, &la, &D, &dl, &ee, &U, &ldd, &lam, &xi, &S, &e2, &mi, &fo, &bar, &err, &it, &sd};
  count_launches(1);
  return cudaLaunchCooperativeKernel((const void*)k_pcg_persistent, dim3(grid), dim3(kPT), args, dsm, st);
}

}  // namespace nys
