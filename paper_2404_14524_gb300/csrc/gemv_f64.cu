// FP64 streaming kernels for the normal-equations operator of Eq. normal-eq:
//   (N + delta I) v = A (D .* (A^T v)) + delta v,   N = A D A^T, A row-major.
//
// A^T v is a column reduction of a row-major matrix: blocks own a strip of
// 512 columns (two per thread, 16-byte loads, fully coalesced rows) and a
// band of rows; per-band partial sums go to a split buffer that a second
// kernel reduces in a fixed order (deterministic, no atomics).
// A t is a row reduction: one warp per row, 16-byte loads, xor-shuffle sum.
// When there are too few rows to fill the GPU (short, wide A: m of order 100,
// n of order 10^5, as in the dual-SVM constraint matrix) each row is also cut
// into column chunks whose partial sums a second kernel adds in a fixed
// order (deterministic).
//
// On GB300 the FP64 form of these kernels is bound by DFMA throughput (one
// fused multiply-add per element of A), not by HBM bandwidth.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace nys {

namespace {

constexpr int kColsPerThread = 2;
constexpr int kTileCols = kNT * kColsPerThread;   // 512 columns per block
constexpr int kTargetBlocks = 152 * 4;

template <bool kVec>
__global__ void __launch_bounds__(kNT) k_atv_partial(int m, int n, const double* __restrict__ A,
                                                     long long lda, const double* __restrict__ v,
                                                     int rows_per_split, const double* __restrict__ D,
                                                     double* __restrict__ out, int direct,
                                                     const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int j = (blockIdx.x * kNT + threadIdx.x) * kColsPerThread;
  const int i0 = blockIdx.y * rows_per_split;
  const int i1 = min(m, i0 + rows_per_split);
  double a0 = 0.0, a1 = 0.0;
  if (j < n) {
    if (kVec && j + 1 < n) {
      const double* col = A + j;
      int i = i0;
      for (; i + 4 <= i1; i += 4) {
        const double2 x0 = __ldg(reinterpret_cast<const double2*>(col + (long long)(i + 0) * lda));
        const double2 x1 = __ldg(reinterpret_cast<const double2*>(col + (long long)(i + 1) * lda));
        const double2 x2 = __ldg(reinterpret_cast<const double2*>(col + (long long)(i + 2) * lda));
        const double2 x3 = __ldg(reinterpret_cast<const double2*>(col + (long long)(i + 3) * lda));
        const double v0 = __ldg(v + i), v1 = __ldg(v + i + 1), v2 = __ldg(v + i + 2), v3 = __ldg(v + i + 3);
        a0 = fma(x0.x, v0, a0); a1 = fma(x0.y, v0, a1);
        a0 = fma(x1.x, v1, a0); a1 = fma(x1.y, v1, a1);
        a0 = fma(x2.x, v2, a0); a1 = fma(x2.y, v2, a1);
        a0 = fma(x3.x, v3, a0); a1 = fma(x3.y, v3, a1);
      }
      for (; i < i1; ++i) {
        const double2 x0 = __ldg(reinterpret_cast<const double2*>(col + (long long)i * lda));
        const double vi = __ldg(v + i);
        a0 = fma(x0.x, vi, a0); a1 = fma(x0.y, vi, a1);
      }
    } else {
      const bool two = (j + 1 < n);
      for (int i = i0; i < i1; ++i) {
        const double vi = __ldg(v + i);
        const double* row = A + (long long)i * lda;
        a0 = fma(__ldg(row + j), vi, a0);
        if (two) a1 = fma(__ldg(row + j + 1), vi, a1);
      }
    }
    if (direct) {
      const double s0 = D ? D[j] : 1.0;
      out[j] = s0 * a0;
      if (j + 1 < n) out[j + 1] = (D ? D[j + 1] : 1.0) * a1;
    } else {
      double* dst = out + (size_t)blockIdx.y * n;
      dst[j] = a0;
      if (j + 1 < n) dst[j + 1] = a1;
    }
  }
}

__global__ void __launch_bounds__(kNT) k_atv_reduce(int n, int splits, const double* __restrict__ part,
                                                    const double* __restrict__ D, double* __restrict__ t,
                                                    const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int j = blockIdx.x * kNT + threadIdx.x;
  if (j >= n) return;
  double s = 0.0;
  for (int k = 0; k < splits; ++k) s += part[(size_t)k * n + j];
  t[j] = (D ? D[j] : 1.0) * s;
}

// Row dot products over columns [c0, c1) (c0 even).  part == nullptr: the
// whole row, out[row] = sum + beta v[row]; otherwise the chunk's partial sum
// goes to part[blockIdx.y * m + row].
template <bool kVec>
__global__ void __launch_bounds__(kNT) k_av(int m, int n, const double* __restrict__ A, long long lda,
                                            const double* __restrict__ t, double beta,
                                            const double* __restrict__ v, double* __restrict__ out,
                                            const int* __restrict__ skip, const double* __restrict__ beta_dev,
                                            int chunk, double* __restrict__ part) {
  if (skip && *skip) return;
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * kWarps + (threadIdx.x >> 5);
  if (row >= m) return;
  const int c0 = blockIdx.y * chunk;
  const int c1 = min(n, c0 + chunk);
  const double* a = A + (long long)row * lda;
  double acc0 = 0.0, acc1 = 0.0;
  if (kVec) {
#pragma unroll 4
    for (int j = c0 + 2 * lane; j + 1 < c1; j += 64) {
      const double2 x = __ldg(reinterpret_cast<const double2*>(a + j));
      const double2 y = __ldg(reinterpret_cast<const double2*>(t + j));
      acc0 = fma(x.x, y.x, acc0);
      acc1 = fma(x.y, y.y, acc1);
    }
    if ((c1 & 1) && c1 == n && lane == 0) acc0 = fma(__ldg(a + n - 1), __ldg(t + n - 1), acc0);
  } else {
    for (int j = c0 + lane; j < c1; j += 32) acc0 = fma(__ldg(a + j), __ldg(t + j), acc0);
  }
  double s = warp_sum(acc0 + acc1);
  if (lane != 0) return;
  if (part) {
    part[(size_t)blockIdx.y * m + row] = s;
    return;
  }
  if (beta_dev) beta = *beta_dev;
  out[row] = (beta != 0.0) ? fma(beta, v[row], s) : s;
}

// out[row] = sum over the chunks, in chunk order, + beta v[row]
__global__ void __launch_bounds__(kNT) k_av_reduce(int m, int chunks, const double* __restrict__ part, double beta,
                                                   const double* __restrict__ v, double* __restrict__ out,
                                                   const int* __restrict__ skip, const double* __restrict__ beta_dev) {
  if (skip && *skip) return;
  const int row = blockIdx.x * kNT + threadIdx.x;
  if (row >= m) return;
  if (beta_dev) beta = *beta_dev;
  double s = 0.0;
  for (int k = 0; k < chunks; ++k) s += part[(size_t)k * m + row];
  out[row] = (beta != 0.0) ? fma(beta, v[row], s) : s;
}

__global__ void k_scaling(int n, const double* __restrict__ x, const double* __restrict__ z,
                          const double* __restrict__ q, double rho, double* __restrict__ D) {
  const int j = blockIdx.x * kNT + threadIdx.x;
  if (j < n) D[j] = 1.0 / (q[j] + z[j] / x[j] + rho);
}

int pick_splits(int m, int n) {
  const int bx = (n + kTileCols - 1) / kTileCols;
  int s = (kTargetBlocks + bx - 1) / bx;
  const int max_s = m / 16 > 1 ? m / 16 : 1;
  if (s > max_s) s = max_s;
  if (s < 1) s = 1;
  return s;
}

}  // namespace

size_t gemv_t_split_elems(int m, int n) {
  const int s = pick_splits(m, n);
  return s > 1 ? (size_t)s * n : 0;
}

cudaError_t gemv_t_f64(cudaStream_t st, int m, int n, const double* A, long long lda,
                       const double* v, const double* D, double* t, double* split_buf,
                       size_t split_cap, const int* skip) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  int s = pick_splits(m, n);
  while (s > 1 && (size_t)s * n > split_cap) s = (s + 1) / 2;
  const int rows = (m + s - 1) / s;
  s = (m + rows - 1) / rows;
  const bool vec = (lda % 2 == 0) && ((reinterpret_cast<uintptr_t>(A) & 15u) == 0);
  dim3 grid((n + kTileCols - 1) / kTileCols, s);
  if (s == 1) {
    if (vec) { count_launches(1); k_atv_partial<true><<<grid, kNT, 0, st>>>(m, n, A, lda, v, rows, D, t, 1, skip); }
    else { count_launches(1); k_atv_partial<false><<<grid, kNT, 0, st>>>(m, n, A, lda, v, rows, D, t, 1, skip); }
    return cudaGetLastError();
  }
  if (vec) { count_launches(1); k_atv_partial<true><<<grid, kNT, 0, st>>>(m, n, A, lda, v, rows, nullptr, split_buf, 0, skip); }
  else { count_launches(1); k_atv_partial<false><<<grid, kNT, 0, st>>>(m, n, A, lda, v, rows, nullptr, split_buf, 0, skip); }
  count_launches(1);
  k_atv_reduce<<<(n + kNT - 1) / kNT, kNT, 0, st>>>(n, s, split_buf, D, t, skip);
  return cudaGetLastError();
}

int av_chunks(int m, int n, size_t split_cap, int* chunk) {
  // enough (row block, column chunk) pairs for four blocks per SM, chunks of
  // at least 1024 columns, a multiple of 64 wide (16-byte loads stay aligned)
  const int blocks = (m + kWarps - 1) / kWarps;
  long long S = (kTargetBlocks + blocks - 1) / blocks;
  S = std::min<long long>(S, n / 1024);
  if (m > 0) S = std::min<long long>(S, (long long)(split_cap / (size_t)m));
  if (S < 2) {
    *chunk = n;
    return 1;
  }
  const long long w = ((n + S - 1) / S + 63) / 64 * 64;
  *chunk = (int)w;
  return (int)((n + w - 1) / w);
}

cudaError_t gemv_n_f64(cudaStream_t st, int m, int n, const double* A, long long lda,
                       const double* t, double beta, const double* v, double* out,
                       const int* skip, const double* beta_dev, double* split_buf, size_t split_cap) {
  if (m <= 0) return cudaSuccess;
  const bool vec = (lda % 2 == 0) && ((reinterpret_cast<uintptr_t>(A) & 15u) == 0) &&
                   ((reinterpret_cast<uintptr_t>(t) & 15u) == 0);
  const int blocks = (m + kWarps - 1) / kWarps;
  int chunk = n;
  const int S = split_buf ? av_chunks(m, n, split_cap, &chunk) : 1;
  double* part = S > 1 ? split_buf : nullptr;
  dim3 grid(blocks, S);
  count_launches(1);
  if (vec) k_av<true><<<grid, kNT, 0, st>>>(m, n, A, lda, t, beta, v, out, skip, beta_dev, chunk, part);
  else k_av<false><<<grid, kNT, 0, st>>>(m, n, A, lda, t, beta, v, out, skip, beta_dev, chunk, part);
  if (S > 1) {
    count_launches(1);
    k_av_reduce<<<(m + kNT - 1) / kNT, kNT, 0, st>>>(m, S, split_buf, beta, v, out, skip, beta_dev);
  }
  return cudaGetLastError();
}

cudaError_t scaling_f64(cudaStream_t st, int n, const double* x, const double* z, const double* q,
                        double rho, double* D) {
  if (n <= 0) return cudaSuccess;
  count_launches(1);
  k_scaling<<<(n + kNT - 1) / kNT, kNT, 0, st>>>(n, x, z, q, rho, D);
  return cudaGetLastError();
}

}  // namespace nys
