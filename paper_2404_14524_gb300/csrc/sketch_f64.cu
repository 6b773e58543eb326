// Gaussian test matrices and the FP64 sketch Y = A (D .* (A^T Omega))
// (Algorithm 1, first two steps).
//
// The FP64 sketch is two SIMT DFMA GEMMs (GB300 has no FP64 tensor-core
// kind for tcgen05, and its DFMA rate is the bound): 64x64 output tiles (32x32
// when the sketch has at most 32 columns), 16-deep k-slices staged in shared
// memory, register blocking per thread, split-K with a fixed-order reduction
// when there are too few output tiles to fill the 152 SMs.
#include "common.cuh"
#include "internal.h"

namespace nys {

namespace {

// ---- SplitMix64 (Steele, Lea, Flood 2014) at an arbitrary stream position.
__device__ __forceinline__ unsigned long long splitmix_at(unsigned long long seed,
                                                          unsigned long long pos) {
  unsigned long long z = seed + (pos + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_gaussian(unsigned long long seed, int k, int m, int ell, int cols, double* __restrict__ Om,
                           int ld) {
  const long long idx = (long long)blockIdx.x * kNT + threadIdx.x;
  if (idx >= (long long)m * cols) return;
  const int i = (int)(idx % m);
  const int j = (int)(idx / m);
  const unsigned long long c = ((unsigned long long)k * ell + j) * (unsigned long long)m + i;
  const unsigned long long b1 = splitmix_at(seed, 2ull * c);
  const unsigned long long b2 = splitmix_at(seed, 2ull * c + 1ull);
  const double u1 = ((double)(b1 >> 11) + 0.5) * 0x1.0p-53;
  const double u2 = ((double)(b2 >> 11) + 0.5) * 0x1.0p-53;
  const double two_pi = 2.0 * 3.141592653589793;
  Om[(size_t)j * ld + i] = sqrt(-2.0 * log(u1)) * cos(two_pi * u2);
}

__global__ void k_gaussian_dev(unsigned long long seed, const int* __restrict__ k_dev, int k0, int m, int ell,
                               double* __restrict__ Om, int ld) {
  const long long idx = (long long)blockIdx.x * kNT + threadIdx.x;
  if (idx >= (long long)m * ell) return;
  const int i = (int)(idx % m);
  const int j = (int)(idx / m);
  const unsigned long long k = (unsigned long long)(*k_dev + k0);
  const unsigned long long c = (k * ell + j) * (unsigned long long)m + i;
  const unsigned long long b1 = splitmix_at(seed, 2ull * c);
  const unsigned long long b2 = splitmix_at(seed, 2ull * c + 1ull);
  const double u1 = ((double)(b1 >> 11) + 0.5) * 0x1.0p-53;
  const double u2 = ((double)(b2 >> 11) + 0.5) * 0x1.0p-53;
  const double two_pi = 2.0 * 3.141592653589793;
  Om[(size_t)j * ld + i] = sqrt(-2.0 * log(u1)) * cos(two_pi * u2);
}

// ---- FP64 SIMT GEMM
// TBM x TBN output tiles (64 x 64, or 32 x 32 for the skinny products of a
// small sketch, so that few DFMAs go to padding), 16-deep k-slices staged in
// shared memory, (TBM/16) x (TBN/16) outputs per thread.
constexpr int BK = 16;

template <bool kAK, int TBM, int TBN>  // kAK: A's k index is contiguous (sak == 1); else r is (sar == 1)
__global__ void __launch_bounds__(256) k_gemm_f64(int M, int N, int K, int kchunk,
                                                  const double* __restrict__ A, long long sar,
                                                  long long sak, const double* __restrict__ B,
                                                  long long sbc, const double* __restrict__ scale,
                                                  double* __restrict__ C, long long scr,
                                                  long long scc, double* __restrict__ part) {
  constexpr int RM = TBM / 16, RN = TBN / 16;   // outputs per thread
  constexpr int EA = BK * TBM / 256, EB = BK * TBN / 256;
  __shared__ double As[BK][TBM + 1];
  __shared__ double Bs[BK][TBN + 1];
  const int tid = threadIdx.x;
  const int r0 = blockIdx.x * TBM, c0 = blockIdx.y * TBN;
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);
  const int tr = tid >> 4, tc = tid & 15;
  double acc[RM][RN];
#pragma unroll
  for (int a = 0; a < RM; ++a)
#pragma unroll
    for (int b = 0; b < RN; ++b) acc[a][b] = 0.0;

  for (int kk = kbeg; kk < kend; kk += BK) {
#pragma unroll
    for (int e = 0; e < EA; ++e) {
      const int idx = tid + e * 256;
      int r, k;
      if (kAK) { r = idx / BK; k = idx % BK; } else { r = idx % TBM; k = idx / TBM; }
      const int gr = r0 + r, gk = kk + k;
      double val = 0.0;
      if (gr < M && gk < kend) val = __ldg(A + (long long)gr * sar + (long long)gk * sak);
      As[k][r] = val;
    }
#pragma unroll
    for (int e = 0; e < EB; ++e) {
      const int idx = tid + e * 256;
      const int k = idx % BK, c = idx / BK;
      const int gk = kk + k, gc = c0 + c;
      double val = 0.0;
      if (gc < N && gk < kend) {
        val = __ldg(B + (long long)gk + (long long)gc * sbc);
        if (scale) val *= __ldg(scale + gk);
      }
      Bs[k][c] = val;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      double a[RM], b[RN];
#pragma unroll
      for (int t = 0; t < RM; ++t) a[t] = As[k][tr * RM + t];
#pragma unroll
      for (int t = 0; t < RN; ++t) b[t] = Bs[k][tc * RN + t];
#pragma unroll
      for (int x = 0; x < RM; ++x)
#pragma unroll
        for (int y = 0; y < RN; ++y) acc[x][y] = fma(a[x], b[y], acc[x][y]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int x = 0; x < RM; ++x) {
    const int gr = r0 + tr * RM + x;
    if (gr >= M) continue;
#pragma unroll
    for (int y = 0; y < RN; ++y) {
      const int gc = c0 + tc * RN + y;
      if (gc >= N) continue;
      if (part) part[(size_t)blockIdx.z * M * N + (size_t)gc * M + gr] = acc[x][y];
      else C[(long long)gr * scr + (long long)gc * scc] = acc[x][y];
    }
  }
}

__global__ void k_splitk_reduce(int M, int N, int S, const double* __restrict__ part,
                                double* __restrict__ C, long long scr, long long scc) {
  const long long idx = (long long)blockIdx.x * kNT + threadIdx.x;
  if (idx >= (long long)M * N) return;
  const int r = (int)(idx % M), c = (int)(idx / M);
  double s = 0.0;
  for (int z = 0; z < S; ++z) s += part[(size_t)z * M * N + idx];
  C[(long long)r * scr + (long long)c * scc] = s;
}

}  // namespace

cudaError_t gaussian_omega(cudaStream_t st, unsigned long long seed, int k, int m, int ell,
                           double* Om, int ld, int cols) {
  if (cols < 0 || cols > ell) cols = ell;
  const long long total = (long long)m * cols;
  if (total <= 0) return cudaSuccess;
  count_launches(1);
  k_gaussian<<<(unsigned)((total + kNT - 1) / kNT), kNT, 0, st>>>(seed, k, m, ell, cols, Om, ld);
  return cudaGetLastError();
}

cudaError_t gaussian_omega_dev(cudaStream_t st, unsigned long long seed, const int* k_dev, int k0, int m, int ell,
                               double* Om, int ld) {
  const long long total = (long long)m * ell;
  if (total <= 0) return cudaSuccess;
  count_launches(1);
  k_gaussian_dev<<<(unsigned)((total + kNT - 1) / kNT), kNT, 0, st>>>(seed, k_dev, k0, m, ell, Om, ld);
  return cudaGetLastError();
}

cudaError_t gemm_f64(cudaStream_t st, int M, int N, int K, const double* A, long long sar,
                     long long sak, const double* B, long long sbk, long long sbc,
                     const double* scale, double* C, long long scr, long long scc,
                     double* split_buf, size_t split_cap) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (sbk != 1 || (sar != 1 && sak != 1)) return cudaErrorInvalidValue;
  // small N (a sketch of rank <= 32): 32 x 32 tiles
  const bool skinny = N <= 32;
  const int tbm = skinny ? 32 : 64, tbn = skinny ? 32 : 64;
  const int tiles = ((M + tbm - 1) / tbm) * ((N + tbn - 1) / tbn);
  const int ksteps = (K + BK - 1) / BK;
  // split K until the grid covers the GPU about four times (each split keeps
  // at least two 16-deep slices), within the partial-sum scratch
  int S = (152 * 4 + tiles - 1) / tiles;
  if (S > ksteps / 2) S = ksteps / 2;
  if (S < 1) S = 1;
  while (S > 1 && (size_t)S * M * N > split_cap) --S;
  const int kchunk = ((ksteps + S - 1) / S) * BK;
  S = (K + kchunk - 1) / kchunk;
  if (S < 1) S = 1;
  dim3 grid((M + tbm - 1) / tbm, (N + tbn - 1) / tbn, S);
  double* part = (S > 1) ? split_buf : nullptr;
  count_launches(1);
  if (skinny) {
    if (sak == 1)
      k_gemm_f64<true, 32, 32><<<grid, 256, 0, st>>>(M, N, K, kchunk, A, sar, sak, B, sbc, scale, C, scr, scc, part);
    else
      k_gemm_f64<false, 32, 32><<<grid, 256, 0, st>>>(M, N, K, kchunk, A, sar, sak, B, sbc, scale, C, scr, scc, part);
  } else {
    if (sak == 1)
      k_gemm_f64<true, 64, 64><<<grid, 256, 0, st>>>(M, N, K, kchunk, A, sar, sak, B, sbc, scale, C, scr, scc, part);
    else
      k_gemm_f64<false, 64, 64><<<grid, 256, 0, st>>>(M, N, K, kchunk, A, sar, sak, B, sbc, scale, C, scr, scc, part);
  }
  if (S > 1) {
    const long long total = (long long)M * N;
    count_launches(1);
    k_splitk_reduce<<<(unsigned)((total + kNT - 1) / kNT), kNT, 0, st>>>(M, N, S, part, C, scr, scc);
  }
  return cudaGetLastError();
}

cudaError_t sketch_f64(cudaStream_t st, int m, int n, const double* A, long long lda,
                       const double* D, int ell, const double* Om, int ld, double* Y,
                       double* T, int ld_t, double* split_buf, size_t split_cap) {
  // T (n x ell) = A^T Omega
  cudaError_t e = gemm_f64(st, n, ell, m, A, 1, lda, Om, 1, ld, nullptr, T, 1, ld_t, split_buf, split_cap);
  if (e != cudaSuccess) return e;
  // Y (m x ell) = A (D .* T)
  return gemm_f64(st, m, ell, n, A, lda, 1, T, 1, ld_t, D, Y, 1, ld, split_buf, split_cap);
}

}  // namespace nys
