// Streaming row-reduction GEMVs for the precision form (reduced-precision
// storage of A, Section 2.1.2's operator N = A D A^T applied in two passes).
//
// Both passes of the operator are row reductions because the precision form
// keeps A and A^T as separate row-major copies (A^T v = rows of A^T times v):
// every pass streams its matrix once, fully coalesced, 16 bytes per lane.
//
//   k_rows<T, R>   out[r] = scale[r] * sum_c M[r, c] x[c] (+ beta v[r])
//                  T = FP8 (E4M3), BF16 or FP32 storage, FP32 products and
//                  accumulation;
//                  one warp owns R rows and reuses each 8-element chunk of x
//                  for all R rows (x traffic is 1/R of the naive one).
//   k_rows_ff<R>   the same with FP32 storage and a float-float (hi + lo)
//                  accumulator: x is split into hi/lo FP32 parts, every
//                  product a*x_hi is made exact with an FMA (Dekker/Knuth
//                  two-product) and summed with two-sum; the lane and warp
//                  totals are combined in FP64.  About 2^-44 relative
//                  accuracy at FP32 throughput: GB300 runs FP32 ~70x faster
//                  than FP64.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "common.cuh"
#include "internal.h"

namespace nys {

namespace {

constexpr int kRowsPerWarp = 4;       // measured best of 4 and 8 (also with 8 warps per block)
constexpr int kWarpsPerBlock = 4;

__device__ __forceinline__ void load8(const __nv_bfloat16* p, float (&v)[8]) {
  const uint4 u = __ldg(reinterpret_cast<const uint4*>(p));
  const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float2 f = __bfloat1622float2(h[i]);
    v[2 * i] = f.x;
    v[2 * i + 1] = f.y;
  }
}

__device__ __forceinline__ void load8(const float* p, float (&v)[8]) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(p));
  const float4 b = __ldg(reinterpret_cast<const float4*>(p + 4));
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

// 16 FP8 E4M3 values (16 bytes) to FP32
__device__ __forceinline__ void load16(const __nv_fp8_e4m3* p, float (&v)[16]) {
  const uint4 u = __ldg(reinterpret_cast<const uint4*>(p));
  const __nv_fp8x2_storage_t* q = reinterpret_cast<const __nv_fp8x2_storage_t*>(&u);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2(q[i], __NV_E4M3);
    const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&hr));
    v[2 * i] = f.x;
    v[2 * i + 1] = f.y;
  }
}

// the same 16-element step for the 2- and 4-byte types (two 8-element loads)
__device__ __forceinline__ void load16(const __nv_bfloat16* p, float (&v)[16]) {
  float a[8], b[8];
  load8(p, a);
  load8(p + 8, b);
#pragma unroll
  for (int i = 0; i < 8; ++i) { v[i] = a[i]; v[8 + i] = b[i]; }
}
__device__ __forceinline__ void load16(const float* p, float (&v)[16]) {
  float a[8], b[8];
  load8(p, a);
  load8(p + 8, b);
#pragma unroll
  for (int i = 0; i < 8; ++i) { v[i] = a[i]; v[8 + i] = b[i]; }
}

template <typename TA>
__device__ __forceinline__ float load1(const TA* p);
template <>
__device__ __forceinline__ float load1<__nv_fp8_e4m3>(const __nv_fp8_e4m3* p) { return float(p[0]); }
template <>
__device__ __forceinline__ float load1<__nv_bfloat16>(const __nv_bfloat16* p) { return __bfloat162float(p[0]); }
template <>
__device__ __forceinline__ float load1<float>(const float* p) { return __ldg(p); }

// out[r] = scale[r] * sum_c A[r, c] x[c] + beta * v[r]  (FP32 accumulate)
// vec: rows start 16-byte aligned (lda a multiple of 8 for BF16, 4 for FP32)
template <typename TA, typename TO, bool kVec>
__global__ void __launch_bounds__(32 * kWarpsPerBlock)
    k_rows(int rows, int cols, const TA* __restrict__ A, long long lda, const float* __restrict__ x,
           const float* __restrict__ scale, double beta, const double* __restrict__ v, TO* __restrict__ out,
           const int* __restrict__ skip, const double* __restrict__ beta_dev, int cols_per_split,
           double* __restrict__ part) {
  if (skip && *skip) return;
  if (beta_dev) beta = *beta_dev;
  const int lane = threadIdx.x & 31;
  const int r0 = (blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5)) * kRowsPerWarp;
  if (r0 >= rows) return;
  // this block's column range (a multiple of 16 wide, except the last)
  const int cb = blockIdx.y * cols_per_split;
  const int ce = min(cols, cb + cols_per_split);
  float acc[kRowsPerWarp];
#pragma unroll
  for (int i = 0; i < kRowsPerWarp; ++i) acc[i] = 0.0f;
  // 16 elements a lane per step for FP8 (one 16-byte load), 8 otherwise
  constexpr int kE = sizeof(TA) == 1 ? 16 : 8;
  const int cvec = kVec ? cb + ((ce - cb) / kE) * kE : cb;
  for (int c = cb + lane * kE; c < cvec; c += 32 * kE) {
    if constexpr (kE == 16) {
      float xv[16];
      load8(x + c, *reinterpret_cast<float(*)[8]>(xv));
      load8(x + c + 8, *reinterpret_cast<float(*)[8]>(xv + 8));
#pragma unroll
      for (int i = 0; i < kRowsPerWarp; ++i) {
        const int r = min(r0 + i, rows - 1);
        float a[16];
        load16(A + (long long)r * lda + c, a);
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[i] = fmaf(a[j], xv[j], acc[i]);
      }
    } else {
      float xv[8];
      load8(x + c, xv);
#pragma unroll
      for (int i = 0; i < kRowsPerWarp; ++i) {
        const int r = min(r0 + i, rows - 1);
        float a[8];
        load8(A + (long long)r * lda + c, a);
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i] = fmaf(a[j], xv[j], acc[i]);
      }
    }
  }
  for (int c = cvec + lane; c < ce; c += 32) {
    const float xc = __ldg(x + c);
#pragma unroll
    for (int i = 0; i < kRowsPerWarp; ++i) {
      const int r = min(r0 + i, rows - 1);
      acc[i] = fmaf(load1<TA>(A + (long long)r * lda + c), xc, acc[i]);
    }
  }
#pragma unroll
  for (int i = 0; i < kRowsPerWarp; ++i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], o);
  }
  if (lane < kRowsPerWarp) {
    float mine = acc[0];
#pragma unroll
    for (int i = 1; i < kRowsPerWarp; ++i)
      if (lane == i) mine = acc[i];
    const int r = r0 + lane;
    if (r < rows && part) {
      part[(size_t)blockIdx.y * rows + r] = (double)mine;
    } else if (r < rows) {
      double val = (double)mine * (scale ? (double)scale[r] : 1.0);
      if (beta != 0.0) val = fma(beta, v[r], val);
      out[r] = (TO)val;
    }
  }
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// FP32 matrix times a float-float vector (xh + xl), float-float accumulation.
// out[r] = scale[r] * (sum) + beta v[r] in FP64.
template <bool kVec>
__global__ void __launch_bounds__(32 * kWarpsPerBlock)
    k_rows_ff(int rows, int cols, const float* __restrict__ A, long long lda, const float* __restrict__ xh,
              const float* __restrict__ xl, const double* __restrict__ scale, double beta,
              const double* __restrict__ v, double* __restrict__ out, const int* __restrict__ skip,
              const double* __restrict__ beta_dev, int cols_per_split, double* __restrict__ part) {
  if (skip && *skip) return;
  if (beta_dev) beta = *beta_dev;
  const int lane = threadIdx.x & 31;
  const int r0 = (blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5)) * kRowsPerWarp;
  if (r0 >= rows) return;
  const int cb = blockIdx.y * cols_per_split;
  const int ce = min(cols, cb + cols_per_split);
  float sh[kRowsPerWarp], sl[kRowsPerWarp];
#pragma unroll
  for (int i = 0; i < kRowsPerWarp; ++i) { sh[i] = 0.0f; sl[i] = 0.0f; }
  const int cvec = kVec ? cb + ((ce - cb) / 8) * 8 : cb;
  for (int c = cb + lane * 8; c < cvec; c += 256) {
    float xa[8], xb[8];
    load8(xh + c, xa);
    load8(xl + c, xb);
#pragma unroll
    for (int i = 0; i < kRowsPerWarp; ++i) {
      const int r = min(r0 + i, rows - 1);
      float a[8];
      load8(A + (long long)r * lda + c, a);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const float p = a[j] * xa[j];
        const float pe = fmaf(a[j], xa[j], -p) + a[j] * xb[j];   // exact low part + a * x_lo
        float s, e;
        two_sum(sh[i], p, s, e);
        sh[i] = s;
        sl[i] += e + pe;
      }
    }
  }
  for (int c = cvec + lane; c < ce; c += 32) {
    const float xa = __ldg(xh + c), xb = __ldg(xl + c);
#pragma unroll
    for (int i = 0; i < kRowsPerWarp; ++i) {
      const int r = min(r0 + i, rows - 1);
      const float a = __ldg(A + (long long)r * lda + c);
      const float p = a * xa;
      const float pe = fmaf(a, xa, -p) + a * xb;
      float s, e;
      two_sum(sh[i], p, s, e);
      sh[i] = s;
      sl[i] += e + pe;
    }
  }
  double tot[kRowsPerWarp];
#pragma unroll
  for (int i = 0; i < kRowsPerWarp; ++i) {
    double d = (double)sh[i] + (double)sl[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    tot[i] = d;
  }
  if (lane < kRowsPerWarp) {
    double mine = tot[0];
#pragma unroll
    for (int i = 1; i < kRowsPerWarp; ++i)
      if (lane == i) mine = tot[i];
    const int r = r0 + lane;
    if (r < rows && part) {
      part[(size_t)blockIdx.y * rows + r] = mine;
    } else if (r < rows) {
      double val = mine * (scale ? scale[r] : 1.0);
      if (beta != 0.0) val = fma(beta, v[r], val);
      out[r] = val;
    }
  }
}

// out[r] = scale[r] * sum_z part[z][r] + beta v[r]   (fixed order over z)
template <typename TS, typename TO>
__global__ void k_rows_finish(int rows, int splits, const double* __restrict__ part, const TS* __restrict__ scale,
                              double beta, const double* __restrict__ v, TO* __restrict__ out,
                              const int* __restrict__ skip, const double* __restrict__ beta_dev) {
  if (skip && *skip) return;
  if (beta_dev) beta = *beta_dev;
  const int r = blockIdx.x * kNT + threadIdx.x;
  if (r >= rows) return;
  double s = 0.0;
  for (int z = 0; z < splits; ++z) s += part[(size_t)z * rows + r];
  double val = s * (scale ? (double)scale[r] : 1.0);
  if (beta != 0.0) val = fma(beta, v[r], val);
  out[r] = (TO)val;
}

// x (FP64) -> hi, lo FP32 parts with x ~ hi + lo; padded entries are zero.
__global__ void k_split_ff(int n, int npad, const double* __restrict__ x, const double* __restrict__ scale,
                           float* __restrict__ hi, float* __restrict__ lo, const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int j = blockIdx.x * kNT + threadIdx.x;
  if (j >= npad) return;
  double v = 0.0;
  if (j < n) v = scale ? x[j] * scale[j] : x[j];
  const float h = (float)v;
  hi[j] = h;
  lo[j] = (float)(v - (double)h);
}

// FP64 -> FP32 (optionally scaled), zero padded to npad.
__global__ void k_to_f32(int n, int npad, const double* __restrict__ x, const double* __restrict__ scale,
                         float* __restrict__ y, const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int j = blockIdx.x * kNT + threadIdx.x;
  if (j >= npad) return;
  y[j] = j < n ? (float)(scale ? x[j] * scale[j] : x[j]) : 0.0f;
}

// Row-major src (rows x cols, lds) -> BF16 row-major copy and BF16 transpose,
// both zero padded to their leading dimensions.  32x32 tiles through shared memory.
template <typename TS>
__global__ void k_convert_transpose(int rows, int cols, const TS* __restrict__ src, long long lds,
                                    __nv_bfloat16* __restrict__ dst, long long ldd,
                                    __nv_bfloat16* __restrict__ dstT, long long ldt,
                                    float* __restrict__ dstTf, long long ldtf) {
  __shared__ float tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8 threads
  for (int k = ty; k < 32; k += 8) {
    const int r = r0 + k, c = c0 + tx;
    float v = 0.0f;
    if (r < rows && c < cols) v = (float)src[(long long)r * lds + c];
    tile[k][tx] = v;
    if (dst && r < rows && c < ldd) dst[(long long)r * ldd + c] = __float2bfloat16_rn(v);
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    const int c = c0 + k, r = r0 + tx;     // output row c of the transpose, column r
    if (c < cols) {
      if (dstT && r < ldt) dstT[(long long)c * ldt + r] = __float2bfloat16_rn(tile[tx][k]);
      if (dstTf && r < ldtf) dstTf[(long long)c * ldtf + r] = tile[tx][k];
    }
  }
}

// Per-row scales of an FP32 matrix for E4M3 storage: s_r = max_c |A[r, c]| / 448
// (448 = the largest finite E4M3 value), 1 for an all-zero row; one warp per row.
__global__ void k_row_scale_fp8(int rows, int cols, const float* __restrict__ A, long long lda,
                                float* __restrict__ s32, double* __restrict__ s64) {
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (r >= rows) return;
  float mx = 0.0f;
  for (int c = lane; c < cols; c += 32) mx = fmaxf(mx, fabsf(__ldg(A + (long long)r * lda + c)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) {
    const float sc = mx > 0.0f ? mx / 448.0f : 1.0f;
    s32[r] = sc;
    s64[r] = (double)sc;
  }
}

// Q[r, c] = E4M3(A[r, c] / s_r) (round to nearest, saturating) and its
// transpose QT[c, r]; padding columns zeroed.  32 x 32 tiles.
__global__ void k_quant_fp8(int rows, int cols, const float* __restrict__ A, long long lda,
                            const float* __restrict__ s32, __nv_fp8_e4m3* __restrict__ Q, long long ldq,
                            __nv_fp8_e4m3* __restrict__ QT, long long ldqt) {
  __shared__ __nv_fp8_storage_t tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8 threads
  for (int k = ty; k < 32; k += 8) {
    const int r = r0 + k, c = c0 + tx;
    __nv_fp8_storage_t q = 0;
    if (r < rows && c < cols) q = __nv_cvt_float_to_fp8(__ldg(A + (long long)r * lda + c) / s32[r], __NV_SATFINITE, __NV_E4M3);
    tile[k][tx] = q;
    if (r < rows && c < ldq) reinterpret_cast<__nv_fp8_storage_t*>(Q)[(long long)r * ldq + c] = q;
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    const int c = c0 + k, r = r0 + tx;     // output row c of the transpose, column r
    if (c < cols && r < ldqt) reinterpret_cast<__nv_fp8_storage_t*>(QT)[(long long)c * ldqt + r] = tile[tx][k];
  }
}

int row_blocks(int rows) {
  const int per = kRowsPerWarp * kWarpsPerBlock;
  return (rows + per - 1) / per;
}

// Column splits: enough blocks for ~4 per SM; every split at least 2048
// columns wide; limited by the partial-sum scratch.
int col_splits(int rows, int cols, size_t part_cap) {
  const int rb = row_blocks(rows);
  int s = (152 * 4 + rb - 1) / rb;
  const int smax = cols / 2048;
  if (s > smax) s = smax;
  while (s > 1 && (size_t)s * rows > part_cap) --s;
  return s < 1 ? 1 : s;
}

}  // namespace

cudaError_t gemv_rows_lp(cudaStream_t st, int rows, int cols, int a_type, const void* A, long long lda,
                         const float* x, const float* scale, double beta, const double* v, void* out,
                         int out_f64, const int* skip, const double* beta_dev, double* part, size_t part_cap) {
  if (rows <= 0) return cudaSuccess;
  const int S = part ? col_splits(rows, cols, part_cap) : 1;
  const int cps = S > 1 ? ((cols + S - 1) / S + 15) / 16 * 16 : cols;
  const int nsplit = (cols + cps - 1) / cps;
  double* pp = nsplit > 1 ? part : nullptr;
  dim3 grid(row_blocks(rows), nsplit);
  const int T = 32 * kWarpsPerBlock;
  count_launches(1);
  if (a_type == kLpFp8) {
    const bool vec = (lda % 16 == 0) && ((reinterpret_cast<uintptr_t>(A) & 15u) == 0);
    const auto* a = static_cast<const __nv_fp8_e4m3*>(A);
    if (out_f64) {
      if (vec) k_rows<__nv_fp8_e4m3, double, true><<<grid, T, 0, st>>>(rows, cols, a, lda, x, scale, beta, v, (double*)out, skip, beta_dev, cps, pp);
      else k_rows<__nv_fp8_e4m3, double, false><<<grid, T, 0, st>>>(rows, cols, a, lda, x, scale, beta, v, (double*)out, skip, beta_dev, cps, pp);
    } else {
      if (vec) k_rows<__nv_fp8_e4m3, float, true><<<grid, T, 0, st>>>(rows, cols, a, lda, x, scale, beta, v, (float*)out, skip, beta_dev, cps, pp);
      else k_rows<__nv_fp8_e4m3, float, false><<<grid, T, 0, st>>>(rows, cols, a, lda, x, scale, beta, v, (float*)out, skip, beta_dev, cps, pp);
    }
  } else if (a_type == kLpBf16) {
    const bool vec = (lda % 8 == 0) && ((reinterpret_cast<uintptr_t>(A) & 15u) == 0);
    const auto* a = static_cast<const __nv_bfloat16*>(A);
    if (out_f64) {
      if (vec) k_rows<__nv_bfloat16, double, true><<<grid, T, 0, st>>>(rows, cols, a, lda, x, scale, beta, v, (double*)out, skip, beta_dev, cps, pp);
      else k_rows<__nv_bfloat16, double, false><<<grid, T, 0, st>>>(rows, cols, a, lda, x, scale, beta, v, (double*)out, skip, beta_dev, cps, pp);
    } else {
      if (vec) k_rows<__nv_bfloat16, float, true><<<grid, T, 0, st>>>(rows, cols, a, lda, x, scale, beta, v, (float*)out, skip, beta_dev, cps, pp);
      else k_rows<__nv_bfloat16, float, false><<<grid, T, 0, st>>>(rows, cols, a, lda, x, scale, beta, v, (float*)out, skip, beta_dev, cps, pp);
    }
  } else {
    const bool vec = (lda % 4 == 0) && ((reinterpret_cast<uintptr_t>(A) & 15u) == 0);
    const auto* a = static_cast<const float*>(A);
    if (out_f64) {
      if (vec) k_rows<float, double, true><<<grid, T, 0, st>>>(rows, cols, a, lda, x, scale, beta, v, (double*)out, skip, beta_dev, cps, pp);
      else k_rows<float, double, false><<<grid, T, 0, st>>>(rows, cols, a, lda, x, scale, beta, v, (double*)out, skip, beta_dev, cps, pp);
    } else {
      if (vec) k_rows<float, float, true><<<grid, T, 0, st>>>(rows, cols, a, lda, x, scale, beta, v, (float*)out, skip, beta_dev, cps, pp);
      else k_rows<float, float, false><<<grid, T, 0, st>>>(rows, cols, a, lda, x, scale, beta, v, (float*)out, skip, beta_dev, cps, pp);
    }
  }
  if (pp) {
    count_launches(1);
    const int fb = (rows + kNT - 1) / kNT;
    if (out_f64) k_rows_finish<float, double><<<fb, kNT, 0, st>>>(rows, nsplit, pp, scale, beta, v, (double*)out, skip, beta_dev);
    else k_rows_finish<float, float><<<fb, kNT, 0, st>>>(rows, nsplit, pp, scale, beta, v, (float*)out, skip, beta_dev);
  }
  return cudaGetLastError();
}

cudaError_t gemv_rows_ff(cudaStream_t st, int rows, int cols, const float* A, long long lda, const float* xh,
                         const float* xl, const double* scale, double beta, const double* v, double* out,
                         const int* skip, const double* beta_dev, double* part, size_t part_cap) {
  if (rows <= 0) return cudaSuccess;
  const int S = part ? col_splits(rows, cols, part_cap) : 1;
  const int cps = S > 1 ? ((cols + S - 1) / S + 7) / 8 * 8 : cols;
  const int nsplit = (cols + cps - 1) / cps;
  double* pp = nsplit > 1 ? part : nullptr;
  dim3 grid(row_blocks(rows), nsplit);
  const bool vec = (lda % 4 == 0) && ((reinterpret_cast<uintptr_t>(A) & 15u) == 0);
  count_launches(1);
  if (vec) k_rows_ff<true><<<grid, 32 * kWarpsPerBlock, 0, st>>>(rows, cols, A, lda, xh, xl, scale, beta, v, out, skip, beta_dev, cps, pp);
  else k_rows_ff<false><<<grid, 32 * kWarpsPerBlock, 0, st>>>(rows, cols, A, lda, xh, xl, scale, beta, v, out, skip, beta_dev, cps, pp);
  if (pp) {
    count_launches(1);
    k_rows_finish<double, double><<<(rows + kNT - 1) / kNT, kNT, 0, st>>>(rows, nsplit, pp, scale, beta, v, out, skip, beta_dev);
  }
  return cudaGetLastError();
}

cudaError_t split_ff(cudaStream_t st, int n, int npad, const double* x, const double* scale, float* hi, float* lo,
                     const int* skip) {
  count_launches(1);
  k_split_ff<<<(npad + kNT - 1) / kNT, kNT, 0, st>>>(n, npad, x, scale, hi, lo, skip);
  return cudaGetLastError();
}

cudaError_t to_f32(cudaStream_t st, int n, int npad, const double* x, const double* scale, float* y,
                   const int* skip) {
  count_launches(1);
  k_to_f32<<<(npad + kNT - 1) / kNT, kNT, 0, st>>>(n, npad, x, scale, y, skip);
  return cudaGetLastError();
}

cudaError_t convert_transpose(cudaStream_t st, int rows, int cols, int src_f64, const void* src, long long lds,
                              __nv_bfloat16* dst, long long ldd, __nv_bfloat16* dstT, long long ldt,
                              float* dstTf, long long ldtf) {
  // cover the padded extents of the copies (zero fill)
  long long cext = cols, rext = rows;
  if (dst && ldd > cext) cext = ldd;
  if (dstT && ldt > rext) rext = ldt;
  if (dstTf && ldtf > rext) rext = ldtf;
  dim3 grid((unsigned)((cext + 31) / 32), (unsigned)((rext + 31) / 32));
  count_launches(1);
  if (src_f64)
    k_convert_transpose<double><<<grid, 256, 0, st>>>(rows, cols, (const double*)src, lds, dst, ldd, dstT, ldt, dstTf, ldtf);
  else
    k_convert_transpose<float><<<grid, 256, 0, st>>>(rows, cols, (const float*)src, lds, dst, ldd, dstT, ldt, dstTf, ldtf);
  return cudaGetLastError();
}

cudaError_t quantize_fp8(cudaStream_t st, int rows, int cols, const float* A, long long lda, float* s32,
                         double* s64, void* Q, long long ldq, void* QT, long long ldqt) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  count_launches(2);
  k_row_scale_fp8<<<(rows + 7) / 8, 256, 0, st>>>(rows, cols, A, lda, s32, s64);
  dim3 grid((cols + 31) / 32, (rows + 31) / 32);
  k_quant_fp8<<<grid, 256, 0, st>>>(rows, cols, A, lda, s32, static_cast<__nv_fp8_e4m3*>(Q), ldq,
                                    static_cast<__nv_fp8_e4m3*>(QT), ldqt);
  return cudaGetLastError();
}

}  // namespace nys
