// Vector kernels of the practical initial point (the supplement's
// construction for the initial point, after Mehrotra and
// Pougkakiotis-Gondzio): the candidate's dual slacks and bound multipliers,
// the shifts that make it strictly interior, and the shifted start.  FP64;
// reductions are the deterministic last-block sums and minima of common.cuh.
//
// vk may be null (problem (P): every variable in I); then w and s are not
// touched.  Kinds as in ipm_box.cu: 0 = I, 1 = F (free), 2 = J (boxed).
#include "common.cuh"
#include "internal.h"

namespace nys {

namespace {

constexpr signed char kI = 0, kF = 1, kJ = 2;

int grid_for(long long len) {
  long long b = (len + kNT - 1) / kNT;
  if (b > 2 * 152) b = 2 * 152;
  return b < 1 ? 1 : (int)b;
}

__global__ void k_fill(int len, double v, double* __restrict__ out) {
  const int j = blockIdx.x * kNT + threadIdx.x;
  if (j < len) out[j] = v;
}

// g = c - A^T y~ + Q x~;  z~ = g/2 on J, g on I (0 on F: the start has z_F = 0);
// on J s~ = -z~ and w~ = u - x~.
// out[0] = min of x~ over I u J and of w~ over J; out[1] = min of z~ over
// I u J and of s~ over J (+inf when the sets are empty).
__global__ void __launch_bounds__(kNT) k_start_candidate(int n, const signed char* __restrict__ vk,
                                                         const double* __restrict__ c, const double* __restrict__ q,
                                                         const double* __restrict__ u, const double* __restrict__ x,
                                                         const double* __restrict__ Aty, double* __restrict__ z,
                                                         double* __restrict__ w, double* __restrict__ s, double* out,
                                                         double* part, unsigned* cnt) {
  double pm = INFINITY, dm = INFINITY;
  for (int j = blockIdx.x * kNT + threadIdx.x; j < n; j += gridDim.x * kNT) {
    const signed char k = vk ? vk[j] : kI;
    const double xj = x[j];
    const double g = c[j] - Aty[j] + q[j] * xj;
    const double zt = k == kJ ? 0.5 * g : g;
    z[j] = k == kF ? 0.0 : zt;
    if (k != kF) {
      pm = fmin(pm, xj);
      dm = fmin(dm, zt);
    }
    if (k == kJ) {
      const double wt = u[j] - xj, st = -zt;
      w[j] = wt;
      s[j] = st;
      pm = fmin(pm, wt);
      dm = fmin(dm, st);
    }
  }
  double o;
  if (grid_min<kNT>(pm, part, cnt, &o) && threadIdx.x == 0) out[0] = o;
  if (grid_min<kNT>(dm, part + gridDim.x, cnt + 1, &o) && threadIdx.x == 0) out[1] = o;
}

// out[0] = gamma = (x~ + dp)_IJ^T (z~ + dd)_IJ + (w~ + dp)_J^T (s~ + dd)_J,
// out[1] = sum of (z~ + dd) over I u J and (s~ + dd) over J,
// out[2] = sum of (x~ + dp) over I u J and (w~ + dp) over J.
__global__ void __launch_bounds__(kNT) k_start_sums(int n, const signed char* __restrict__ vk,
                                                    const double* __restrict__ x, const double* __restrict__ z,
                                                    const double* __restrict__ w, const double* __restrict__ s,
                                                    double dp, double dd, double* out, double* part, unsigned* cnt) {
  double v[3] = {0.0, 0.0, 0.0};
  for (int j = blockIdx.x * kNT + threadIdx.x; j < n; j += gridDim.x * kNT) {
    const signed char k = vk ? vk[j] : kI;
    if (k == kF) continue;
    const double xp = x[j] + dp, zd = z[j] + dd;
    v[0] = fma(xp, zd, v[0]);
    v[1] += zd;
    v[2] += xp;
    if (k == kJ) {
      const double wp = w[j] + dp, sd = s[j] + dd;
      v[0] = fma(wp, sd, v[0]);
      v[1] += sd;
      v[2] += wp;
    }
  }
  double tot[3];
  if (grid_sum<kNT, 3>(v, part, cnt, tot) && threadIdx.x == 0)
    for (int i = 0; i < 3; ++i) out[i] = tot[i];
}

// x_IJ += dpt, w_J += dpt, z_IJ += ddt, s_J += ddt (x_F unshifted, z_F = 0)
__global__ void k_start_shift(int n, const signed char* __restrict__ vk, double dpt, double ddt,
                              double* __restrict__ x, double* __restrict__ z, double* __restrict__ w,
                              double* __restrict__ s) {
  const int j = blockIdx.x * kNT + threadIdx.x;
  if (j >= n) return;
  const signed char k = vk ? vk[j] : kI;
  if (k == kF) return;
  x[j] += dpt;
  z[j] += ddt;
  if (k == kJ) {
    w[j] += dpt;
    s[j] += ddt;
  }
}

}  // namespace

cudaError_t fill_f64(cudaStream_t st, int len, double v, double* out) {
  if (len <= 0) return cudaSuccess;
  count_launches(1);
  k_fill<<<(len + kNT - 1) / kNT, kNT, 0, st>>>(len, v, out);
  return cudaGetLastError();
}

cudaError_t start_candidate_f64(cudaStream_t st, int n, const signed char* vk, const double* c, const double* q,
                                const double* u, const double* x, const double* Aty, double* z, double* w,
                                double* s, double* out, RedBuf red) {
  count_launches(1);
  k_start_candidate<<<grid_for(n), kNT, 0, st>>>(n, vk, c, q, u, x, Aty, z, w, s, out, red.part, red.cnt + 13);
  return cudaGetLastError();
}

cudaError_t start_sums_f64(cudaStream_t st, int n, const signed char* vk, const double* x, const double* z,
                           const double* w, const double* s, double dp, double dd, double* out, RedBuf red) {
  count_launches(1);
  k_start_sums<<<grid_for(n), kNT, 0, st>>>(n, vk, x, z, w, s, dp, dd, out, red.part, red.cnt + 12);
  return cudaGetLastError();
}

cudaError_t start_shift_f64(cudaStream_t st, int n, const signed char* vk, double dpt, double ddt, double* x,
                            double* z, double* w, double* s) {
  count_launches(1);
  k_start_shift<<<(n + kNT - 1) / kNT, kNT, 0, st>>>(n, vk, dpt, ddt, x, z, w, s);
  return cudaGetLastError();
}

}  // namespace nys
