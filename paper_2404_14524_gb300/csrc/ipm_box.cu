// Vector kernels of the IP-PMM iteration for problems with free and
// box-constrained variables, (P~)/(D~): Algorithm 4 with the slack
// w = u - x and its multiplier s, the right-hand sides of Eq. predictor-RHS
// and Eq. corrector-RHS, the step lengths of Eq. stepsize-p / stepsize-d and
// the duality measure of Algorithm 5.  FP64; reductions are the deterministic
// last-block sums of common.cuh.
//
// vk[j] is the kind of variable j: kI (x_j >= 0), kF (free), kJ
// (0 <= x_j <= u_j).  Invariants kept by every kernel: z_j = 0 on F, and
// w_j = s_j = u_j = 0 outside J (the convention u_{I u F} = 0, z_F = 0,
// s_{I u F} = 0 of the section on free and box-constrained variables), so
// sums over all j equal the sums over the index sets the paper writes.
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

// Start of a (P~) solve, in place on the handle's copies: z_F = 0; on J,
// for a given start, the slack w = w0 (or u - x0) and s = s0 (the practical
// start writes w and s on J itself); elsewhere u = w = s = 0.
// out[0] = |I u J| + |J| (the divisor of mu), out[1] = ||u_J||^2,
// out[2] = number of invalid entries (kind outside {I, F, J}; on J a missing
// or non-finite u, and for a given start w <= 0, s <= 0 or s0 missing).
__global__ void __launch_bounds__(kNT) k_box_start(int n, const signed char* __restrict__ vk, double* __restrict__ u,
                                                   const double* __restrict__ x, double* __restrict__ z,
                                                   double* __restrict__ w, double* __restrict__ s, int has_u,
                                                   int has_w0, int has_s0, int given_start, double* out,
                                                   double* part, unsigned* cnt) {
  double v[3] = {0.0, 0.0, 0.0};
  for (int j = blockIdx.x * kNT + threadIdx.x; j < n; j += gridDim.x * kNT) {
    const signed char k = vk[j];
    if (k != kI && k != kF && k != kJ) {
      v[2] += 1.0;
      continue;
    }
    if (k == kF) z[j] = 0.0;
    if (k == kJ) {
      if (!has_u || (given_start && !has_s0)) {
        v[2] += 1.0;
        continue;
      }
      const double uj = u[j];
      if (!isfinite(uj)) v[2] += 1.0;
      if (given_start) {
        const double wj = has_w0 ? w[j] : uj - x[j];
        w[j] = wj;
        if (!(wj > 0.0) || !(s[j] > 0.0)) v[2] += 1.0;
      }
      v[1] = fma(uj, uj, v[1]);
    } else {
      u[j] = 0.0;
      w[j] = 0.0;
      s[j] = 0.0;
    }
    v[0] += (k != kF ? 1.0 : 0.0) + (k == kJ ? 1.0 : 0.0);
  }
  double tot[3];
  if (grid_sum<kNT, 3>(v, part, cnt, tot) && threadIdx.x == 0)
    for (int i = 0; i < 3; ++i) out[i] = tot[i];
}

// D_j = 1 / (q_j + Theta^{-1}_j + rho), Theta^{-1} = z/x on I, z/x + s/w on
// J, 0 on F (the diagonal left by eliminating dz, dw, ds from
// Eq. Newton-free-box).
__global__ void k_box_scaling(int n, const signed char* __restrict__ vk, const double* __restrict__ x,
                              const double* __restrict__ z, const double* __restrict__ w,
                              const double* __restrict__ s, const double* __restrict__ q, double rho,
                              double* __restrict__ D) {
  const int j = blockIdx.x * kNT + threadIdx.x;
  if (j >= n) return;
  const signed char k = vk[j];
  double ti = 0.0;
  if (k != kF) ti = z[j] / x[j];
  if (k == kJ) ti += s[j] / w[j];
  D[j] = 1.0 / (q[j] + ti + rho);
}

// n-part of the predictor right-hand sides (Eq. predictor-RHS):
//   rd_true = c + Q x - A^T y - z + s;  r_d = rd_true + rho (x - zeta);
//   r_u = u - x - w on J;  r_xz = -x z on I u J;  r_ws = -w s on J (0 elsewhere).
// out[0] = ||rd_true||^2, out[1] = x_IJ^T z_IJ + w_J^T s_J, out[2] = ||r_u||^2.
__global__ void __launch_bounds__(kNT) k_box_res_n(int n, const signed char* __restrict__ vk,
                                                   const double* __restrict__ c, const double* __restrict__ q,
                                                   const double* __restrict__ u, const double* __restrict__ x,
                                                   const double* __restrict__ z, const double* __restrict__ w,
                                                   const double* __restrict__ s, const double* __restrict__ Aty,
                                                   const double* __restrict__ zeta, double rho,
                                                   double* __restrict__ r_d, double* __restrict__ r_u,
                                                   double* __restrict__ r_xz, double* __restrict__ r_ws,
                                                   double* out, double* part, unsigned* cnt) {
  double v[3] = {0.0, 0.0, 0.0};
  for (int j = blockIdx.x * kNT + threadIdx.x; j < n; j += gridDim.x * kNT) {
    const signed char k = vk[j];
    const double xj = x[j], zj = z[j], wj = w[j], sj = s[j];
    const double rd = c[j] + q[j] * xj - Aty[j] - zj + sj;
    v[0] = fma(rd, rd, v[0]);
    r_d[j] = fma(rho, xj - zeta[j], rd);
    double ru = 0.0, rxz = 0.0, rws = 0.0;
    if (k != kF) {
      rxz = -xj * zj;
      v[1] = fma(xj, zj, v[1]);
    }
    if (k == kJ) {
      ru = u[j] - xj - wj;
      rws = -wj * sj;
      v[1] = fma(wj, sj, v[1]);
      v[2] = fma(ru, ru, v[2]);
    }
    r_u[j] = ru;
    r_xz[j] = rxz;
    r_ws[j] = rws;
  }
  double tot[3];
  if (grid_sum<kNT, 3>(v, part, cnt, tot) && threadIdx.x == 0)
    for (int i = 0; i < 3; ++i) out[i] = tot[i];
}

// xi_au of Algorithm 4: 0 on F, -r_xz/x on I, -r_xz/x + r_ws/w - s r_u/w on J.
__device__ __forceinline__ double xi_au(signed char k, double xj, double wj, double sj, double rxz, double rws,
                                        double ru) {
  double v = 0.0;
  if (k != kF) v = -rxz / xj;
  if (k == kJ) v += (rws - sj * ru) / wj;
  return v;
}

// t = D (r_d + xi_au)   (null r_d, r_u mean zero: the corrector)
__global__ void k_box_newton_rhs(int n, const signed char* __restrict__ vk, const double* __restrict__ D,
                                 const double* __restrict__ r_d, const double* __restrict__ r_u,
                                 const double* __restrict__ r_xz, const double* __restrict__ r_ws,
                                 const double* __restrict__ x, const double* __restrict__ w,
                                 const double* __restrict__ s, double* __restrict__ t) {
  const int j = blockIdx.x * kNT + threadIdx.x;
  if (j >= n) return;
  const double rd = r_d ? r_d[j] : 0.0, ru = r_u ? r_u[j] : 0.0;
  t[j] = D[j] * (rd + xi_au(vk[j], x[j], w[j], s[j], r_xz[j], r_ws[j], ru));
}

// dx = D (A^T dy - r_d - xi_au); dw = r_u - dx on J; dz = X^{-1}(r_xz - Z dx)
// on I u J; ds = W^{-1}(r_ws - S dw) on J; zero where a kind has no such
// variable.
__global__ void k_box_newton_back(int n, const signed char* __restrict__ vk, const double* __restrict__ D,
                                  const double* __restrict__ g, const double* __restrict__ r_d,
                                  const double* __restrict__ r_u, const double* __restrict__ r_xz,
                                  const double* __restrict__ r_ws, const double* __restrict__ x,
                                  const double* __restrict__ z, const double* __restrict__ w,
                                  const double* __restrict__ s, double* __restrict__ dx, double* __restrict__ dz,
                                  double* __restrict__ dw, double* __restrict__ ds) {
  const int j = blockIdx.x * kNT + threadIdx.x;
  if (j >= n) return;
  const signed char k = vk[j];
  const double rd = r_d ? r_d[j] : 0.0, ru = r_u ? r_u[j] : 0.0;
  const double xj = x[j], wj = w[j], sj = s[j], rxz = r_xz[j], rws = r_ws[j];
  const double dxj = D[j] * (g[j] - rd - xi_au(k, xj, wj, sj, rxz, rws, ru));
  dx[j] = dxj;
  double dzj = 0.0, dwj = 0.0, dsj = 0.0;
  if (k != kF) dzj = (rxz - z[j] * dxj) / xj;
  if (k == kJ) {
    dwj = ru - dxj;
    dsj = (rws - sj * dwj) / wj;
  }
  dz[j] = dzj;
  dw[j] = dwj;
  ds[j] = dsj;
}

// out[0] = min of -x/dx over I u J with dx < 0 and of -w/dw over J with
// dw < 0; out[1] likewise for (z, dz) and (s, ds)  (+inf when none).
__global__ void __launch_bounds__(kNT) k_box_step_ratios(int n, const signed char* __restrict__ vk,
                                                         const double* __restrict__ x, const double* __restrict__ dx,
                                                         const double* __restrict__ w, const double* __restrict__ dw,
                                                         const double* __restrict__ z, const double* __restrict__ dz,
                                                         const double* __restrict__ s, const double* __restrict__ ds,
                                                         double* out, double* part, unsigned* cnt) {
  double rp = INFINITY, rdual = INFINITY;
  for (int j = blockIdx.x * kNT + threadIdx.x; j < n; j += gridDim.x * kNT) {
    const signed char k = vk[j];
    if (k == kF) continue;
    const double a = dx[j], b = dz[j];
    if (a < 0.0) rp = fmin(rp, -x[j] / a);
    if (b < 0.0) rdual = fmin(rdual, -z[j] / b);
    if (k == kJ) {
      const double e = dw[j], f = ds[j];
      if (e < 0.0) rp = fmin(rp, -w[j] / e);
      if (f < 0.0) rdual = fmin(rdual, -s[j] / f);
    }
  }
  double o;
  if (grid_min<kNT>(rp, part, cnt, &o) && threadIdx.x == 0) out[0] = o;
  if (grid_min<kNT>(rdual, part + gridDim.x, cnt + 1, &o) && threadIdx.x == 0) out[1] = o;
}

// out = (x + ap dx)_IJ^T (z + ad dz)_IJ + (w + ap dw)_J^T (s + ad ds)_J
__global__ void __launch_bounds__(kNT) k_box_mu_aff(int n, const signed char* __restrict__ vk,
                                                    const double* __restrict__ x, const double* __restrict__ dx,
                                                    const double* __restrict__ z, const double* __restrict__ dz,
                                                    const double* __restrict__ w, const double* __restrict__ dw,
                                                    const double* __restrict__ s, const double* __restrict__ ds,
                                                    double ap, double ad, double* out, double* part,
                                                    unsigned* cnt) {
  double v[1] = {0.0};
  for (int j = blockIdx.x * kNT + threadIdx.x; j < n; j += gridDim.x * kNT) {
    const signed char k = vk[j];
    if (k != kF) v[0] = fma(fma(ap, dx[j], x[j]), fma(ad, dz[j], z[j]), v[0]);
    if (k == kJ) v[0] = fma(fma(ap, dw[j], w[j]), fma(ad, ds[j], s[j]), v[0]);
  }
  double tot[1];
  if (grid_sum<kNT, 1>(v, part, cnt, tot) && threadIdx.x == 0) out[0] = tot[0];
}

// Eq. corrector-RHS: r_xz = mu_t - dxp dzp on I u J, r_ws = mu_t - dwp dsp on J.
__global__ void k_box_corrector_rhs(int n, const signed char* __restrict__ vk, double mu_t,
                                    const double* __restrict__ dxp, const double* __restrict__ dzp,
                                    const double* __restrict__ dwp, const double* __restrict__ dsp,
                                    double* __restrict__ r_xz, double* __restrict__ r_ws) {
  const int j = blockIdx.x * kNT + threadIdx.x;
  if (j >= n) return;
  const signed char k = vk[j];
  r_xz[j] = k != kF ? mu_t - dxp[j] * dzp[j] : 0.0;
  r_ws[j] = k == kJ ? mu_t - dwp[j] * dsp[j] : 0.0;
}

}  // namespace

cudaError_t box_start_f64(cudaStream_t st, int n, const signed char* vk, double* u, const double* x, double* z,
                          double* w, double* s, int has_u, int has_w0, int has_s0, int given_start, double* out,
                          RedBuf red) {
  count_launches(1);
  k_box_start<<<grid_for(n), kNT, 0, st>>>(n, vk, u, x, z, w, s, has_u, has_w0, has_s0, given_start, out, red.part,
                                           red.cnt + 11);
  return cudaGetLastError();
}

cudaError_t box_scaling_f64(cudaStream_t st, int n, const signed char* vk, const double* x, const double* z,
                            const double* w, const double* s, const double* q, double rho, double* D) {
  count_launches(1);
  k_box_scaling<<<(n + kNT - 1) / kNT, kNT, 0, st>>>(n, vk, x, z, w, s, q, rho, D);
  return cudaGetLastError();
}

cudaError_t box_residuals_n_f64(cudaStream_t st, int n, const signed char* vk, const double* c, const double* q,
                                const double* u, const double* x, const double* z, const double* w,
                                const double* s, const double* Aty, const double* zeta, double rho, double* r_d,
                                double* r_u, double* r_xz, double* r_ws, double* out, RedBuf red) {
  count_launches(1);
  k_box_res_n<<<grid_for(n), kNT, 0, st>>>(n, vk, c, q, u, x, z, w, s, Aty, zeta, rho, r_d, r_u, r_xz, r_ws, out,
                                           red.part, red.cnt + 12);
  return cudaGetLastError();
}

cudaError_t box_newton_rhs_f64(cudaStream_t st, int n, const BoxVectors& bx, const double* D, const double* r_d,
                               const double* r_u, const double* r_xz, const double* r_ws, const double* x,
                               double* t) {
  count_launches(1);
  k_box_newton_rhs<<<(n + kNT - 1) / kNT, kNT, 0, st>>>(n, bx.vk, D, r_d, r_u, r_xz, r_ws, x, bx.w, bx.s, t);
  return cudaGetLastError();
}

cudaError_t box_newton_back_f64(cudaStream_t st, int n, const BoxVectors& bx, const double* D, const double* g,
                                const double* r_d, const double* r_u, const double* r_xz, const double* r_ws,
                                const double* x, const double* z, double* dx, double* dz, double* dw,
                                double* ds) {
  count_launches(1);
  k_box_newton_back<<<(n + kNT - 1) / kNT, kNT, 0, st>>>(n, bx.vk, D, g, r_d, r_u, r_xz, r_ws, x, z, bx.w, bx.s,
                                                         dx, dz, dw, ds);
  return cudaGetLastError();
}

cudaError_t box_step_ratios_f64(cudaStream_t st, int n, const signed char* vk, const double* x, const double* dx,
                                const double* w, const double* dw, const double* z, const double* dz,
                                const double* s, const double* ds, double* out, RedBuf red) {
  count_launches(1);
  k_box_step_ratios<<<grid_for(n), kNT, 0, st>>>(n, vk, x, dx, w, dw, z, dz, s, ds, out, red.part, red.cnt + 13);
  return cudaGetLastError();
}

cudaError_t box_mu_aff_f64(cudaStream_t st, int n, const signed char* vk, const double* x, const double* dx,
                           const double* z, const double* dz, const double* w, const double* dw, const double* s,
                           const double* ds, double ap, double ad, double* out, RedBuf red) {
  count_launches(1);
  k_box_mu_aff<<<grid_for(n), kNT, 0, st>>>(n, vk, x, dx, z, dz, w, dw, s, ds, ap, ad, out, red.part,
                                            red.cnt + 15);
  return cudaGetLastError();
}

cudaError_t box_corrector_rhs_f64(cudaStream_t st, int n, const signed char* vk, double mu_t, const double* dxp,
                                  const double* dzp, const double* dwp, const double* dsp, double* r_xz,
                                  double* r_ws) {
  count_launches(1);
  k_box_corrector_rhs<<<(n + kNT - 1) / kNT, kNT, 0, st>>>(n, vk, mu_t, dxp, dzp, dwp, dsp, r_xz, r_ws);
  return cudaGetLastError();
}

}  // namespace nys
