// Vector kernels of the IP-PMM iteration (Algorithms 4 and 5 with I = all,
// step lengths of Eq. stepsize-p / stepsize-d), FP64.  Reductions are the
// deterministic last-block sums of common.cuh.
#include "common.cuh"
#include "internal.h"

namespace nys {

namespace {

int grid_for(long long len) {
  long long b = (len + kNT - 1) / kNT;
  if (b > 2 * 152) b = 2 * 152;
  return b < 1 ? 1 : (int)b;
}

// n-part of the residuals: rd_true, r_d (predictor), r_xz; sums ||rd_true||^2, x^T z
__global__ void __launch_bounds__(kNT) k_res_n(int n, const double* __restrict__ c, const double* __restrict__ q,
                                               const double* __restrict__ x, const double* __restrict__ z,
                                               const double* __restrict__ Aty, const double* __restrict__ zeta,
                                               double rho, double* __restrict__ r_d, double* __restrict__ r_xz,
                                               double* out, double* part, unsigned* cnt) {
  double v[2] = {0.0, 0.0};
  for (int j = blockIdx.x * kNT + threadIdx.x; j < n; j += gridDim.x * kNT) {
    const double xj = x[j], zj = z[j];
    const double rd = c[j] + q[j] * xj - Aty[j] - zj;
    v[0] = fma(rd, rd, v[0]);
    v[1] = fma(xj, zj, v[1]);
    r_d[j] = fma(rho, xj - zeta[j], rd);
    r_xz[j] = -xj * zj;
  }
  double tot[2];
  if (grid_sum<kNT, 2>(v, part, cnt, tot) && threadIdx.x == 0) { out[0] = tot[0]; out[1] = tot[1]; }
}

// m-part: rp_true = b - Ax, r_p = rp_true - delta (y - lam); sum ||rp_true||^2
__global__ void __launch_bounds__(kNT) k_res_m(int m, const double* __restrict__ b, const double* __restrict__ Ax,
                                               const double* __restrict__ y, const double* __restrict__ lam,
                                               double delta, double* __restrict__ r_p, double* out,
                                               double* part, unsigned* cnt) {
  double v[1] = {0.0};
  for (int i = blockIdx.x * kNT + threadIdx.x; i < m; i += gridDim.x * kNT) {
    const double rp = b[i] - Ax[i];
    v[0] = fma(rp, rp, v[0]);
    r_p[i] = fma(-delta, y[i] - lam[i], rp);
  }
  double tot[1];
  if (grid_sum<kNT, 1>(v, part, cnt, tot) && threadIdx.x == 0) out[0] = tot[0];
}

__global__ void k_newton_rhs(int n, const double* __restrict__ D, const double* __restrict__ r_d,
                             const double* __restrict__ r_xz, const double* __restrict__ x,
                             double* __restrict__ t) {
  const int j = blockIdx.x * kNT + threadIdx.x;
  if (j >= n) return;
  // xi_au = -r_xz / x;  t = D (r_d + xi_au)
  const double rd = r_d ? r_d[j] : 0.0;
  t[j] = D[j] * (rd - r_xz[j] / x[j]);
}

__global__ void k_newton_back(int n, const double* __restrict__ D, const double* __restrict__ g,
                              const double* __restrict__ r_d, const double* __restrict__ r_xz,
                              const double* __restrict__ x, const double* __restrict__ z,
                              double* __restrict__ dx, double* __restrict__ dz) {
  const int j = blockIdx.x * kNT + threadIdx.x;
  if (j >= n) return;
  const double rd = r_d ? r_d[j] : 0.0;
  const double xj = x[j], rxz = r_xz[j];
  // dx = D (A^T dy - r_d - xi_au),  xi_au = -r_xz / x
  const double dxj = D[j] * (g[j] - rd + rxz / xj);
  dx[j] = dxj;
  // dz = X^{-1} (r_xz - Z dx)
  dz[j] = (rxz - z[j] * dxj) / xj;
}

__global__ void __launch_bounds__(kNT) k_step_ratios(int n, const double* __restrict__ x,
                                                     const double* __restrict__ dx,
                                                     const double* __restrict__ z,
                                                     const double* __restrict__ dz, double* out,
                                                     double* part, unsigned* cnt) {
  double rx = INFINITY, rz = INFINITY;
  for (int j = blockIdx.x * kNT + threadIdx.x; j < n; j += gridDim.x * kNT) {
    const double a = dx[j], b = dz[j];
    if (a < 0.0) rx = fmin(rx, -x[j] / a);
    if (b < 0.0) rz = fmin(rz, -z[j] / b);
  }
  // two independent min reductions sharing the partial buffer halves
  double o;
  if (grid_min<kNT>(rx, part, cnt, &o) && threadIdx.x == 0) out[0] = o;
  if (grid_min<kNT>(rz, part + gridDim.x, cnt + 1, &o) && threadIdx.x == 0) out[1] = o;
}

__global__ void __launch_bounds__(kNT) k_mu_aff(int n, const double* __restrict__ x, const double* __restrict__ dx,
                                                const double* __restrict__ z, const double* __restrict__ dz,
                                                double ap, double ad, double* out, double* part, unsigned* cnt) {
  double v[1] = {0.0};
  for (int j = blockIdx.x * kNT + threadIdx.x; j < n; j += gridDim.x * kNT)
    v[0] = fma(fma(ap, dx[j], x[j]), fma(ad, dz[j], z[j]), v[0]);
  double tot[1];
  if (grid_sum<kNT, 1>(v, part, cnt, tot) && threadIdx.x == 0) out[0] = tot[0];
}

__global__ void k_corrector_rhs(int n, double mu_t, const double* __restrict__ dxp,
                                const double* __restrict__ dzp, double* __restrict__ r_xz) {
  const int j = blockIdx.x * kNT + threadIdx.x;
  if (j < n) r_xz[j] = mu_t - dxp[j] * dzp[j];
}

__global__ void k_add_dirs(int m, int n, const double* __restrict__ dxp, const double* __restrict__ dyp,
                           const double* __restrict__ dzp, double* __restrict__ dx, double* __restrict__ dy,
                           double* __restrict__ dz) {
  const int j = blockIdx.x * kNT + threadIdx.x;
  if (j < n) {
    dx[j] += dxp[j];
    dz[j] += dzp[j];
  }
  if (j < m) dy[j] += dyp[j];
}

__global__ void k_update(int m, int n, double ap, double ad, const double* __restrict__ dx,
                         const double* __restrict__ dy, const double* __restrict__ dz,
                         double* __restrict__ x, double* __restrict__ y, double* __restrict__ z) {
  const int j = blockIdx.x * kNT + threadIdx.x;
  if (j < n) {
    x[j] = fma(ap, dx[j], x[j]);
    z[j] = fma(ad, dz[j], z[j]);
  }
  if (j < m) y[j] = fma(ad, dy[j], y[j]);
}

__global__ void __launch_bounds__(kNT) k_dot(int len, const double* __restrict__ a, const double* __restrict__ b,
                                             double* out, double* part, unsigned* cnt) {
  double v[1] = {0.0};
  for (int j = blockIdx.x * kNT + threadIdx.x; j < len; j += gridDim.x * kNT) v[0] = fma(a[j], b[j], v[0]);
  double tot[1];
  if (grid_sum<kNT, 1>(v, part, cnt, tot) && threadIdx.x == 0) out[0] = tot[0];
}

__global__ void __launch_bounds__(kNT) k_objective(int m, int n, const double* __restrict__ q,
                                                   const double* __restrict__ c, const double* __restrict__ b,
                                                   const double* __restrict__ x, const double* __restrict__ y,
                                                   const double* __restrict__ z, double* out, double* part,
                                                   unsigned* cnt) {
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  const int len = n > m ? n : m;
  for (int j = blockIdx.x * kNT + threadIdx.x; j < len; j += gridDim.x * kNT) {
    if (j < n) {
      const double xj = x[j];
      v[0] = fma(xj, q[j] * xj, v[0]);
      v[1] = fma(c[j], xj, v[1]);
      if (!isfinite(xj) || !isfinite(z[j])) v[3] += 1.0;
    }
    if (j < m) {
      v[2] = fma(b[j], y[j], v[2]);
      if (!isfinite(y[j])) v[3] += 1.0;
    }
  }
  double tot[4];
  if (grid_sum<kNT, 4>(v, part, cnt, tot) && threadIdx.x == 0)
    for (int k = 0; k < 4; ++k) out[k] = tot[k];
}

// out = a x + b y
__global__ void k_axpby(int len, double a, const double* __restrict__ x, double b, const double* __restrict__ y,
                        double* __restrict__ out) {
  const int j = blockIdx.x * kNT + threadIdx.x;
  if (j < len) out[j] = fma(a, x[j], b * y[j]);
}

// Round a column-major FP64 panel to BF16 (rows of the transposed BF16 copy)
// and write the rounded values back, so both views hold the same numbers.
__global__ void k_round_panel_bf16(int m, int ell, double* __restrict__ P, int ld, __nv_bfloat16* __restrict__ Pb,
                                   int ldb) {
  const long long idx = (long long)blockIdx.x * kNT + threadIdx.x;
  if (idx >= (long long)m * ell) return;
  const int i = (int)(idx % m), c = (int)(idx / m);
  const __nv_bfloat16 v = __float2bfloat16_rn((float)P[(size_t)c * ld + i]);
  Pb[(size_t)c * ldb + i] = v;
  P[(size_t)c * ld + i] = (double)__bfloat162float(v);
}

__global__ void k_panel_f32_to_f64(int m, int ell, const float* __restrict__ src, int lds, double* __restrict__ dst,
                                   int ldd) {
  const long long idx = (long long)blockIdx.x * kNT + threadIdx.x;
  if (idx >= (long long)m * ell) return;
  const int i = (int)(idx % m), c = (int)(idx / m);
  dst[(size_t)c * ldd + i] = (double)src[(size_t)c * lds + i];
}

__global__ void k_vmul(int len, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ out) {
  const int j = blockIdx.x * kNT + threadIdx.x;
  if (j < len) out[j] = a[j] * b[j];
}

// out[i, j] = alpha u_i v_j + beta w_i s_j  (row-major m x n, leading dimension ldo)
template <typename TO>
__global__ void k_rank2(int m, int n, double alpha, const double* __restrict__ u, const double* __restrict__ v,
                        double beta, const double* __restrict__ w, const double* __restrict__ s, TO* __restrict__ out,
                        long long ldo) {
  const int i = blockIdx.y;
  const double ui = alpha * u[i], wi = beta * w[i];
  TO* row = out + (long long)i * ldo;
  for (int j = blockIdx.x * kNT + threadIdx.x; j < n; j += gridDim.x * kNT) row[j] = (TO)fma(ui, v[j], wi * s[j]);
}

}  // namespace

cudaError_t vmul_f64(cudaStream_t st, int len, const double* a, const double* b, double* out) {
  if (len <= 0) return cudaSuccess;
  count_launches(1);
  k_vmul<<<(len + kNT - 1) / kNT, kNT, 0, st>>>(len, a, b, out);
  return cudaGetLastError();
}

cudaError_t rank2_update(cudaStream_t st, int m, int n, double alpha, const double* u, const double* v, double beta,
                         const double* w, const double* s, void* out, long long ldo, int out_f32) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  int gx = (n + kNT - 1) / kNT;
  if (gx > 8) gx = 8;
  dim3 grid(gx, m);
  count_launches(1);
  if (out_f32) k_rank2<float><<<grid, kNT, 0, st>>>(m, n, alpha, u, v, beta, w, s, (float*)out, ldo);
  else k_rank2<double><<<grid, kNT, 0, st>>>(m, n, alpha, u, v, beta, w, s, (double*)out, ldo);
  return cudaGetLastError();
}

cudaError_t axpby_f64(cudaStream_t st, int len, double a, const double* x, double b, const double* y, double* out) {
  if (len <= 0) return cudaSuccess;
  count_launches(1);
  k_axpby<<<(len + kNT - 1) / kNT, kNT, 0, st>>>(len, a, x, b, y, out);
  return cudaGetLastError();
}

cudaError_t round_panel_bf16(cudaStream_t st, int m, int ell, double* P, int ld, __nv_bfloat16* Pb, int ldb) {
  const long long total = (long long)m * ell;
  count_launches(1);
  k_round_panel_bf16<<<(unsigned)((total + kNT - 1) / kNT), kNT, 0, st>>>(m, ell, P, ld, Pb, ldb);
  return cudaGetLastError();
}

cudaError_t panel_f32_to_f64(cudaStream_t st, int m, int ell, const float* src, int lds, double* dst, int ldd) {
  const long long total = (long long)m * ell;
  count_launches(1);
  k_panel_f32_to_f64<<<(unsigned)((total + kNT - 1) / kNT), kNT, 0, st>>>(m, ell, src, lds, dst, ldd);
  return cudaGetLastError();
}

cudaError_t ipm_residuals_f64(cudaStream_t st, int m, int n, const double* b, const double* c,
                              const double* q, const double* x, const double* y,
                              const double* z, const double* Ax, const double* Aty,
                              const double* lam, const double* zeta, double rho, double delta,
                              double* r_d, double* r_p, double* r_xz, double* red_out,
                              RedBuf red) {
  count_launches(1);
  k_res_n<<<grid_for(n), kNT, 0, st>>>(n, c, q, x, z, Aty, zeta, rho, r_d, r_xz, red_out, red.part,
                                       red.cnt + 4);
  count_launches(1);
  k_res_m<<<grid_for(m), kNT, 0, st>>>(m, b, Ax, y, lam, delta, r_p, red_out + 2,
                                       red.part + 4 * 2 * 152, red.cnt + 5);
  return cudaGetLastError();
}

cudaError_t ipm_residuals_m_f64(cudaStream_t st, int m, const double* b, const double* Ax, const double* y,
                                const double* lam, double delta, double* r_p, double* red_out, RedBuf red) {
  count_launches(1);
  k_res_m<<<grid_for(m), kNT, 0, st>>>(m, b, Ax, y, lam, delta, r_p, red_out, red.part + 4 * 2 * 152,
                                       red.cnt + 5);
  return cudaGetLastError();
}

cudaError_t newton_rhs_f64(cudaStream_t st, int n, const double* D, const double* r_d,
                           const double* r_xz, const double* x, double* t) {
  count_launches(1);
  k_newton_rhs<<<(n + kNT - 1) / kNT, kNT, 0, st>>>(n, D, r_d, r_xz, x, t);
  return cudaGetLastError();
}

cudaError_t newton_back_f64(cudaStream_t st, int n, const double* D, const double* g,
                            const double* r_d, const double* r_xz, const double* x,
                            const double* z, double* dx, double* dz) {
  count_launches(1);
  k_newton_back<<<(n + kNT - 1) / kNT, kNT, 0, st>>>(n, D, g, r_d, r_xz, x, z, dx, dz);
  return cudaGetLastError();
}

cudaError_t step_ratios_f64(cudaStream_t st, int n, const double* x, const double* dx,
                            const double* z, const double* dz, double* out, RedBuf red) {
  count_launches(1);
  k_step_ratios<<<grid_for(n), kNT, 0, st>>>(n, x, dx, z, dz, out, red.part, red.cnt + 6);
  return cudaGetLastError();
}

cudaError_t mu_aff_f64(cudaStream_t st, int n, const double* x, const double* dx,
                       const double* z, const double* dz, double ap, double ad, double* out,
                       RedBuf red) {
  count_launches(1);
  k_mu_aff<<<grid_for(n), kNT, 0, st>>>(n, x, dx, z, dz, ap, ad, out, red.part, red.cnt + 8);
  return cudaGetLastError();
}

cudaError_t corrector_rhs_f64(cudaStream_t st, int n, double mu_t, const double* dxp,
                              const double* dzp, double* r_xz) {
  count_launches(1);
  k_corrector_rhs<<<(n + kNT - 1) / kNT, kNT, 0, st>>>(n, mu_t, dxp, dzp, r_xz);
  return cudaGetLastError();
}

cudaError_t add_dirs_f64(cudaStream_t st, int m, int n, const double* dxp, const double* dyp,
                         const double* dzp, double* dx, double* dy, double* dz) {
  const int len = n > m ? n : m;
  count_launches(1);
  k_add_dirs<<<(len + kNT - 1) / kNT, kNT, 0, st>>>(m, n, dxp, dyp, dzp, dx, dy, dz);
  return cudaGetLastError();
}

cudaError_t ipm_update_f64(cudaStream_t st, int m, int n, double ap, double ad, const double* dx,
                           const double* dy, const double* dz, double* x, double* y, double* z) {
  const int len = n > m ? n : m;
  count_launches(1);
  k_update<<<(len + kNT - 1) / kNT, kNT, 0, st>>>(m, n, ap, ad, dx, dy, dz, x, y, z);
  return cudaGetLastError();
}

cudaError_t dot_f64(cudaStream_t st, int len, const double* a, const double* b, double* out,
                    RedBuf red) {
  count_launches(1);
  k_dot<<<grid_for(len), kNT, 0, st>>>(len, a, b, out, red.part, red.cnt + 10);
  return cudaGetLastError();
}

cudaError_t objective_terms_f64(cudaStream_t st, int m, int n, const double* q, const double* c,
                                const double* b, const double* x, const double* y,
                                const double* z, double* out, RedBuf red) {
  const int len = n > m ? n : m;
  count_launches(1);
  k_objective<<<grid_for(len), kNT, 0, st>>>(m, n, q, c, b, x, y, z, out, red.part, red.cnt + 9);
  return cudaGetLastError();
}

}  // namespace nys
