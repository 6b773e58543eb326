// Nystrom-preconditioned CG for (N + delta I) dy = xi (Section 2.2 with the
// preconditioner of Eq. Nys_precond_inv) in FP64.
//
//   P^{-1} r = r + U [ w .* (U^T r) ],  w_c = (lam_ell + delta) / (lam_c + delta) - 1
//
// is algebraically Eq. Nys_precond_inv ((lam_ell + delta) U (Lam + delta I)^{-1} U^T r
// + r - U U^T r) written with one pass over U for U^T r and one for U(.).
//
// All CG scalars live on the device; every kernel of an iteration is
// predicated on the device flag SI_DONE, so the host issues iterations
// without reading anything back until it polls the flag.
#include "common.cuh"
#include "internal.h"

namespace nys {

namespace {

// Rows handled by one block in the kernels that touch U (m x ell):
// small bands spread the ell*m DFMAs over many SMs.
int band_rows(int m) {
  int r = (m + 2 * 152 - 1) / (2 * 152);
  r = (r + 63) / 64 * 64;
  return r < 64 ? 64 : r;
}

// Block-level partials of U^T r (ell values) and of extra sums, then the last
// block reduces over blocks in a fixed order.  part layout: [block][ell + kx].
template <int KX>
__device__ bool band_reduce(int m, int ell, const double* __restrict__ U, int ld,
                            const double* __restrict__ r, int i0, int i1, double (&xs)[KX],
                            double* part, unsigned* cnt, double* s_out, double (&x_out)[KX]) {
  __shared__ double sh[KX * kWarps];
  __shared__ double tot[KX];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int stride = ell + KX;
  double* mine = part + (size_t)blockIdx.x * stride;
  for (int c = wid; c < ell; c += kWarps) {
    const double* u = U + (size_t)c * ld;
    double acc = 0.0;
    for (int i = i0 + lane; i < i1; i += 32) acc = fma(u[i], r[i], acc);
    acc = warp_sum(acc);
    if (lane == 0) mine[c] = acc;
  }
  __threadfence();
  block_sum<kNT, KX>(xs, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < KX; ++k) mine[ell + k] = xs[k];
    __threadfence();
    const unsigned t = atomicAdd(cnt, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  for (int e = threadIdx.x; e < stride; e += kNT) {
    double acc = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) acc += __ldcg(part + (size_t)b * stride + e);
    if (e < ell) s_out[e] = acc;
    else tot[e - ell] = acc;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < KX; ++k) x_out[k] = tot[k];
  if (threadIdx.x == 0) *cnt = 0u;
  return true;
}

// Setup (1): r = xi, x = 0, ||xi||^2, s = U^T xi, weights, flags.
__global__ void __launch_bounds__(kNT) k_pcg_setup1(int m, int ell, const double* __restrict__ U,
                                                    int ld, const double* __restrict__ lam, double delta,
                                                    const double* __restrict__ xi, double eta2,
                                                    int max_iter, int forced, double* __restrict__ x,
                                                    double* __restrict__ r, double* __restrict__ s,
                                                    double* __restrict__ wts, double* sd, int* si,
                                                    double* part, unsigned* cnt, int rows) {
  const int i0 = blockIdx.x * rows, i1 = min(m, i0 + rows);
  double xs[1] = {0.0};
  for (int i = i0 + threadIdx.x; i < i1; i += kNT) {
    const double v = xi[i];
    r[i] = v;
    x[i] = 0.0;
    xs[0] = fma(v, v, xs[0]);
  }
  __syncthreads();
  double tot[1];
  if (band_reduce<1>(m, ell, U, ld, xi, i0, i1, xs, part, cnt, s, tot)) {
    if (threadIdx.x == 0) {
      sd[SD_BNORM2] = tot[0];
      sd[SD_RR] = tot[0];
      sd[SD_ETA2] = eta2;
      si[SI_ITERS] = 0;
      si[SI_FORCED] = forced;
      si[SI_MAXIT] = max_iter;
      sd[SD_DELTA] = delta;
      const int limit = forced >= 0 ? forced : max_iter;
      si[SI_DONE] = (tot[0] == 0.0 || limit <= 0) ? 1 : 0;
      if (!isfinite(tot[0])) { si[SI_DONE] = 1; set_error(si + SI_ERR, kErrNumeric); }
    }
    const double lam_ell = ell > 0 ? lam[ell - 1] : 0.0;
    for (int c = threadIdx.x; c < ell; c += kNT) wts[c] = (lam_ell + delta) / (lam[c] + delta) - 1.0;
  }
}

// z = r + U (wts .* s);  rz = r^T z.  mode 0: setup (rz <- total),
// mode 1: iteration (beta = total / rz, rz <- total), mode 2: plain apply.
__global__ void __launch_bounds__(kNT) k_pcg_precond(int m, int ell, const double* __restrict__ U,
                                                     int ld, const double* __restrict__ r,
                                                     const double* __restrict__ s,
                                                     const double* __restrict__ wts,
                                                     double* __restrict__ z, double* sd, int* si,
                                                     double* part, unsigned* cnt, int mode) {
  if (mode == 1 && si[SI_DONE]) return;
  __shared__ double ws[1024];
  for (int c = threadIdx.x; c < ell && c < 1024; c += kNT) ws[c] = wts[c] * s[c];
  __syncthreads();
  double v[1] = {0.0};
  for (int i = blockIdx.x * kNT + threadIdx.x; i < m; i += gridDim.x * kNT) {
    double acc = 0.0;
    for (int c = 0; c < ell; ++c) {
      const double wc = c < 1024 ? ws[c] : wts[c] * s[c];
      acc = fma(U[(size_t)c * ld + i], wc, acc);
    }
    const double zi = r[i] + acc;
    z[i] = zi;
    v[0] = fma(r[i], zi, v[0]);
  }
  if (mode == 2) return;
  double out[1];
  if (grid_sum<kNT, 1>(v, part, cnt, out) && threadIdx.x == 0) {
    const double rz = out[0];
    if (!(rz > 0.0) || !isfinite(rz)) {
      // r^T P^{-1} r must be positive for r != 0; stop the solve otherwise
      if (rz != 0.0) set_error(si + SI_ERR, kErrNumeric);
      si[SI_DONE] = 1;
    }
    if (mode == 1) sd[SD_BETA] = rz / sd[SD_RZ];
    sd[SD_RZ] = rz;
  }
}

__global__ void k_pcg_p(int m, const double* __restrict__ z, double* __restrict__ p, const double* sd,
                        const int* si, int first) {
  if (!first && si[SI_DONE]) return;
  const int i = blockIdx.x * kNT + threadIdx.x;
  if (i >= m) return;
  p[i] = first ? z[i] : fma(sd[SD_BETA], p[i], z[i]);
}

// pw = p^T w;  alpha = rz / pw
__global__ void __launch_bounds__(kNT) k_pcg_alpha(int m, const double* __restrict__ p,
                                                   const double* __restrict__ w, double* sd, int* si,
                                                   double* part, unsigned* cnt) {
  if (si[SI_DONE]) return;
  double v[1] = {0.0};
  for (int i = blockIdx.x * kNT + threadIdx.x; i < m; i += gridDim.x * kNT) v[0] = fma(p[i], w[i], v[0]);
  double out[1];
  if (grid_sum<kNT, 1>(v, part, cnt, out) && threadIdx.x == 0) {
    const double pw = out[0];
    if (!(pw > 0.0) || !isfinite(pw)) {
      set_error(si + SI_ERR, kErrNumeric);
      si[SI_DONE] = 1;
      sd[SD_ALPHA] = 0.0;
    } else {
      sd[SD_ALPHA] = sd[SD_RZ] / pw;
    }
  }
}

// x += alpha p; r -= alpha w; ||r||^2 and s = U^T r; iteration count and stop test.
__global__ void __launch_bounds__(kNT) k_pcg_update(int m, int ell, const double* __restrict__ U, int ld,
                                                    const double* __restrict__ p,
                                                    const double* __restrict__ w, double* __restrict__ x,
                                                    double* __restrict__ r, double* __restrict__ s,
                                                    double* sd, int* si, double* part, unsigned* cnt,
                                                    int rows) {
  if (si[SI_DONE]) return;
  const double alpha = sd[SD_ALPHA];
  const int i0 = blockIdx.x * rows, i1 = min(m, i0 + rows);
  double xs[1] = {0.0};
  for (int i = i0 + threadIdx.x; i < i1; i += kNT) {
    x[i] = fma(alpha, p[i], x[i]);
    const double ri = fma(-alpha, w[i], r[i]);
    r[i] = ri;
    xs[0] = fma(ri, ri, xs[0]);
  }
  __syncthreads();
  double tot[1];
  if (band_reduce<1>(m, ell, U, ld, r, i0, i1, xs, part, cnt, s, tot) && threadIdx.x == 0) {
    const double rr = tot[0];
    sd[SD_RR] = rr;
    const int it = si[SI_ITERS] + 1;
    si[SI_ITERS] = it;
    const int forced = si[SI_FORCED];
    if (forced >= 0) {
      if (it >= forced) si[SI_DONE] = 1;
    } else if (rr <= sd[SD_ETA2] * sd[SD_BNORM2] || it >= si[SI_MAXIT]) {
      si[SI_DONE] = 1;
    }
    if (!isfinite(rr)) { set_error(si + SI_ERR, kErrNumeric); si[SI_DONE] = 1; }
  }
}

__global__ void __launch_bounds__(kNT) k_ut_r(int m, int ell, const double* __restrict__ U, int ld,
                                              const double* __restrict__ lam, double delta,
                                              const double* __restrict__ r, double* __restrict__ s,
                                              double* __restrict__ wts, double* part, unsigned* cnt,
                                              int rows) {
  const int i0 = blockIdx.x * rows, i1 = min(m, i0 + rows);
  double xs[1] = {0.0};
  double tot[1];
  if (band_reduce<1>(m, ell, U, ld, r, i0, i1, xs, part, cnt, s, tot)) {
    const double lam_ell = lam[ell - 1];
    for (int c = threadIdx.x; c < ell; c += kNT) wts[c] = (lam_ell + delta) / (lam[c] + delta) - 1.0;
  }
}

__global__ void k_pcg_cond(cudaGraphConditionalHandle cond, const int* si) {
  cudaGraphSetConditional(cond, si[SI_DONE] ? 0u : 1u);
}

int vec_blocks(int m) {
  int b = (m + kNT - 1) / kNT;
  return b > 2 * 152 ? 2 * 152 : (b < 1 ? 1 : b);
}

}  // namespace

cudaError_t pcg_loop_condition(cudaStream_t st, cudaGraphConditionalHandle cond, const int* si) {
  count_launches(1);
  k_pcg_cond<<<1, 1, 0, st>>>(cond, si);
  return cudaGetLastError();
}

cudaError_t precond_apply_f64(cudaStream_t st, int m, int ell, const double* U, int ld,
                              const double* lam, double delta, const double* r, double* out,
                              double* s, double* wts, RedBuf red) {
  const int rows = band_rows(m);
  const int nb = (m + rows - 1) / rows;
  count_launches(1);
  k_ut_r<<<nb, kNT, 0, st>>>(m, ell, U, ld, lam, delta, r, s, wts, red.part, red.cnt + 1, rows);
  count_launches(1);
  k_pcg_precond<<<vec_blocks(m), kNT, 0, st>>>(m, ell, U, ld, r, s, wts, out, nullptr, nullptr,
                                               red.part, red.cnt + 2, 2);
  return cudaGetLastError();
}

cudaError_t pcg_setup_f64(cudaStream_t st, int m, int ell, const double* U, int ld,
                          const double* lam, double delta, const double* xi, double eta,
                          int max_iter, int forced, PcgWork w, double* sd, int* si, RedBuf red) {
  const int rows = band_rows(m);
  const int nb = (m + rows - 1) / rows;
  count_launches(1);
  k_pcg_setup1<<<nb, kNT, 0, st>>>(m, ell, U, ld, lam, delta, xi, eta * eta, max_iter, forced,
                                   w.x, w.r, w.s, w.wts, sd, si, red.part, red.cnt + 1, rows);
  count_launches(1);
  k_pcg_precond<<<vec_blocks(m), kNT, 0, st>>>(m, ell, U, ld, w.r, w.s, w.wts, w.z, sd, si,
                                               red.part, red.cnt + 2, 0);
  count_launches(1);
  k_pcg_p<<<(m + kNT - 1) / kNT, kNT, 0, st>>>(m, w.z, w.p, sd, si, 1);
  return cudaGetLastError();
}

// CG vector updates of one iteration after w = (N + delta I) p is available.
static cudaError_t pcg_tail(cudaStream_t st, int m, int ell, const double* U, int ld, PcgWork w,
                            double* sd, int* si, RedBuf red) {
  count_launches(1);
  k_pcg_alpha<<<vec_blocks(m), kNT, 0, st>>>(m, w.p, w.w, sd, si, red.part, red.cnt + 3);
  const int rows = band_rows(m);
  const int nb = (m + rows - 1) / rows;
  count_launches(1);
  k_pcg_update<<<nb, kNT, 0, st>>>(m, ell, U, ld, w.p, w.w, w.x, w.r, w.s, sd, si, red.part,
                                   red.cnt + 1, rows);
  count_launches(1);
  k_pcg_precond<<<vec_blocks(m), kNT, 0, st>>>(m, ell, U, ld, w.r, w.s, w.wts, w.z, sd, si,
                                               red.part, red.cnt + 2, 1);
  count_launches(1);
  k_pcg_p<<<(m + kNT - 1) / kNT, kNT, 0, st>>>(m, w.z, w.p, sd, si, 0);
  return cudaGetLastError();
}

cudaError_t pcg_iteration_f64(cudaStream_t st, int m, int n, const double* A, long long lda,
                              const double* D, int ell, const double* U, int ld,
                              PcgWork w, double* sd, int* si, RedBuf red) {
  const int* done = si + SI_DONE;
  cudaError_t e = gemv_t_f64(st, m, n, A, lda, w.p, D, w.t, w.split_buf, w.split_cap, done);
  if (e != cudaSuccess) return e;
  e = gemv_n_f64(st, m, n, A, lda, w.t, 1.0, w.p, w.w, done, sd + SD_DELTA, w.split_buf, w.split_cap);
  if (e != cudaSuccess) return e;
  return pcg_tail(st, m, ell, U, ld, w, sd, si, red);
}

cudaError_t pcg_iteration_lp(cudaStream_t st, int m, int n, const LpOperator& op, int ell,
                             const double* U, int ld, PcgWork w, double* sd, int* si, RedBuf red) {
  const int* done = si + SI_DONE;
  if (op.ff) {
    // float-float: t = D .* (A^T p) in FP64, w = A t + delta p
    cudaError_t e = split_ff(st, m, op.ld_mpad, w.p, nullptr, op.xh, op.xl, done);
    if (e != cudaSuccess) return e;
    e = gemv_rows_ff(st, n, m, static_cast<const float*>(op.AT), op.ldat, op.xh, op.xl, op.D64, 0.0, nullptr,
                     op.t64, done, nullptr, op.part, op.part_cap);
    if (e != cudaSuccess) return e;
    e = split_ff(st, n, op.ld_npad, op.t64, nullptr, op.xh, op.xl, done);
    if (e != cudaSuccess) return e;
    e = gemv_rows_ff(st, m, n, static_cast<const float*>(op.A), op.lda, op.xh, op.xl, nullptr, 1.0, w.p, w.w, done,
                     sd + SD_DELTA, op.part, op.part_cap);
    if (e != cudaSuccess) return e;
    return pcg_tail(st, m, ell, U, ld, w, sd, si, red);
  }
  // pf = FP32(s .* p);  tf = Df .* (Q^T pf);  w = s .* (Q tf) + delta p, with
  // s the per-row scales of FP8 storage (A = diag(s) Q) and s = 1 otherwise
  cudaError_t e = to_f32(st, m, op.ld_mpad, w.p, op.rs64, op.xf, done);
  if (e != cudaSuccess) return e;
  e = gemv_rows_lp(st, n, m, op.a_type, op.AT, op.ldat, op.xf, op.Df, 0.0, nullptr, op.tf, 0, done, nullptr, op.part,
                   op.part_cap);
  if (e != cudaSuccess) return e;
  e = gemv_rows_lp(st, m, n, op.a_type, op.A, op.lda, op.tf, op.rs32, 1.0, w.p, w.w, 1, done, sd + SD_DELTA, op.part,
                   op.part_cap);
  if (e != cudaSuccess) return e;
  return pcg_tail(st, m, ell, U, ld, w, sd, si, red);
}

}  // namespace nys
