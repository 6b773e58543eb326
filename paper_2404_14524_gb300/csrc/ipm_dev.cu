// Device-resident IP-PMM iteration for problems (P) in the FP64 form.
//
// The host path (IpmRun in solver.cu) reads six scalars back per IPM
// iteration to decide what to launch next: the residual norms (termination
// and the PMM update of Algorithm 6), the step lengths of Eq. stepsize-p/-d
// (twice), mu_aff of Algorithm 5, and each PCG solve's count.  Here one-thread
// kernels compute those decisions into an IpmDev block in device memory and
// the vector kernels read their scalars from it, so a whole solve is one CUDA
// graph: the first iteration's top, then a conditional while node around
// "Newton steps of iteration k + top of iteration k+1".  The arithmetic and
// its order are those of the host path and of the oracle (products that the
// host does not fuse are written with explicit rounding here).
#include "common.cuh"
#include "internal.h"

namespace nys {

namespace {

int grid_for(long long len) {
  long long b = (len + kNT - 1) / kNT;
  if (b > 2 * 152) b = 2 * 152;
  return b < 1 ? 1 : (int)b;
}

// n-part of the residuals (as k_res_n) with rho and zeta from the device block
__global__ void __launch_bounds__(kNT) k_res_n_dev(int n, const double* __restrict__ c, const double* __restrict__ q,
                                                   const double* __restrict__ x, const double* __restrict__ z,
                                                   const double* __restrict__ Aty, const double* __restrict__ zeta,
                                                   const IpmDev* __restrict__ s, double* __restrict__ r_d,
                                                   double* __restrict__ r_xz, double* out, double* part,
                                                   unsigned* cnt) {
  const double rho = s->rho;
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

// m-part (as k_res_m) with delta and lambda from the device block
__global__ void __launch_bounds__(kNT) k_res_m_dev(int m, const double* __restrict__ b, const double* __restrict__ Ax,
                                                   const double* __restrict__ y, const double* __restrict__ lam,
                                                   const IpmDev* __restrict__ s, double* __restrict__ r_p,
                                                   double* out, double* part, unsigned* cnt) {
  const double delta = s->delta;
  double v[1] = {0.0};
  for (int i = blockIdx.x * kNT + threadIdx.x; i < m; i += gridDim.x * kNT) {
    const double rp = b[i] - Ax[i];
    v[0] = fma(rp, rp, v[0]);
    r_p[i] = fma(-delta, y[i] - lam[i], rp);
  }
  double tot[1];
  if (grid_sum<kNT, 1>(v, part, cnt, tot) && threadIdx.x == 0) out[0] = tot[0];
}

__global__ void k_scaling_dev(int n, const double* __restrict__ x, const double* __restrict__ z,
                              const double* __restrict__ q, const IpmDev* __restrict__ s, double* __restrict__ D) {
  const int j = blockIdx.x * kNT + threadIdx.x;
  if (j < n) D[j] = 1.0 / (q[j] + z[j] / x[j] + s->rho);
}

__global__ void __launch_bounds__(kNT) k_mu_aff_dev(int n, const double* __restrict__ x, const double* __restrict__ dx,
                                                    const double* __restrict__ z, const double* __restrict__ dz,
                                                    const IpmDev* __restrict__ s, double* out, double* part,
                                                    unsigned* cnt) {
  const double ap = s->ap_bar, ad = s->ad_bar;
  double v[1] = {0.0};
  for (int j = blockIdx.x * kNT + threadIdx.x; j < n; j += gridDim.x * kNT)
    v[0] = fma(fma(ap, dx[j], x[j]), fma(ad, dz[j], z[j]), v[0]);
  double tot[1];
  if (grid_sum<kNT, 1>(v, part, cnt, tot) && threadIdx.x == 0) out[0] = tot[0];
}

__global__ void k_corrector_rhs_dev(int n, const IpmDev* __restrict__ s, const double* __restrict__ dxp,
                                    const double* __restrict__ dzp, double* __restrict__ r_xz) {
  const int j = blockIdx.x * kNT + threadIdx.x;
  if (j < n) r_xz[j] = s->mu_t - dxp[j] * dzp[j];
}

__global__ void k_update_dev(int m, int n, const IpmDev* __restrict__ s, const double* __restrict__ dx,
                             const double* __restrict__ dy, const double* __restrict__ dz, double* __restrict__ x,
                             double* __restrict__ y, double* __restrict__ z) {
  const double ap = s->ap, ad = s->ad;
  const int j = blockIdx.x * kNT + threadIdx.x;
  if (j < n) {
    x[j] = fma(ap, dx[j], x[j]);
    z[j] = fma(ad, dz[j], z[j]);
  }
  if (j < m) y[j] = fma(ad, dy[j], y[j]);
}

// lambda <- y and zeta <- x where the PMM update re-centred them
__global__ void k_recentre(int m, int n, const IpmDev* __restrict__ s, const double* __restrict__ y,
                           const double* __restrict__ x, double* __restrict__ lam, double* __restrict__ zeta) {
  const int j = blockIdx.x * kNT + threadIdx.x;
  if (s->recentre_p && j < m) lam[j] = y[j];
  if (s->recentre_d && j < n) zeta[j] = x[j];
}

// Top of iteration k from the residual sums red = (||rd||^2, x^T z,
// ||b - Ax||^2): the device error word, the measures, the PMM update (k > 0),
// the termination test, eta_k, and the two PCG tasks of the iteration.
__global__ void k_ipm_top(IpmDev* s, const double* red, ClusterPcgTask* tasks, const int* forced, int* err) {
  if (threadIdx.x != 0 || blockIdx.x != 0 || s->done) return;
  const int e = *err;
  if (e != 0) {
    s->status = e;
    s->done = 1;
    return;
  }
  const double nrd = sqrt(red[0]), nrp = sqrt(red[2]);
  const double mu = red[1] / s->nmu;
  if (!isfinite(nrd) || !isfinite(nrp) || !isfinite(mu)) {
    s->status = kErrNumeric;
    s->done = 1;
    return;
  }
  const double rel_p = nrp / s->pden, rel_d = nrd / s->dden;
  if (s->ref_p < 0.0) s->ref_p = rel_p;
  if (s->ref_d < 0.0) s->ref_d = rel_d;
  s->recentre_p = 0;
  s->recentre_d = 0;
  const double tol = s->tol;
  if (s->k > 0) {
    // PMM update (Algorithm 6, last step): each estimate re-centred with the
    // cut 1 - r when its infeasibility progressed, else kept with 1 - (2/3) r
    const double den = fmax(s->mu_prev, mu);
    const double r = den > 0.0 ? fabs(__dadd_rn(mu, -s->mu_prev)) / den : 0.0;
    const double fast = __dadd_rn(1.0, -r);
    const double slow = __dadd_rn(1.0, -__dmul_rn(2.0 / 3.0, r));
    double delta = s->delta, rho = s->rho;
    if (s->ref_p <= tol || rel_p <= fmax(__dmul_rn(0.95, s->ref_p), tol)) {
      s->recentre_p = 1;
      s->ref_p = rel_p;
      delta = __dmul_rn(fast, delta);
    } else {
      delta = __dmul_rn(slow, delta);
    }
    if (s->ref_d <= tol || rel_d <= fmax(__dmul_rn(0.95, s->ref_d), tol)) {
      s->recentre_d = 1;
      s->ref_d = rel_d;
      rho = __dmul_rn(fast, rho);
    } else {
      rho = __dmul_rn(slow, rho);
    }
    s->delta = fmax(s->floor, delta);
    s->rho = fmax(s->floor, rho);
  }
  s->rel_p = rel_p;
  s->rel_d = rel_d;
  s->mu = mu;
  const bool kkt = rel_p <= tol && rel_d <= tol && mu <= tol;
  if (s->forced_ipm >= 0) {
    if (s->k >= s->forced_ipm) {
      s->status = kkt ? 0 : 1;          // NYS_OK / NYS_WARN_MAXITER
      s->done = 1;
    }
  } else if (kkt) {
    s->status = 0;
    s->done = 1;
  }
  if (!s->done && s->k >= s->max_ipm) {
    s->status = 1;
    s->done = 1;
  }
  const double eta = fmax(1e-10, fmin(1e-2, __dmul_rn(0.1, mu)));
  s->eta = eta;
  for (int w = 0; w < 2; ++w) {
    ClusterPcgTask& t = tasks[w];
    t.delta = s->delta;
    t.eta2 = __dmul_rn(eta, eta);
    t.max_iter = s->max_pcg;
    const int idx = s->solves + w;
    t.forced = idx < s->n_forced ? forced[idx] : -1;
    if (s->done) t.forced = 0;          // nothing to solve
  }
}

// After a PCG solve: its count into the log and the running total, and the
// warning when it stopped at max_iter without meeting its test.
__global__ void k_ipm_after_pcg(IpmDev* s, const ClusterPcgTask* task, const int* si, const double* sd, int* log,
                                int log_cap) {
  if (threadIdx.x != 0 || blockIdx.x != 0 || s->done) return;
  const int it = si[SI_ITERS];
  if (s->solves < log_cap) log[s->solves] = it;
  s->solves += 1;
  s->pcg_total += it;
  if (task->forced < 0 && it >= task->max_iter && !(sd[SD_RR] <= sd[SD_ETA2] * sd[SD_BNORM2])) s->warn = 2;
}

// Step lengths 0.995 min(1, ratio) from the step-ratio sums (Eq. stepsize-p/-d).
__global__ void k_ipm_steps(IpmDev* s, const double* red, int final_step) {
  if (threadIdx.x != 0 || blockIdx.x != 0 || s->done) return;
  const double ap = __dmul_rn(0.995, fmin(1.0, red[0]));
  const double ad = __dmul_rn(0.995, fmin(1.0, red[1]));
  if (final_step) {
    s->ap = ap;
    s->ad = ad;
  } else {
    s->ap_bar = ap;
    s->ad_bar = ad;
  }
}

// mu_aff and the corrector target mu_t = mu_aff^3 / mu^2 (Algorithm 5).
__global__ void k_ipm_mu_t(IpmDev* s, const double* red) {
  if (threadIdx.x != 0 || blockIdx.x != 0 || s->done) return;
  const double mu_aff = red[0] / s->nmu;
  const double mu = s->mu;
  s->mu_t = mu > 0.0 ? __dmul_rn(__dmul_rn(mu_aff, mu_aff), mu_aff) / __dmul_rn(mu, mu) : 0.0;
}

__global__ void k_ipm_iter_end(IpmDev* s) {
  if (threadIdx.x != 0 || blockIdx.x != 0 || s->done) return;
  s->mu_prev = s->mu;
  s->k += 1;
}

__global__ void k_ipm_cond(cudaGraphConditionalHandle cond, const IpmDev* s) {
  cudaGraphSetConditional(cond, s->done ? 0u : 1u);
}

}  // namespace

cudaError_t ipm_residuals_dev(cudaStream_t st, int m, int n, const double* b, const double* c, const double* q,
                              const double* x, const double* y, const double* z, const double* Ax,
                              const double* Aty, const double* lam, const double* zeta, const IpmDev* s,
                              double* r_d, double* r_p, double* r_xz, double* red_out, RedBuf red) {
  count_launches(1);
  k_res_n_dev<<<grid_for(n), kNT, 0, st>>>(n, c, q, x, z, Aty, zeta, s, r_d, r_xz, red_out, red.part, red.cnt + 4);
  count_launches(1);
  k_res_m_dev<<<grid_for(m), kNT, 0, st>>>(m, b, Ax, y, lam, s, r_p, red_out + 2, red.part + 4 * 2 * 152,
                                           red.cnt + 5);
  return cudaGetLastError();
}

cudaError_t scaling_dev(cudaStream_t st, int n, const double* x, const double* z, const double* q, const IpmDev* s,
                        double* D) {
  count_launches(1);
  k_scaling_dev<<<(n + kNT - 1) / kNT, kNT, 0, st>>>(n, x, z, q, s, D);
  return cudaGetLastError();
}

cudaError_t mu_aff_dev(cudaStream_t st, int n, const double* x, const double* dx, const double* z, const double* dz,
                       const IpmDev* s, double* out, RedBuf red) {
  count_launches(1);
  k_mu_aff_dev<<<grid_for(n), kNT, 0, st>>>(n, x, dx, z, dz, s, out, red.part, red.cnt + 8);
  return cudaGetLastError();
}

cudaError_t corrector_rhs_dev(cudaStream_t st, int n, const IpmDev* s, const double* dxp, const double* dzp,
                              double* r_xz) {
  count_launches(1);
  k_corrector_rhs_dev<<<(n + kNT - 1) / kNT, kNT, 0, st>>>(n, s, dxp, dzp, r_xz);
  return cudaGetLastError();
}

cudaError_t ipm_update_dev(cudaStream_t st, int m, int n, const IpmDev* s, const double* dx, const double* dy,
                           const double* dz, double* x, double* y, double* z) {
  const int len = n > m ? n : m;
  count_launches(1);
  k_update_dev<<<(len + kNT - 1) / kNT, kNT, 0, st>>>(m, n, s, dx, dy, dz, x, y, z);
  return cudaGetLastError();
}

cudaError_t ipm_recentre(cudaStream_t st, int m, int n, const IpmDev* s, const double* y, const double* x,
                         double* lam, double* zeta) {
  const int len = n > m ? n : m;
  count_launches(1);
  k_recentre<<<(len + kNT - 1) / kNT, kNT, 0, st>>>(m, n, s, y, x, lam, zeta);
  return cudaGetLastError();
}

cudaError_t ipm_top_dev(cudaStream_t st, IpmDev* s, const double* red_out, ClusterPcgTask* tasks, const int* forced,
                        int* err) {
  count_launches(1);
  k_ipm_top<<<1, 32, 0, st>>>(s, red_out, tasks, forced, err);
  return cudaGetLastError();
}

cudaError_t ipm_after_pcg_dev(cudaStream_t st, IpmDev* s, const ClusterPcgTask* task, const int* si, const double* sd,
                              int* log, int log_cap) {
  count_launches(1);
  k_ipm_after_pcg<<<1, 32, 0, st>>>(s, task, si, sd, log, log_cap);
  return cudaGetLastError();
}

cudaError_t ipm_steps_dev(cudaStream_t st, IpmDev* s, const double* red_out, int final_step) {
  count_launches(1);
  k_ipm_steps<<<1, 32, 0, st>>>(s, red_out, final_step);
  return cudaGetLastError();
}

cudaError_t ipm_mu_t_dev(cudaStream_t st, IpmDev* s, const double* red_out) {
  count_launches(1);
  k_ipm_mu_t<<<1, 32, 0, st>>>(s, red_out);
  return cudaGetLastError();
}

cudaError_t ipm_iter_end_dev(cudaStream_t st, IpmDev* s) {
  count_launches(1);
  k_ipm_iter_end<<<1, 32, 0, st>>>(s);
  return cudaGetLastError();
}

cudaError_t ipm_cond_dev(cudaStream_t st, cudaGraphConditionalHandle cond, const IpmDev* s) {
  count_launches(1);
  k_ipm_cond<<<1, 1, 0, st>>>(cond, s);
  return cudaGetLastError();
}

}  // namespace nys
