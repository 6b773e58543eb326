// Host-side interface between the translation units of the library.
// Every launcher issues its kernels on `st` and returns a cudaError_t of the
// launch (kernel-side failures are reported through the device error word).
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

namespace nys {

// Number of kernels this library has launched (all handles, all threads).
void count_launches(unsigned n);

// Device scalars shared by the PCG kernels (one block of doubles + ints).
enum ScalarD : int {
  SD_RZ = 0,      // r^T z of the current PCG iteration
  SD_ALPHA,       // CG step
  SD_BETA,        // CG direction update
  SD_RR,          // ||r||^2
  SD_BNORM2,      // ||rhs||^2
  SD_ETA2,        // eta^2 (relative tolerance squared)
  SD_FROB2,       // ||Y||_F^2 of the sketch
  SD_NU,          // nu of Algorithm 1
  SD_RED0,        // generic reduction outputs
  SD_RED1,
  SD_RED2,
  SD_RED3,
  SD_RED4,
  SD_COUNT
};
enum ScalarI : int {
  SI_DONE = 0,    // PCG finished (converged, forced count or max_iter)
  SI_ITERS,       // PCG iterations taken
  SI_FORCED,      // forced iteration count (< 0: none)
  SI_MAXIT,
  SI_ERR,         // device error word (nys_status code, 0 = ok)
  SI_SWEEPS,      // Jacobi sweeps used
  SI_COUNT
};

// Reduction scratch: a counter array and a partial-sum buffer.
struct RedBuf {
  double* part = nullptr;        // kPartCap doubles
  unsigned int* cnt = nullptr;   // kCntCap counters (zero at rest)
  static constexpr size_t kPartCap = 1 << 20;
  static constexpr int kCntCap = 16;
};

// ---------------------------------------------------------------- GEMV (FP64)
// t[j] = scale_j * sum_i A[i, j] v[i],  scale_j = D[j] (or 1 when D == nullptr)
cudaError_t gemv_t_f64(cudaStream_t st, int m, int n, const double* A, long long lda,
                       const double* v, const double* D, double* t, double* split_buf,
                       size_t split_cap, const int* skip = nullptr);
// out[i] = sum_j A[i, j] t[j] + beta * v[i]   (v may be nullptr when beta == 0)
cudaError_t gemv_n_f64(cudaStream_t st, int m, int n, const double* A, long long lda,
                       const double* t, double beta, const double* v, double* out,
                       const int* skip = nullptr);
// Rows of split-reduction scratch that gemv_t_f64 needs for an m x n matrix.
size_t gemv_t_split_elems(int m, int n);

// D_j = 1 / (q_j + z_j / x_j + rho)
cudaError_t scaling_f64(cudaStream_t st, int n, const double* x, const double* z, const double* q,
                        double rho, double* D);

// ---------------------------------------------------------------- sketch
cudaError_t gaussian_omega(cudaStream_t st, unsigned long long seed, int k, int m, int ell,
                           double* Om, int ld);
// C(r, c) = sum_k Aop(r, k) * Bop(k, c) * (scale ? scale[k] : 1), FP64.
// Aop(r, k) = A[r * sar + k * sak], Bop(k, c) = B[k * sbk + c * sbc], C[r * scr + c * scc].
// One of sar/sak must be 1, and sbk must be 1.
cudaError_t gemm_f64(cudaStream_t st, int M, int N, int K, const double* A, long long sar,
                     long long sak, const double* B, long long sbk, long long sbc,
                     const double* scale, double* C, long long scr, long long scc,
                     double* split_buf, size_t split_cap);
// Y = A (D .* (A^T Omega)); T: n x ell scratch (ld_t)
cudaError_t sketch_f64(cudaStream_t st, int m, int n, const double* A, long long lda,
                       const double* D, int ell, const double* Om, int ld, double* Y,
                       double* T, int ld_t, double* split_buf, size_t split_cap);

// ---------------------------------------------------------------- Nystrom core
struct CoreWork {
  double* Ynu;      // m x ell (ld)   Y + nu Omega, then B in place
  double* G;        // ell x ell      Omega^T Y_nu, then C (upper Cholesky factor)
  double* sumsq;    // ell            squared column norms of the converged B
  int* perm;        // ell            column of B that becomes column r of U
  unsigned int* bar;  // 2 words      grid barrier
  int* sweep_flags;   // kMaxSweeps   rotation flags per Jacobi sweep
  double* split_buf;
  size_t split_cap;
  static constexpr int kMaxSweeps = 40;
};
// Algorithm 1 steps 3-8 from a sketch.  Writes U (m x ell, ld), lam (ell) and
// the device scalar SD_NU; errors go to the device error word.
cudaError_t nystrom_core_f64(cudaStream_t st, int m, int ell, const double* Y, const double* Om,
                             int ld, double* U, double* lam, double* sd, int* si, RedBuf red,
                             CoreWork cw, int num_sms);

// ---------------------------------------------------------------- PCG / P^{-1}
struct PcgWork {
  double *x, *r, *z, *p, *w;  // m each
  double* s;                  // ell: U^T r
  double* wts;                // ell: (lam_ell + delta) / (lam + delta) - 1
  double* t;                  // n  : A^T p scratch
  double* split_buf;
  size_t split_cap;
};
// out = P^{-1} r; wts computed from lam and delta.
cudaError_t precond_apply_f64(cudaStream_t st, int m, int ell, const double* U, int ld,
                              const double* lam, double delta, const double* r, double* out,
                              double* s, double* wts, RedBuf red);
// Issue the PCG setup kernels (solution reset, residual, first direction).
cudaError_t pcg_setup_f64(cudaStream_t st, int m, int ell, const double* U, int ld,
                          const double* lam, double delta, const double* xi, double eta,
                          int max_iter, int forced, PcgWork w, double* sd, int* si, RedBuf red);
// Issue one predicated PCG iteration (no-op once SI_DONE is set).
cudaError_t pcg_iteration_f64(cudaStream_t st, int m, int n, const double* A, long long lda,
                              const double* D, double delta, int ell, const double* U, int ld,
                              PcgWork w, double* sd, int* si, RedBuf red);

// ---------------------------------------------------------------- IPM vectors
// Residuals at the top of an IPM iteration (Eq. predictor-RHS, I = all):
//  n-part: rd_true = c + q x - Aty - z; r_d = rd_true + rho (x - zeta); r_xz = -x z
//          reductions: ||rd_true||^2, x^T z
//  m-part: rp_true = b - Ax;  r_p = rp_true - delta (y - lam)
//          reductions: ||rp_true||^2
// Outputs: red_out[0] = ||rd_true||^2, [1] = x^T z, [2] = ||rp_true||^2 (device)
cudaError_t ipm_residuals_f64(cudaStream_t st, int m, int n, const double* b, const double* c,
                              const double* q, const double* x, const double* y,
                              const double* z, const double* Ax, const double* Aty,
                              const double* lam, const double* zeta, double rho, double delta,
                              double* r_d, double* r_p, double* r_xz, double* red_out,
                              RedBuf red);
// t = D (r_d - r_xz / x)   (null r_d means zero)
cudaError_t newton_rhs_f64(cudaStream_t st, int n, const double* D, const double* r_d,
                           const double* r_xz, const double* x, double* t);
// dx = D (g - r_d + r_xz / x); dz = (r_xz - z dx) / x
cudaError_t newton_back_f64(cudaStream_t st, int n, const double* D, const double* g,
                            const double* r_d, const double* r_xz, const double* x,
                            const double* z, double* dx, double* dz);
// out[0] = min over dx<0 of -x/dx, out[1] likewise for (z, dz)  (+inf if none); device
cudaError_t step_ratios_f64(cudaStream_t st, int n, const double* x, const double* dx,
                            const double* z, const double* dz, double* out, RedBuf red);
// out = (x + ap dx)^T (z + ad dz)   (device scalar)
cudaError_t mu_aff_f64(cudaStream_t st, int n, const double* x, const double* dx,
                       const double* z, const double* dz, double ap, double ad, double* out,
                       RedBuf red);
// r_xz = mu_t - dxp .* dzp
cudaError_t corrector_rhs_f64(cudaStream_t st, int n, double mu_t, const double* dxp,
                              const double* dzp, double* r_xz);
// dx += dxp; dy += dyp; dz += dzp  (final direction = predictor + corrector)
cudaError_t add_dirs_f64(cudaStream_t st, int m, int n, const double* dxp, const double* dyp,
                         const double* dzp, double* dx, double* dy, double* dz);
// x += ap dx; z += ad dz (n);  y += ad dy (m)
cudaError_t ipm_update_f64(cudaStream_t st, int m, int n, double ap, double ad, const double* dx,
                           const double* dy, const double* dz, double* x, double* y, double* z);
// out = a^T b (device scalar)
cudaError_t dot_f64(cudaStream_t st, int len, const double* a, const double* b, double* out,
                    RedBuf red);
// out[0] = x^T (q x), out[1] = c^T x, out[2] = b^T y, out[3] = any non-finite in x,y,z
cudaError_t objective_terms_f64(cudaStream_t st, int m, int n, const double* q, const double* c,
                                const double* b, const double* x, const double* y,
                                const double* z, double* out, RedBuf red);

}  // namespace nys
