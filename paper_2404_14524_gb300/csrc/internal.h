// Host-side interface between the translation units of the library.
// Every launcher issues its kernels on `st` and returns a cudaError_t of the
// launch (kernel-side failures are reported through the device error word).
#pragma once
#include <cuda_bf16.h>
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
  SD_DELTA,       // delta of the system being solved by PCG
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
// out[i] = sum_j A[i, j] t[j] + beta * v[i]   (v may be nullptr when beta == 0);
// when beta_dev is given, beta is read from device memory instead.  With a
// split buffer, rows too few to fill the GPU are cut into column chunks
// (partials in split_buf, then a fixed-order sum).
cudaError_t gemv_n_f64(cudaStream_t st, int m, int n, const double* A, long long lda,
                       const double* t, double beta, const double* v, double* out,
                       const int* skip = nullptr, const double* beta_dev = nullptr,
                       double* split_buf = nullptr, size_t split_cap = 0);
// Rows of split-reduction scratch that gemv_t_f64 needs for an m x n matrix.
size_t gemv_t_split_elems(int m, int n);

// D_j = 1 / (q_j + z_j / x_j + rho)
cudaError_t scaling_f64(cudaStream_t st, int n, const double* x, const double* z, const double* q,
                        double rho, double* D);

// ---------------------------------------------------------------- sketch
// Omega_k of width ell (the counter stride); only its first `cols` columns
// are written (cols < 0: all ell).
cudaError_t gaussian_omega(cudaStream_t st, unsigned long long seed, int k, int m, int ell,
                           double* Om, int ld, int cols = -1);
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
  double* B2;       // m x ell (ld)   Q W for the QR route (large ell)
  double* R;        // ell x ell      accumulated R of the QR passes, then W = R V
  double* Rt;       // ell x ell      scratch product
  unsigned int* bar;  // 2 words      grid barrier
  int* sweep_flags;   // kMaxSweeps   rotation flags per Jacobi sweep
  double* split_buf;
  size_t split_cap;
  int f32_start = 1;  // FP32 Jacobi start for small B (NYS_JACOBI_F32=0 turns it off)
  int gram = 1;       // after it, FP64 sweeps on B^T B in one CTA (NYS_JACOBI_GRAM=0: on B, cluster)
  static constexpr int kMaxSweeps = 40;
};
// Algorithm 1 steps 3-8 from a sketch.  Writes U (m x ell, ld), lam (ell) and
// the device scalar SD_NU; errors go to the device error word.
cudaError_t nystrom_core_f64(cudaStream_t st, int m, int ell, const double* Y, const double* Om,
                             int ld, double* U, double* lam, double* sd, int* si, RedBuf red,
                             CoreWork cw, int num_sms);

// ---------------------------------------------------------------- precision-form GEMVs
// Storage types of the reduced-precision operator.
constexpr int kLpFp32 = 0;
constexpr int kLpBf16 = 1;
constexpr int kLpFp8 = 2;     // E4M3 with per-row scales
// out[r] = scale[r] * sum_c A[r, c] x[c] + beta v[r]; A row-major in FP32,
// BF16 or FP8 E4M3 (a_type), x/scale FP32, FP32 accumulation; out FP64
// (out_f64) or FP32.
// With `part` (>= splits * rows doubles) short, wide matrices are split over
// columns as well, with a fixed-order reduction of the partial sums.
cudaError_t gemv_rows_lp(cudaStream_t st, int rows, int cols, int a_type, const void* A, long long lda,
                         const float* x, const float* scale, double beta, const double* v, void* out,
                         int out_f64, const int* skip = nullptr, const double* beta_dev = nullptr,
                         double* part = nullptr, size_t part_cap = 0);
// FP32 A times x = xh + xl with float-float accumulation, FP64 out.
cudaError_t gemv_rows_ff(cudaStream_t st, int rows, int cols, const float* A, long long lda, const float* xh,
                         const float* xl, const double* scale, double beta, const double* v, double* out,
                         const int* skip = nullptr, const double* beta_dev = nullptr, double* part = nullptr,
                         size_t part_cap = 0);
// hi/lo FP32 split of scale .* x, zero padded to npad
cudaError_t split_ff(cudaStream_t st, int n, int npad, const double* x, const double* scale, float* hi, float* lo,
                     const int* skip = nullptr);
cudaError_t to_f32(cudaStream_t st, int n, int npad, const double* x, const double* scale, float* y,
                   const int* skip = nullptr);
// BF16 copy (dst, ldd), BF16 transpose (dstT, ldt) and FP32 transpose (dstTf,
// ldtf) of a row-major FP32/FP64 matrix; any output may be null; padding zeroed.
cudaError_t convert_transpose(cudaStream_t st, int rows, int cols, int src_f64, const void* src, long long lds,
                              __nv_bfloat16* dst, long long ldd, __nv_bfloat16* dstT, long long ldt,
                              float* dstTf, long long ldtf);

// FP8 E4M3 copies of a row-major FP32 matrix with per-row scales:
// s_r = max_c |A[r, c]| / 448 (1 for a zero row), Q[r, c] = E4M3(A[r, c] / s_r)
// (ldq >= cols, padding zeroed) and QT = Q^T (ldqt >= rows); s in FP32 and FP64.
cudaError_t quantize_fp8(cudaStream_t st, int rows, int cols, const float* A, long long lda, float* s32,
                         double* s64, void* Q, long long ldq, void* QT, long long ldqt);

// ---------------------------------------------------------------- tcgen05 BF16 GEMM
// out[c * ldo + r] = op(sum_k A[r, k] B[c, k]) for r < M, c < N; A: M x K,
// B: N x K, both BF16 row-major (K contiguous, leading dimensions multiples
// of 8), N <= 512, FP32 accumulation.  mode 0: FP32 out; mode 1: scaled by
// D[r] (FP64) and stored as BF16.  The CTA-pair kernel (M = 256 per pair,
// stream-K over k-blocks) runs when clusters of two can be launched and
// `part` holds its partial tiles, else the one-SM kernel with split-K;
// *kernel_used (if given) receives 2 or 1.  part_cap is in floats; size it
// with umma_part_elems.
size_t umma_part_elems(int M, int N, int K, int num_sms);
cudaError_t umma_gemm_bf16(cudaStream_t st, int M, int N, int K, const void* A, long long lda,
                           const void* B, long long ldb, float* part, size_t part_cap, int num_sms, int mode,
                           const double* D, void* out, long long ldo, int* err, int* kernel_used = nullptr);

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
// Issue one predicated PCG iteration (no-op once SI_DONE is set).  delta is
// read from sd[SD_DELTA] (written by the setup), so a captured iteration
// stays valid across solves.
cudaError_t pcg_iteration_f64(cudaStream_t st, int m, int n, const double* A, long long lda,
                              const double* D, int ell, const double* U, int ld,
                              PcgWork w, double* sd, int* si, RedBuf red);
// Reduced-precision operator (N + delta I) p for the precision form: A and
// A^T stored row-major in BF16 (bf16 = 1) or FP32, D in FP32; scratch xf
// (ld_mpad floats, zero padded) and tf (n floats).
struct LpOperator {
  int ff;                           // 1: FP32 storage with float-float sums (A, AT FP32)
  const double* D64;                // ff: FP64 D
  double* t64;                      // ff: FP64 scratch of n for D .* (A^T p)
  float *xh, *xl;                   // ff: hi/lo split scratch, max(m, n) padded
  int ld_npad;
  int a_type;                       // kLpFp32, kLpBf16 or kLpFp8
  const void* A;  long long lda;    // m x n
  const void* AT; long long ldat;   // n x m
  const float* rs32;                // kLpFp8: row scales of A (m), FP32
  const double* rs64;               //   and FP64
  const float* Df;
  float* xf;
  float* tf;
  int ld_mpad;
  double* part;                     // column-split partial sums
  size_t part_cap;
};
cudaError_t pcg_iteration_lp(cudaStream_t st, int m, int n, const LpOperator& op, int ell,
                             const double* U, int ld, PcgWork w, double* sd, int* si, RedBuf red);
// Whole PCG solve in one cooperative launch (small problems): same result
// semantics as pcg_setup_f64 + pcg_iteration_f64 (solution in w.x, SI_ITERS,
// SD_RR); part needs grid * (ell + 2) doubles, bar two zeroable words.
bool pcg_persistent_fits(int m, int n, int ell);
cudaError_t pcg_persistent_f64(cudaStream_t st, int m, int n, const double* A, long long lda, const double* D,
                               double delta, int ell, const double* U, int ld, const double* lam, const double* xi,
                               double eta, int max_iter, int forced, PcgWork w, double* part, size_t part_cap,
                               unsigned* bar, double* sd, int* si, int num_sms);
// Whole PCG solves in thread-block clusters (small problems): one cluster of
// C CTAs per system, the column band of A in shared memory when it fits.
struct ClusterPcgTask {
  int m, n, ell, ld;
  long long lda;
  const double *A, *D, *U, *lam, *xi;   // device: m x n (lda), n, m x ell (ld), ell, m
  double delta, eta2;
  int max_iter, forced;
  double* x;                            // device, m: the solution
  int* iters;                           // device: iterations taken
  double* sd;                           // device scalars: SD_RR, SD_BNORM2, SD_ETA2 written
  int* err;                             // device error word
  unsigned long long* t_ns;             // device, optional: the launch's duration is added (ns)
};
struct ClusterPlan {
  int C = 0;                            // CTAs per cluster (4, 8 or 16)
  int a_smem = 0;                       // A's column band held in shared memory
  size_t smem_bytes = 0;                // dynamic shared memory per CTA
};
// Plan for an m x n system with rank ell: policy 0 for the latency of one
// solve, 1 for many solves side by side, 2 the latency plan if one exists,
// else the throughput plan; false when no cluster fits.
bool pcg_cluster_plan(int m, int n, int ell, int policy, ClusterPlan* plan);
// Every cluster plan that fits an m x n system of rank ell (16, 8, 4 CTAs
// with A on chip, then 8, 4 with A read from L2), at most cap; returns the
// count.
int pcg_cluster_candidates(int m, int n, int ell, ClusterPlan* out, int cap);
// The plan of C CTAs (A on chip if a_smem) for this exact shape, if it fits.
bool pcg_cluster_plan_for(int m, int n, int ell, int C, int a_smem, ClusterPlan* plan);
// One system (`task`, tasks == nullptr) or `count` systems from the device
// array `tasks`, each planned no larger than `plan`.
cudaError_t pcg_cluster_f64(cudaStream_t st, const ClusterPlan& plan, const ClusterPcgTask& task,
                            const ClusterPcgTask* tasks, int count);
// ---------------------------------------------------------------- device-resident IPM iteration
// Scalars of one IP-PMM run kept in device memory (see ipm_dev.cu).
struct IpmDev {
  double mu, mu_prev, rho, delta, ref_p, ref_d, rel_p, rel_d, eta;
  double ap, ad, ap_bar, ad_bar, mu_t;
  double tol, floor, pden, dden, nmu;   // tolerance, PMM floor, 1 + ||b||, 1 + ||c||, n
  int k, k0, done, status, warn;
  int forced_ipm, max_ipm, n_forced, max_pcg;
  int solves, pcg_total, recentre_p, recentre_d;
  unsigned long long pcg_ns;            // device time of the PCG launches
};
cudaError_t ipm_residuals_dev(cudaStream_t st, int m, int n, const double* b, const double* c, const double* q,
                              const double* x, const double* y, const double* z, const double* Ax,
                              const double* Aty, const double* lam, const double* zeta, const IpmDev* s,
                              double* r_d, double* r_p, double* r_xz, double* red_out, RedBuf red);
cudaError_t scaling_dev(cudaStream_t st, int n, const double* x, const double* z, const double* q, const IpmDev* s,
                        double* D);
cudaError_t mu_aff_dev(cudaStream_t st, int n, const double* x, const double* dx, const double* z, const double* dz,
                       const IpmDev* s, double* out, RedBuf red);
cudaError_t corrector_rhs_dev(cudaStream_t st, int n, const IpmDev* s, const double* dxp, const double* dzp,
                              double* r_xz);
cudaError_t ipm_update_dev(cudaStream_t st, int m, int n, const IpmDev* s, const double* dx, const double* dy,
                           const double* dz, double* x, double* y, double* z);
cudaError_t ipm_recentre(cudaStream_t st, int m, int n, const IpmDev* s, const double* y, const double* x,
                         double* lam, double* zeta);
cudaError_t ipm_top_dev(cudaStream_t st, IpmDev* s, const double* red_out, ClusterPcgTask* tasks, const int* forced,
                        int* err);
cudaError_t ipm_after_pcg_dev(cudaStream_t st, IpmDev* s, const ClusterPcgTask* task, const int* si, const double* sd,
                              int* log, int log_cap);
cudaError_t ipm_steps_dev(cudaStream_t st, IpmDev* s, const double* red_out, int final_step);
cudaError_t ipm_mu_t_dev(cudaStream_t st, IpmDev* s, const double* red_out);
cudaError_t ipm_iter_end_dev(cudaStream_t st, IpmDev* s);
cudaError_t ipm_cond_dev(cudaStream_t st, cudaGraphConditionalHandle cond, const IpmDev* s);
// Omega_k with k = *k_dev + k0 read on the device (width ell, as gaussian_omega)
cudaError_t gaussian_omega_dev(cudaStream_t st, unsigned long long seed, const int* k_dev, int k0, int m, int ell,
                               double* Om, int ld);
// Whether the Nystrom core of an m x ell sketch runs as plain and cluster
// kernel launches only (no cooperative launch, no copy): capturable in a
// conditional graph body.
bool nystrom_core_capturable(int m, int ell);

// Body-graph tail of a conditional while node: keep looping while !SI_DONE.
cudaError_t pcg_loop_condition(cudaStream_t st, cudaGraphConditionalHandle cond, const int* si);

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
// m-part alone: r_p = b - Ax - delta (y - lam); red_out[0] = ||b - Ax||^2 (device)
cudaError_t ipm_residuals_m_f64(cudaStream_t st, int m, const double* b, const double* Ax, const double* y,
                                const double* lam, double delta, double* r_p, double* red_out, RedBuf red);
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
// ---------------------------------------------------------------- free and box-constrained variables
// Problems (P~)/(D~): kind per variable vk[j] in {0 = I (x_j >= 0), 1 = F
// (free), 2 = J (0 <= x_j <= u_j)}, slack w = u - x and multiplier s on J.
// Every kernel keeps z = 0 on F and u = w = s = 0 outside J.
struct BoxVectors {
  const signed char* vk = nullptr;
  const double* w = nullptr;
  const double* s = nullptr;
};
// In place on the handle's copies: z_F = 0; on J w = w0 (has_w0) or u - x,
// s = s0 (only when given_start: the practical start writes w, s on J
// itself); elsewhere u = w = s = 0.  out[0] = |I u J| + |J|,
// out[1] = ||u_J||^2, out[2] = count of invalid entries (device).
cudaError_t box_start_f64(cudaStream_t st, int n, const signed char* vk, double* u, const double* x, double* z,
                          double* w, double* s, int has_u, int has_w0, int has_s0, int given_start, double* out,
                          RedBuf red);
// D = 1 / (q + Theta^{-1} + rho), Theta^{-1} = z/x on I, z/x + s/w on J, 0 on F
cudaError_t box_scaling_f64(cudaStream_t st, int n, const signed char* vk, const double* x, const double* z,
                            const double* w, const double* s, const double* q, double rho, double* D);
// n-part of Eq. predictor-RHS: r_d, r_u, r_xz, r_ws; out[0] = ||c + Qx - A^T y - z + s||^2,
// out[1] = x_IJ^T z_IJ + w_J^T s_J, out[2] = ||u_J - x_J - w_J||^2 (device)
cudaError_t box_residuals_n_f64(cudaStream_t st, int n, const signed char* vk, const double* c, const double* q,
                                const double* u, const double* x, const double* z, const double* w,
                                const double* s, const double* Aty, const double* zeta, double rho, double* r_d,
                                double* r_u, double* r_xz, double* r_ws, double* out, RedBuf red);
// t = D (r_d + xi_au) of Algorithm 4 (null r_d / r_u mean zero)
cudaError_t box_newton_rhs_f64(cudaStream_t st, int n, const BoxVectors& bx, const double* D, const double* r_d,
                               const double* r_u, const double* r_xz, const double* r_ws, const double* x,
                               double* t);
// dx = D (g - r_d - xi_au), dw, dz, ds of Algorithm 4 (g = A^T dy)
cudaError_t box_newton_back_f64(cudaStream_t st, int n, const BoxVectors& bx, const double* D, const double* g,
                                const double* r_d, const double* r_u, const double* r_xz, const double* r_ws,
                                const double* x, const double* z, double* dx, double* dz, double* dw,
                                double* ds);
// out[0] = min ratio over (x, dx) on I u J and (w, dw) on J; out[1] over (z, dz), (s, ds)
cudaError_t box_step_ratios_f64(cudaStream_t st, int n, const signed char* vk, const double* x, const double* dx,
                                const double* w, const double* dw, const double* z, const double* dz,
                                const double* s, const double* ds, double* out, RedBuf red);
// out = (x + ap dx)_IJ^T (z + ad dz)_IJ + (w + ap dw)_J^T (s + ad ds)_J
cudaError_t box_mu_aff_f64(cudaStream_t st, int n, const signed char* vk, const double* x, const double* dx,
                           const double* z, const double* dz, const double* w, const double* dw, const double* s,
                           const double* ds, double ap, double ad, double* out, RedBuf red);
// r_xz = mu_t - dxp dzp on I u J, r_ws = mu_t - dwp dsp on J (0 elsewhere)
cudaError_t box_corrector_rhs_f64(cudaStream_t st, int n, const signed char* vk, double mu_t, const double* dxp,
                                  const double* dzp, const double* dwp, const double* dsp, double* r_xz,
                                  double* r_ws);
// ---------------------------------------------------------------- practical initial point
// out[0..len) = v
cudaError_t fill_f64(cudaStream_t st, int len, double v, double* out);
// candidate z~ (g/2 on J, 0 on F), w~ = u - x~ and s~ = -z~ on J from g = c - A^T y~ + Q x~;
// out[0] = min over x~_IJ, w~_J; out[1] = min over z~_IJ, s~_J (device; +inf if empty).
// vk null: problem (P), w and s untouched.
cudaError_t start_candidate_f64(cudaStream_t st, int n, const signed char* vk, const double* c, const double* q,
                                const double* u, const double* x, const double* Aty, double* z, double* w,
                                double* s, double* out, RedBuf red);
// out[0] = gamma, out[1] = sum (z~ + dd, s~ + dd), out[2] = sum (x~ + dp, w~ + dp) (device)
cudaError_t start_sums_f64(cudaStream_t st, int n, const signed char* vk, const double* x, const double* z,
                           const double* w, const double* s, double dp, double dd, double* out, RedBuf red);
// x_IJ, w_J += dpt; z_IJ, s_J += ddt
cudaError_t start_shift_f64(cudaStream_t st, int n, const signed char* vk, double dpt, double ddt, double* x,
                            double* z, double* w, double* s);
// out = a .* b
cudaError_t vmul_f64(cudaStream_t st, int len, const double* a, const double* b, double* out);
// out[i, j] = alpha u_i v_j + beta w_i s_j, row-major m x n (FP32 or FP64 out)
cudaError_t rank2_update(cudaStream_t st, int m, int n, double alpha, const double* u, const double* v, double beta,
                         const double* w, const double* s, void* out, long long ldo, int out_f32);
// out = a x + b y
cudaError_t axpby_f64(cudaStream_t st, int len, double a, const double* x, double b, const double* y, double* out);
// P (m x ell, column-major, FP64) rounded to BF16 in place; the BF16 copy goes
// to Pb with leading dimension ldb (rows of the transposed panel).
cudaError_t round_panel_bf16(cudaStream_t st, int m, int ell, double* P, int ld, __nv_bfloat16* Pb, int ldb);
cudaError_t panel_f32_to_f64(cudaStream_t st, int m, int ell, const float* src, int lds, double* dst, int ldd);
// out = a^T b (device scalar)
cudaError_t dot_f64(cudaStream_t st, int len, const double* a, const double* b, double* out,
                    RedBuf red);
// out[0] = x^T (q x), out[1] = c^T x, out[2] = b^T y, out[3] = any non-finite in x,y,z
cudaError_t objective_terms_f64(cudaStream_t st, int m, int n, const double* q, const double* c,
                                const double* b, const double* x, const double* y,
                                const double* z, double* out, RedBuf red);

}  // namespace nys
