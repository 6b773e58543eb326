// Nystrom core factorisation (Algorithm 1, steps 3-8) in FP64:
//   nu = eps(||Y||_F);  Y_nu = Y + nu Omega;  G = Omega^T Y_nu (symmetrised);
//   C = chol(G) (upper, G = C^T C);  B = Y_nu C^{-1};  thin SVD of B;
//   lam = max(0, Sigma^2 - nu) in descending order, U = left singular vectors.
//
// The thin SVD is a one-sided (Hestenes) Jacobi iteration, run as one
// cooperative launch: each round rotates ell/2 disjoint column pairs in
// parallel (one CTA per pair, round-robin ordering), with a bounded grid
// barrier between rounds.  One-sided Jacobi orthogonalises columns directly,
// so small singular values keep their relative accuracy (no Gram matrix, no
// squared condition number).  After convergence the column norms are the
// singular values and the normalised columns the left singular vectors.
// For ell <= 96 it runs on B itself; for larger ell on the triangular factor
// R of B = Q R (shifted three-pass Cholesky QR), and B V = Q (R V).
#include "common.cuh"
#include "internal.h"

namespace nys {

namespace {

// Above this sketch size the thin SVD goes through a QR of B first: one-sided
// Jacobi directly on B costs ~3.5 m ell^2 DFMAs per sweep (8-10 sweeps),
// the QR route ~4 m ell^2 DFMAs in total plus sweeps on an ell x ell matrix.
constexpr int kJacobiDirectMaxEll = 96;

__global__ void __launch_bounds__(kNT) k_frob(int m, int ell, const double* __restrict__ Y, int ld,
                                              double* sd, int* err, double* part, unsigned* cnt) {
  const long long total = (long long)m * ell;
  double v[1] = {0.0};
  for (long long idx = (long long)blockIdx.x * kNT + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * kNT) {
    const int i = (int)(idx % m), j = (int)(idx / m);
    const double y = Y[(size_t)j * ld + i];
    v[0] = fma(y, y, v[0]);
  }
  double out[1];
  if (grid_sum<kNT, 1>(v, part, cnt, out) && threadIdx.x == 0) {
    const double f2 = out[0];
    sd[SD_FROB2] = f2;
    const double f = sqrt(f2);
    if (!(f > 0.0) || !isfinite(f)) {
      set_error(err, kErrNumeric);
      sd[SD_NU] = 0.0;
    } else {
      int e;
      frexp(f, &e);                 // f = g 2^e, g in [0.5, 1)
      sd[SD_NU] = ldexp(1.0, e - 53);  // spacing of float64 at f
    }
  }
}

__global__ void k_shift(int m, int ell, const double* __restrict__ Y, const double* __restrict__ Om,
                        int ld, const double* sd, double* __restrict__ Ynu) {
  const long long idx = (long long)blockIdx.x * kNT + threadIdx.x;
  if (idx >= (long long)m * ell) return;
  const int i = (int)(idx % m), j = (int)(idx / m);
  const size_t o = (size_t)j * ld + i;
  Ynu[o] = fma(sd[SD_NU], Om[o], Y[o]);
}

// One CTA: symmetrise G (ell x ell, column-major) and overwrite its upper
// triangle with C, G = C^T C (row j of C computed from rows 0..j-1).
__global__ void __launch_bounds__(kNT) k_chol(int ell, double* G, int* err) {
  __shared__ double sh[kWarps];
  __shared__ double diag;
  const int tid = threadIdx.x;
  for (long long idx = tid; idx < (long long)ell * ell; idx += kNT) {
    const int a = (int)(idx % ell), c = (int)(idx / ell);
    if (a < c) {
      const double s = 0.5 * (G[(size_t)c * ell + a] + G[(size_t)a * ell + c]);
      G[(size_t)c * ell + a] = s;
      G[(size_t)a * ell + c] = s;
    }
  }
  __syncthreads();
  for (int j = 0; j < ell; ++j) {
    const double* colj = G + (size_t)j * ell;       // entries (k, j), k < j hold C
    double v[1] = {0.0};
    for (int k = tid; k < j; k += kNT) v[0] = fma(colj[k], colj[k], v[0]);
    block_sum<kNT, 1>(v, sh);
    if (tid == 0) {
      const double s = G[(size_t)j * ell + j] - v[0];
      if (!(s > 0.0) || !isfinite(s)) {
        set_error(err, kErrCoreBreakdown);
        diag = 0.0;
      } else {
        diag = sqrt(s);
        G[(size_t)j * ell + j] = diag;
      }
    }
    __syncthreads();
    if (!(diag > 0.0)) return;
    for (int i = j + 1 + tid; i < ell; i += kNT) {
      const double* coli = G + (size_t)i * ell;
      double s = coli[j];
      for (int k = 0; k < j; ++k) s = fma(-colj[k], coli[k], s);
      G[(size_t)i * ell + j] = s / diag;
    }
    __syncthreads();
  }
  for (long long idx = tid; idx < (long long)ell * ell; idx += kNT) {
    const int a = (int)(idx % ell), c = (int)(idx / ell);
    if (a > c) G[(size_t)c * ell + a] = 0.0;
  }
}

// B = Y_nu C^{-1} in place, one thread per row: b_j = (y_j - sum_{k<j} b_k C_kj) / C_jj.
__global__ void __launch_bounds__(kNT) k_trsm_rows(int m, int ell, double* __restrict__ B, int ld,
                                                   const double* __restrict__ C, const int* err) {
  if (*err) return;
  const int i = blockIdx.x * kNT + threadIdx.x;
  if (i >= m) return;
  for (int j = 0; j < ell; ++j) {
    const double* cj = C + (size_t)j * ell;
    double s = B[(size_t)j * ld + i];
    for (int k = 0; k < j; ++k) s = fma(-B[(size_t)k * ld + i], __ldg(cj + k), s);
    B[(size_t)j * ld + i] = s / __ldg(cj + j);
  }
}

// One-sided Jacobi on the columns of B (m x ell).  Cooperative launch.
__global__ void __launch_bounds__(kNT) k_jacobi(int m, int ell, double* B, int ld, double tol,
                                                int* sweep_flags, int max_sweeps, unsigned* bar,
                                                int* err, int* sweeps_out) {
  __shared__ double sh[3 * kWarps];
  __shared__ int rotated;
  const int tid = threadIdx.x;
  const int lp = ell + (ell & 1);        // even number of players (one dummy if ell is odd)
  const int npairs = lp / 2;
  const int rounds = lp - 1;
  if (*err) return;                      // an earlier step failed (all blocks see the same word)
  if (tid == 0) rotated = 0;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    for (int r = 0; r < rounds; ++r) {
      for (int pi = blockIdx.x; pi < npairs; pi += gridDim.x) {
        int p, q;
        if (pi == 0) { p = r; q = lp - 1; }
        else { p = (r + pi) % (lp - 1); q = (r - pi + (lp - 1)) % (lp - 1); }
        if (p > q) { const int t = p; p = q; q = t; }
        if (q >= ell) continue;                        // pair with the dummy column
        double* bp = B + (size_t)p * ld;
        double* bq = B + (size_t)q * ld;
        double v[3] = {0.0, 0.0, 0.0};
        for (int i = tid; i < m; i += kNT) {
          const double x = __ldcg(bp + i), y = __ldcg(bq + i);
          v[0] = fma(x, x, v[0]);
          v[1] = fma(y, y, v[1]);
          v[2] = fma(x, y, v[2]);
        }
        block_sum<kNT, 3>(v, sh);
        const double al = v[0], be = v[1], ga = v[2];
        if (al > 0.0 && be > 0.0 && fabs(ga) > tol * sqrt(al) * sqrt(be)) {
          // Rotation that zeroes the inner product (Rutishauser's formulas).
          const double zeta = (be - al) / (2.0 * ga);
          double t;
          if (fabs(zeta) > 1e150) t = 0.5 / zeta;
          else t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(fma(zeta, zeta, 1.0)));
          const double c = 1.0 / sqrt(fma(t, t, 1.0));
          const double s = c * t;
          for (int i = tid; i < m; i += kNT) {
            const double x = __ldcg(bp + i), y = __ldcg(bq + i);
            __stcg(bp + i, c * x - s * y);
            __stcg(bq + i, s * x + c * y);
          }
          if (tid == 0) rotated = 1;
        }
      }
      if (!grid_barrier(bar, err)) return;
    }
    if (tid == 0 && rotated) { atomicOr(sweep_flags + sweep, 1); rotated = 0; }
    if (!grid_barrier(bar, err)) return;
    const int any = __ldcg(sweep_flags + sweep);
    if (!any) {
      if (blockIdx.x == 0 && tid == 0) *sweeps_out = sweep + 1;
      return;
    }
  }
  if (blockIdx.x == 0 && tid == 0) *sweeps_out = max_sweeps + 1;   // not converged
}

// G[j][j] += f * trace(G)  (one CTA): the shift of the first Cholesky-QR pass.
__global__ void __launch_bounds__(kNT) k_shift_trace(int ell, double* G, double f) {
  __shared__ double sh[kWarps];
  double v[1] = {0.0};
  for (int j = threadIdx.x; j < ell; j += kNT) v[0] += G[(size_t)j * ell + j];
  block_sum<kNT, 1>(v, sh);
  const double s = f * v[0];
  for (int j = threadIdx.x; j < ell; j += kNT) G[(size_t)j * ell + j] += s;
}

// out = Rn * Ra for upper-triangular ell x ell column-major matrices.
__global__ void k_trmm_upper(int ell, const double* __restrict__ Rn, const double* __restrict__ Ra,
                             double* __restrict__ out) {
  const long long idx = (long long)blockIdx.x * kNT + threadIdx.x;
  if (idx >= (long long)ell * ell) return;
  const int i = (int)(idx % ell), j = (int)(idx / ell);
  double s = 0.0;
  for (int k = i; k <= j; ++k) s = fma(Rn[(size_t)k * ell + i], Ra[(size_t)j * ell + k], s);
  out[(size_t)j * ell + i] = (i <= j) ? s : 0.0;
}

// Squared column norms, one block per column (fixed-order reduction).
__global__ void __launch_bounds__(kNT) k_colnorm2(int m, const double* __restrict__ B, int ld,
                                                  double* __restrict__ sumsq) {
  __shared__ double sh[kWarps];
  const double* b = B + (size_t)blockIdx.x * ld;
  double v[1] = {0.0};
  for (int i = threadIdx.x; i < m; i += kNT) v[0] = fma(b[i], b[i], v[0]);
  block_sum<kNT, 1>(v, sh);
  if (threadIdx.x == 0) sumsq[blockIdx.x] = v[0];
}

// Descending order (ties keep column order), lam = max(0, sigma^2 - nu).
__global__ void k_order(int ell, const double* __restrict__ sumsq, const double* sd,
                        int* __restrict__ perm, double* __restrict__ lam, const int* err) {
  if (*err) return;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ell) return;
  const double sj = sumsq[j];
  int rank = 0;
  for (int i = 0; i < ell; ++i) {
    const double si = sumsq[i];
    rank += (si > sj) || (si == sj && i < j);
  }
  perm[rank] = j;
  lam[rank] = fmax(0.0, sj - sd[SD_NU]);
}

__global__ void k_normalise(int m, int ell, const double* __restrict__ B, int ld,
                            const double* __restrict__ sumsq, const int* __restrict__ perm,
                            double* __restrict__ U, const int* err) {
  if (*err) return;
  const long long idx = (long long)blockIdx.x * kNT + threadIdx.x;
  if (idx >= (long long)m * ell) return;
  const int i = (int)(idx % m), r = (int)(idx / m);
  const int j = perm[r];
  const double s2 = sumsq[j];
  const double inv = s2 > 0.0 ? 1.0 / sqrt(s2) : 0.0;
  U[(size_t)r * ld + i] = B[(size_t)j * ld + i] * inv;
}

}  // namespace

cudaError_t nystrom_core_f64(cudaStream_t st, int m, int ell, const double* Y, const double* Om,
                             int ld, double* U, double* lam, double* sd, int* si, RedBuf red,
                             CoreWork cw, int num_sms) {
  int* err = si + SI_ERR;
  const long long total = (long long)m * ell;
  int fb = (int)((total + kNT - 1) / kNT);
  if (fb > 2 * num_sms) fb = 2 * num_sms;
  count_launches(1);
  k_frob<<<fb, kNT, 0, st>>>(m, ell, Y, ld, sd, err, red.part, red.cnt + 0);
  const unsigned eb = (unsigned)((total + kNT - 1) / kNT);
  count_launches(1);
  k_shift<<<eb, kNT, 0, st>>>(m, ell, Y, Om, ld, sd, cw.Ynu);
  // G = Omega^T Y_nu (ell x ell, column-major)
  cudaError_t e = gemm_f64(st, ell, ell, m, Om, ld, 1, cw.Ynu, 1, ld, nullptr, cw.G, 1, ell,
                           cw.split_buf, cw.split_cap);
  if (e != cudaSuccess) return e;
  count_launches(1);
  k_chol<<<1, kNT, 0, st>>>(ell, cw.G, err);
  count_launches(1);
  k_trsm_rows<<<(m + kNT - 1) / kNT, kNT, 0, st>>>(m, ell, cw.Ynu, ld, cw.G, err);
  double* Bsv = cw.Ynu;           // matrix whose column norms / directions give U and Sigma
  int jm = m, jld = ld;           // Jacobi problem: rows and leading dimension
  double* Jmat = cw.Ynu;
  if (ell > kJacobiDirectMaxEll) {
    // Large ell: B = Q R by a shifted three-pass Cholesky QR (the first pass
    // shifted by 1e-10 trace(B^T B) so it cannot break down), then the SVD of
    // the small ell x ell R by one-sided Jacobi, W = R V, and B V = Q W.
    for (int pass = 0; pass < 3; ++pass) {
      e = gemm_f64(st, ell, ell, m, cw.Ynu, ld, 1, cw.Ynu, 1, ld, nullptr, cw.G, 1, ell, cw.split_buf,
                   cw.split_cap);
      if (e != cudaSuccess) return e;
      if (pass == 0) {
        count_launches(1);
        k_shift_trace<<<1, kNT, 0, st>>>(ell, cw.G, 1e-10);
      }
      count_launches(1);
      k_chol<<<1, kNT, 0, st>>>(ell, cw.G, err);
      count_launches(1);
      k_trsm_rows<<<(m + kNT - 1) / kNT, kNT, 0, st>>>(m, ell, cw.Ynu, ld, cw.G, err);
      const unsigned sb = (unsigned)(((long long)ell * ell + kNT - 1) / kNT);
      if (pass == 0) {
        cudaMemcpyAsync(cw.R, cw.G, sizeof(double) * ell * ell, cudaMemcpyDeviceToDevice, st);
      } else {
        count_launches(1);
        k_trmm_upper<<<sb, kNT, 0, st>>>(ell, cw.G, cw.R, cw.Rt);
        cudaMemcpyAsync(cw.R, cw.Rt, sizeof(double) * ell * ell, cudaMemcpyDeviceToDevice, st);
      }
    }
    Jmat = cw.R;
    jm = ell;
    jld = ell;
  }
  // one-sided Jacobi (cooperative)
  cudaMemsetAsync(cw.sweep_flags, 0, sizeof(int) * CoreWork::kMaxSweeps, st);
  cudaMemsetAsync(cw.bar, 0, 2 * sizeof(unsigned), st);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jacobi, kNT, 0);
  int grid = (ell + 1) / 2;
  const int cap = per_sm * num_sms;
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  double tol = sqrt((double)jm) * 0x1.0p-53;
  if (tol < 0x1.0p-52) tol = 0x1.0p-52;
  int mm = jm, ee = ell, ldd = jld, ms = CoreWork::kMaxSweeps;
  double* Bp = Jmat;
  int* flags = cw.sweep_flags;
  unsigned* bar = cw.bar;
  int* sweeps = si + SI_SWEEPS;
  void* args[] = {&mm, &ee, &Bp, &ldd, &tol, &flags, &ms, &bar, &err, &sweeps};
  count_launches(1);
  e = cudaLaunchCooperativeKernel((const void*)k_jacobi, dim3(grid), dim3(kNT), args, 0, st);
  if (e != cudaSuccess) return e;
  if (ell > kJacobiDirectMaxEll) {
    // B V = Q W  (m x ell times ell x ell)
    e = gemm_f64(st, m, ell, ell, cw.Ynu, 1, ld, cw.R, 1, ell, nullptr, cw.B2, 1, ld, cw.split_buf,
                 cw.split_cap);
    if (e != cudaSuccess) return e;
    Bsv = cw.B2;
  }
  count_launches(1);
  k_colnorm2<<<ell, kNT, 0, st>>>(m, Bsv, ld, cw.sumsq);
  count_launches(1);
  k_order<<<(ell + 127) / 128, 128, 0, st>>>(ell, cw.sumsq, sd, cw.perm, lam, err);
  count_launches(1);
  k_normalise<<<eb, kNT, 0, st>>>(m, ell, Bsv, ld, cw.sumsq, cw.perm, U, err);
  return cudaGetLastError();
}

}  // namespace nys
