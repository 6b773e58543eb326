// Nystrom core factorisation (Algorithm 1, steps 3-8) in FP64:
//   nu = eps(||Y||_F);  Y_nu = Y + nu Omega;  G = Omega^T Y_nu (symmetrised);
//   C = chol(G) (upper, G = C^T C);  B = Y_nu C^{-1};  thin SVD of B;
//   lam = max(0, Sigma^2 - nu) in descending order, U = left singular vectors.
//
// The thin SVD is a one-sided (Hestenes) Jacobi iteration: each round
// rotates ell/2 disjoint column pairs in parallel (round-robin ordering), with
// a barrier between rounds.  One-sided Jacobi orthogonalises columns directly,
// so small singular values keep their relative accuracy (no Gram matrix, no
// squared condition number).  After convergence the column norms are the
// singular values and the normalised columns the left singular vectors.
// When B is nearly square (m <= 2 ell) and fits one CTA's shared memory it
// runs on B itself; otherwise on the triangular factor R of B = Q R (shifted
// three-pass Cholesky QR), and B V = Q (R V).  A sweep over B costs about
// 3.5 m ell^2 DFMAs, over R 3.5 ell^3, and the FP64 rate of one SM is the
// bound of the rotations, so the QR route wins as soon as m is a few times
// ell.  Matrices of up to 25600 entries are rotated by a single CTA in shared
// memory (__syncthreads between rounds); larger ones by the cooperative
// kernel with grid barriers.
#include <cooperative_groups.h>

#include "common.cuh"
#include "internal.h"

namespace nys {

namespace {

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

// The same factorisation with G in shared memory (ell <= 160), right-looking:
// for each j, the pivot's root and reciprocal root (independent, so their
// latencies overlap), row j of C scaled by the reciprocal, then a rank-one
// update of the trailing upper triangle.
constexpr int kCholSmemMax = 160;

__global__ void __launch_bounds__(kNT) k_chol_smem(int ell, double* G, int* err) {
  extern __shared__ double S[];          // ell x ell, column-major: (a, c) at c * ell + a
  __shared__ double piv[2];
  __shared__ int bad;
  const int tid = threadIdx.x;
  const int n2 = ell * ell;
  for (int idx = tid; idx < n2; idx += kNT) {
    const int a = idx % ell, c = idx / ell;
    S[idx] = a == c ? G[idx] : 0.5 * (G[(size_t)c * ell + a] + G[(size_t)a * ell + c]);
  }
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < ell; ++j) {
    if (tid == 0) {
      const double d = S[j * ell + j];
      if (!(d > 0.0) || !isfinite(d)) {
        bad = 1;
      } else {
        piv[0] = sqrt(d);
        piv[1] = rsqrt(d);
      }
    }
    __syncthreads();
    if (bad) break;
    const double inv = piv[1];
    for (int c = j + 1 + tid; c < ell; c += kNT) S[c * ell + j] *= inv;   // C(j, c)
    __syncthreads();
    if (tid == 0) S[j * ell + j] = piv[0];
    // S(a, c) -= C(j, a) C(j, c) for j < a <= c
    const int w = ell - j - 1;
    for (int idx = tid; idx < w * w; idx += kNT) {
      const int a = j + 1 + idx % w, c = j + 1 + idx / w;
      if (a <= c) S[c * ell + a] = fma(-S[a * ell + j], S[c * ell + j], S[c * ell + a]);
    }
    __syncthreads();
  }
  if (bad) {
    if (tid == 0) set_error(err, kErrCoreBreakdown);
    return;
  }
  for (int idx = tid; idx < n2; idx += kNT) {
    const int a = idx % ell, c = idx / ell;
    G[idx] = a <= c ? S[idx] : 0.0;
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

// The same substitution with the thread's row staged in shared memory
// (re-read from there instead of from global memory), the reciprocals of the
// diagonal computed once, and four partial sums per step; 128 rows per CTA,
// ell <= 200.
constexpr int kTrsmRows = 128;
constexpr int kTrsmSmemMax = 200;

__global__ void __launch_bounds__(kTrsmRows) k_trsm_smem(int m, int ell, double* __restrict__ B, int ld,
                                                         const double* __restrict__ C, const int* err) {
  extern __shared__ double sm[];         // rows: [ell][kTrsmRows], then 1 / C_jj
  double* rows = sm;
  double* invd = sm + (size_t)ell * kTrsmRows;
  if (*err) return;
  const int tid = threadIdx.x;
  for (int j = tid; j < ell; j += kTrsmRows) invd[j] = 1.0 / C[(size_t)j * ell + j];
  const int i = blockIdx.x * kTrsmRows + tid;
  const bool act = i < m;
  if (act)
    for (int j = 0; j < ell; ++j) rows[j * kTrsmRows + tid] = B[(size_t)j * ld + i];
  __syncthreads();
  if (!act) return;
  for (int j = 0; j < ell; ++j) {
    const double* cj = C + (size_t)j * ell;
    double s0 = rows[j * kTrsmRows + tid], s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int k = 0;
    for (; k + 4 <= j; k += 4) {
      s0 = fma(-rows[(k + 0) * kTrsmRows + tid], __ldg(cj + k + 0), s0);
      s1 = fma(-rows[(k + 1) * kTrsmRows + tid], __ldg(cj + k + 1), s1);
      s2 = fma(-rows[(k + 2) * kTrsmRows + tid], __ldg(cj + k + 2), s2);
      s3 = fma(-rows[(k + 3) * kTrsmRows + tid], __ldg(cj + k + 3), s3);
    }
    for (; k < j; ++k) s0 = fma(-rows[k * kTrsmRows + tid], __ldg(cj + k), s0);
    rows[j * kTrsmRows + tid] = ((s0 + s1) + (s2 + s3)) * invd[j];
  }
  for (int j = 0; j < ell; ++j) B[(size_t)j * ld + i] = rows[j * kTrsmRows + tid];
}

// One-sided Jacobi on the columns of B (m x ell).  Cooperative launch.
// Whether columns with squared norms al, be and inner product ga still need
// a rotation: |ga| > tol sqrt(al be), tested on squares when al be is in range
// (FP64 square roots and divisions have long latencies on this GPU).
__device__ __forceinline__ bool jacobi_needs_rotation(double al, double be, double ga, double tol) {
  if (!(al > 0.0) || !(be > 0.0)) return false;
  const double ab = al * be;
  if (ab > 0x1.0p-900 && ab < 0x1.0p+900) return ga * ga > (tol * tol) * ab;
  return fabs(ga) > tol * sqrt(al) * sqrt(be);
}

// Stopping rule shared by the Jacobi kernels.  A sweep stops the iteration
// when none of its rotations had a cosine |ga| / sqrt(al be) above 2^-30:
// cyclic Jacobi converges quadratically, so the cosines left after such a
// sweep are of order 2^-60, far below the rotation threshold `tol`
// (~sqrt(m) 2^-53), and the next sweep would rotate nothing.  (The classical
// rule, a whole sweep without rotations, costs that extra sweep.)  Returns
// 2 for a rotation above that bound, 1 for one below it.
__device__ __forceinline__ int jacobi_rotation_level(double al, double be, double ga) {
  const double ab = al * be;
  if (ab > 0x1.0p-900 && ab < 0x1.0p+900) return ga * ga > 0x1.0p-60 * ab ? 2 : 1;
  return fabs(ga) > 0x1.0p-30 * sqrt(al) * sqrt(be) ? 2 : 1;
}

// Rotation (c, s) that zeroes the inner product (Rutishauser's formulas):
// zeta = (be - al) / (2 ga), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
// c = 1 / sqrt(1 + t^2), s = c t.  Written as t = 2 ga sign(d) /
// (|d| + sqrt(d^2 + 4 ga^2)) with d = be - al (the same number, one root and
// one division instead of two of each; sign(0) = +1 reproduces the sign that
// zeta = +-0 gives) and c from a reciprocal square root.  For |zeta| > 2^13
// the first-order angle t = ga / d (jacobi_small_tangent) with c = 1 - t^2 / 2
// is used, which is
// orthogonal to double precision (c^2 (1 + t^2) = 1 - O(t^4), t^4 < 2^-56);
// its angle error leaves a residual inner product of relative size
// 1/(4 zeta^2) for the next sweep.  FP64 divisions and roots cost hundreds of
// cycles of latency each on this GPU, and a round waits for this chain.
// t = ga / d for the first-order branch.  The reciprocal of d starts from the
// FP32 reciprocal (2^-23 relative) and takes one Newton-Raphson step,
// r <- r (2 - d r), which squares the error (2^-46); exact division where d
// lies outside FP32's normal range.  The branch's own angle error is
// 1/(4 zeta^2) < 2^-28 relative, so 2^-46 changes nothing, and c, s below are
// orthogonal for any t.  (An FP64 division is a chain of several hundred
// cycles on this GPU, and every Jacobi round waits for it.)
__device__ __forceinline__ double jacobi_small_tangent(double ga, double d) {
  const double ad = fabs(d);
  if (ad > 0x1.0p-120 && ad < 0x1.0p+120) {
    double r = (double)__frcp_rn((float)d);
    r = fma(r, fma(-d, r, 1.0), r);
    return ga * r;
  }
  return ga / d;
}

__device__ __forceinline__ void jacobi_rotation(double al, double be, double ga, double& c, double& s) {
  const double d = be - al;
  if (fabs(d) > 16384.0 * fabs(ga)) {
    const double t = jacobi_small_tangent(ga, d);
    c = fma(-0.5 * t, t, 1.0);
    s = c * t;
    return;
  }
  const double h = fma(d, d, 4.0 * ga * ga);
  double t;
  if (isfinite(h)) {
    t = (2.0 * ga) * copysign(1.0, d == 0.0 ? 1.0 : d) / (fabs(d) + sqrt(h));
  } else {                       // squares out of range: the zeta form
    const double zeta = d / (2.0 * ga);
    t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(fma(zeta, zeta, 1.0)));
  }
  c = rsqrt(fma(t, t, 1.0));
  s = c * t;
}

// Sums of three values over a warp in six FP64 additions instead of fifteen
// (a warp-wide FP64 instruction costs a full pipe slot however few lanes
// it uses): the first two exchange levels give each lane one quantity, the
// last three finish it within groups of eight lanes.  On return lanes 0-7
// hold the sum of a, 8-15 that of b, 16-23 that of c.  Whole warp only.
__device__ __forceinline__ double warp_sum3(double a, double b, double c) {
  const int lane = threadIdx.x & 31;
  const bool lo = lane < 16;
  const double r1 = __shfl_xor_sync(0xffffffffu, lo ? c : a, 16);
  const double r2 = __shfl_xor_sync(0xffffffffu, lo ? 0.0 : b, 16);
  const double x = (lo ? a : c) + r1;
  const double y = (lo ? b : 0.0) + r2;
  const bool b3 = (lane & 8) != 0;
  double v = (b3 ? y : x) + __shfl_xor_sync(0xffffffffu, b3 ? x : y, 8);
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

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
        if (jacobi_needs_rotation(al, be, ga, tol)) {
          double c, s;
          jacobi_rotation(al, be, ga, c, s);
          for (int i = tid; i < m; i += kNT) {
            const double x = __ldcg(bp + i), y = __ldcg(bq + i);
            __stcg(bp + i, c * x - s * y);
            __stcg(bq + i, s * x + c * y);
          }
          if (tid == 0) rotated |= jacobi_rotation_level(al, be, ga);
        }
      }
      if (!grid_barrier(bar, err)) return;
    }
    if (tid == 0 && rotated) { atomicOr(sweep_flags + sweep, rotated); rotated = 0; }
    if (!grid_barrier(bar, err)) return;
    const int any = __ldcg(sweep_flags + sweep);
    if (!(any & 2)) {
      if (blockIdx.x == 0 && tid == 0) *sweeps_out = sweep + 1;
      return;
    }
  }
  if (blockIdx.x == 0 && tid == 0) *sweeps_out = max_sweeps + 1;   // not converged
}

// The same Jacobi iteration on one CTA with the matrix in shared memory, for
// matrices of up to kJacobiSmemElems entries: a warp per column pair, a
// __syncthreads between rounds instead of a grid barrier.  Pair order,
// rotation formulas and the stopping rule are those of k_jacobi.
constexpr int kJT = 1024;
constexpr int kJW = kJT / 32;
constexpr int kJacobiSmemElems = 25600;   // 200 KB of doubles

__global__ void __launch_bounds__(kJT) k_jacobi_smem(int m, int ell, double* B, int ld, double tol,
                                                     int max_sweeps, int* err, int* sweeps_out) {
  extern __shared__ double M[];          // m x ell, column-major, ld = m
  __shared__ int rotated;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (*err) return;
  for (long long e = tid; e < (long long)m * ell; e += kJT) {
    const int i = (int)(e % m), c = (int)(e / m);
    M[e] = B[(size_t)c * ld + i];
  }
  const int lp = ell + (ell & 1);
  const int npairs = lp / 2;
  const int rounds = lp - 1;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (tid == 0) rotated = 0;
    __syncthreads();
    for (int r = 0; r < rounds; ++r) {
      for (int pi = wid; pi < npairs; pi += kJW) {
        int p, q;
        if (pi == 0) { p = r; q = lp - 1; }
        else { p = (r + pi) % (lp - 1); q = (r - pi + (lp - 1)) % (lp - 1); }
        if (p > q) { const int t = p; p = q; q = t; }
        if (q >= ell) continue;
        double* bp = M + (size_t)p * m;
        double* bq = M + (size_t)q * m;
        double al = 0.0, be = 0.0, ga = 0.0, al2 = 0.0, be2 = 0.0, ga2 = 0.0;
        int i = lane;
        for (; i + 32 < m; i += 64) {
          const double x = bp[i], y = bq[i], x2 = bp[i + 32], y2 = bq[i + 32];
          al = fma(x, x, al);
          be = fma(y, y, be);
          ga = fma(x, y, ga);
          al2 = fma(x2, x2, al2);
          be2 = fma(y2, y2, be2);
          ga2 = fma(x2, y2, ga2);
        }
        if (i < m) {
          const double x = bp[i], y = bq[i];
          al = fma(x, x, al);
          be = fma(y, y, be);
          ga = fma(x, y, ga);
        }
        {
          const double v = warp_sum3(al + al2, be + be2, ga + ga2);
          al = __shfl_sync(0xffffffffu, v, 0);
          be = __shfl_sync(0xffffffffu, v, 8);
          ga = __shfl_sync(0xffffffffu, v, 16);
        }
        if (jacobi_needs_rotation(al, be, ga, tol)) {
          double c, sn;
          jacobi_rotation(al, be, ga, c, sn);
          for (int i = lane; i < m; i += 32) {
            const double x = bp[i], y = bq[i];
            bp[i] = c * x - sn * y;
            bq[i] = sn * x + c * y;
          }
          if (lane == 0) atomicOr(&rotated, jacobi_rotation_level(al, be, ga));
        }
      }
      __syncthreads();
    }
    if (!(rotated & 2)) break;
    __syncthreads();                     // everyone has read `rotated` before it is reset
  }
  for (long long e = tid; e < (long long)m * ell; e += kJT) {
    const int i = (int)(e % m), c = (int)(e / m);
    B[(size_t)c * ld + i] = M[e];
  }
  if (tid == 0) *sweeps_out = sweep < max_sweeps ? sweep + 1 : max_sweeps + 1;
}

// The same Jacobi iteration on a thread-block cluster, for ell <= 32: the
// rounds are latency chains of FP64 divisions and roots (hundreds of cycles
// each on this GPU), so each of the ceil(ell/2) pairs of a round gets its own
// CTA.  CTA k holds the two columns of pair k of the current round in shared
// memory (double-buffered), rotates them (all threads over the rows, one
// thread for the rotation), and after the round's cluster barrier pulls the
// two columns of its next pair from the CTAs that hold them, through
// distributed shared memory: 2m doubles move per CTA and round.  At the end
// of a sweep each CTA publishes whether it rotated and all CTAs stop on the
// same OR.  Same round-robin pair order, rotations and stopping rule as
// k_jacobi.
constexpr int kJC = 256;
constexpr int kJCW = kJC / 32;
constexpr int kJDW = 4;                  // warps that form the inner products
constexpr int kJacobiClusterMaxEll = 32;
constexpr int kJacobiClusterMaxRows = 6144;   // 4 columns of m doubles per CTA: 192 KB

// Pair pi of round r of the round-robin order on lp (even) players.
__device__ __forceinline__ void rr_pair(int pi, int r, int lp, int& p, int& q) {
  const int L = lp - 1;
  if (pi == 0) { p = r; q = lp - 1; }
  else { p = (r + pi) % L; q = (r - pi + L) % L; }
  if (p > q) { const int t = p; p = q; q = t; }
}

// Pair index that holds column j in round r.
__device__ __forceinline__ int rr_holder(int j, int r, int lp) {
  const int L = lp - 1;
  if (j == lp - 1) return 0;
  const int d = ((j - r) % L + L) % L;
  if (d == 0) return 0;
  return d <= (L - 1) / 2 ? d : L - d;
}

__global__ void __launch_bounds__(kJC) k_jacobi_cluster(int m, int ell, double* B, int ld, double tol,
                                                        int max_sweeps, const int* err, int* sweeps_out) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  extern __shared__ double buf[];        // [2 buffers][2 slots][m], then C sweep flags
  double* flags = buf + 4 * (size_t)m;
  __shared__ double red[3 * kJCW];
  __shared__ double rot[3];              // c, s, rotate?
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (*err) return;                      // every CTA reads the same word: all leave together
  const int lp = ell + (ell & 1);
  const int L = lp - 1;                  // rounds per sweep
  auto col = [&](int b, int slot) { return buf + ((size_t)b * 2 + slot) * m; };
  int cur = 0;
  {
    int p, q;
    rr_pair(rank, 0, lp, p, q);
    for (int i = tid; i < m; i += kJC) {
      col(0, 0)[i] = B[(size_t)p * ld + i];
      col(0, 1)[i] = q < ell ? B[(size_t)q * ld + i] : 0.0;
    }
  }
  cl.sync();
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    double mine = 0.0;
    for (int r = 0; r < L; ++r) {
      int p, q;
      rr_pair(rank, r, lp, p, q);
      if (q < ell) {
        double* bp = col(cur, 0);
        double* bq = col(cur, 1);
        // the three inner products over the rows: four warps (one per
        // sub-partition), packed warp sums, then lane 0 of warp 0 combines
        if (wid < kJDW) {
          double al = 0.0, be = 0.0, ga = 0.0;
          for (int i = tid; i < m; i += 32 * kJDW) {
            const double x = bp[i], y = bq[i];
            al = fma(x, x, al);
            be = fma(y, y, be);
            ga = fma(x, y, ga);
          }
          const double v = warp_sum3(al, be, ga);
          if (lane == 0) red[wid] = v;
          else if (lane == 8) red[kJCW + wid] = v;
          else if (lane == 16) red[2 * kJCW + wid] = v;
        }
        __syncthreads();
        if (wid == 0) {
          const int q8 = lane >> 3, r8 = lane & 7;
          double v = (q8 < 3 && r8 < kJDW) ? red[q8 * kJCW + r8] : 0.0;
#pragma unroll
          for (int o = 4; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
          const double a = v;
          const double b = __shfl_sync(0xffffffffu, v, 8);
          const double g = __shfl_sync(0xffffffffu, v, 16);
          if (lane == 0) {
            if (jacobi_needs_rotation(a, b, g, tol)) {
              double c, sn;
              jacobi_rotation(a, b, g, c, sn);
              rot[0] = c; rot[1] = sn; rot[2] = (double)jacobi_rotation_level(a, b, g);
            } else {
              rot[2] = 0.0;
            }
          }
        }
        __syncthreads();
        if (rot[2] != 0.0) {
          const double c = rot[0], sn = rot[1];
          for (int i = tid; i < m; i += kJC) {
            const double x = bp[i], y = bq[i];
            bp[i] = c * x - sn * y;
            bq[i] = sn * x + c * y;
          }
          mine = fmax(mine, rot[2]);
        }
      }
      cl.sync();                         // every rotation of round r is done
      // pull the two columns of the next round's pair from their holders
      const int rn = (r + 1) % L;
      int pn, qn;
      rr_pair(rank, rn, lp, pn, qn);
      const int nxt = cur ^ 1;
      for (int s = 0; s < 2; ++s) {
        const int j = s == 0 ? pn : qn;
        double* dst = col(nxt, s);
        if (j >= ell) {
          for (int i = tid; i < m; i += kJC) dst[i] = 0.0;
          continue;
        }
        const int h = rr_holder(j, r, lp);
        int hp, hq;
        rr_pair(h, r, lp, hp, hq);
        const double* src = cl.map_shared_rank(col(cur, j == hp ? 0 : 1), h);
        for (int i = tid; i < m; i += kJC) dst[i] = src[i];
      }
      cur = nxt;
      __syncthreads();                   // rot[] and red[] are rewritten next round
    }
    if (tid < C) *cl.map_shared_rank(flags + rank, tid) = mine;
    cl.sync();
    double any = 0.0;
    for (int k = 0; k < C; ++k) any = fmax(any, flags[k]);
    if (any < 2.0) break;
  }
  // the columns of round 0's pairs are current in every CTA: write them back
  {
    int p, q;
    rr_pair(rank, 0, lp, p, q);
    for (int i = tid; i < m; i += kJC) {
      B[(size_t)p * ld + i] = col(cur, 0)[i];
      if (q < ell) B[(size_t)q * ld + i] = col(cur, 1)[i];
    }
  }
  if (rank == 0 && tid == 0) *sweeps_out = sweep < max_sweeps ? sweep + 1 : max_sweeps + 1;
  cl.sync();                             // no CTA leaves while a peer may still read its columns
}

// Mixed-precision start of the one-sided Jacobi SVD (2 <= ell <= 32).  The
// same round-robin iteration runs first in FP32 on a copy of B (FP32
// arithmetic is ~70x the FP64 rate on this GPU, and its roots and divisions
// are single instructions), one warp per column pair, the rotations
// accumulated in V (ell x ell).  V is then made orthogonal to FP64 precision
// by two Newton-Schulz steps in FP64, X <- X (3I - X^T X) / 2 (quadratic:
// an FP32-level defect of ~1e-6 falls below 1e-16), and written out.  B V has
// the singular values and left singular vectors of B (V is orthogonal) and
// nearly orthogonal columns, so the FP64 Jacobi that follows needs two or
// three sweeps instead of six to nine.  B is scaled by a power of two so that
// its largest column norm is about 1 (the FP32 copy keeps small columns in
// range).  The FP32 sweeps stop after a sweep without a rotation whose
// cosine exceeds 2^-9 (kJ32Quad), or after max_sweeps; a pair needs a
// rotation when its inner product exceeds kJ32Tol times the geometric mean
// of its squared norms and also kJ32Noise times the
// largest squared column norm (below that, FP32 rounding of the big columns
// dominates and the FP64 sweeps must decide anyway).
constexpr int kJ32T = 512;
constexpr int kJ32W = kJ32T / 32;
constexpr int kJ32MaxElems = 40960;      // m * ell floats of the copy (160 KB)
constexpr float kJ32Tol = 1e-5f;
constexpr float kJ32Noise = 1e-6f;
// Quadratic stop, as in the FP64 kernels: a sweep whose rotations all had a
// cosine below 2^-9 (squared: 2^-18) leaves cosines near kJ32Tol, so no
// confirming sweep follows it.
constexpr float kJ32Quad = 0x1.0p-18f;

__global__ void __launch_bounds__(kJ32T) k_jacobi_f32_start(int m, int ell, const double* __restrict__ B, int ld,
                                                            double* __restrict__ V, int max_sweeps,
                                                            const int* err) {
  extern __shared__ float F[];           // m x ell copy of B (column-major, ld m), then V32 (ell x ell)
  float* V32 = F + (size_t)m * ell;
  __shared__ double X[32 * 32], W[32 * 32];
  __shared__ float colmax[kJ32W];
  __shared__ int rotated;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (*err) return;
  // power-of-two scale from the largest entry
  float mx = 0.0f;
  for (long long e = tid; e < (long long)m * ell; e += kJ32T) {
    const int i = (int)(e % m), c = (int)(e / m);
    mx = fmaxf(mx, (float)fabs(B[(size_t)c * ld + i]));
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) colmax[wid] = mx;
  __syncthreads();
  mx = 0.0f;
  for (int w = 0; w < kJ32W; ++w) mx = fmaxf(mx, colmax[w]);
  int ex = 0;
  if (mx > 0.0f && isfinite(mx)) frexpf(mx, &ex);
  const double scale = ldexp(1.0, -ex);
  for (long long e = tid; e < (long long)m * ell; e += kJ32T) {
    const int i = (int)(e % m), c = (int)(e / m);
    F[e] = (float)(B[(size_t)c * ld + i] * scale);
  }
  for (int e = tid; e < ell * ell; e += kJ32T) V32[e] = (e % ell == e / ell) ? 1.0f : 0.0f;
  __syncthreads();
  // largest squared column norm of the scaled copy: the FP32 noise level
  float cm = 0.0f;
  for (int c = wid; c < ell; c += kJ32W) {
    float a = 0.0f;
    for (int i = lane; i < m; i += 32) a = fmaf(F[(size_t)c * m + i], F[(size_t)c * m + i], a);
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    cm = fmaxf(cm, a);
  }
  if (lane == 0) colmax[wid] = cm;
  __syncthreads();
  cm = 0.0f;
  for (int w = 0; w < kJ32W; ++w) cm = fmaxf(cm, colmax[w]);
  const float noise = kJ32Noise * cm;
  const int lp = ell + (ell & 1);
  const int npairs = lp / 2;
  const int L = lp - 1;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (tid == 0) rotated = 0;
    __syncthreads();
    for (int r = 0; r < L; ++r) {
      if (wid < npairs) {
        int p, q;
        rr_pair(wid, r, lp, p, q);
        if (q < ell) {
          float* bp = F + (size_t)p * m;
          float* bq = F + (size_t)q * m;
          float al = 0.0f, be = 0.0f, ga = 0.0f;
#pragma unroll 4
          for (int i = lane; i < m; i += 32) {
            const float x = bp[i], y = bq[i];
            al = fmaf(x, x, al);
            be = fmaf(y, y, be);
            ga = fmaf(x, y, ga);
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            al += __shfl_xor_sync(0xffffffffu, al, o);
            be += __shfl_xor_sync(0xffffffffu, be, o);
            ga += __shfl_xor_sync(0xffffffffu, ga, o);
          }
          // |ga| > tol sqrt(al be), on squares (al, be <= ~1 after the scaling;
          // a product that underflows is left to the noise test)
          if (al > 0.0f && be > 0.0f && ga * ga > (kJ32Tol * kJ32Tol) * (al * be) && fabsf(ga) > noise) {
            const float d = be - al;
            const float h = fmaf(d, d, 4.0f * ga * ga);
            // the tangent needs no correct rounding: c and s below are
            // orthogonal for any t, a slightly wrong angle is undone later
            const float t = __fdividef((2.0f * ga) * copysignf(1.0f, d == 0.0f ? 1.0f : d), fabsf(d) + sqrtf(h));
            const float c = rsqrtf(fmaf(t, t, 1.0f));
            const float sn = c * t;
            if (lane == 0) atomicOr(&rotated, ga * ga > kJ32Quad * (al * be) ? 2 : 1);
#pragma unroll 4
            for (int i = lane; i < m; i += 32) {
              const float x = bp[i], y = bq[i];
              bp[i] = c * x - sn * y;
              bq[i] = sn * x + c * y;
            }
            if (lane < ell) {
              float* vp = V32 + (size_t)p * ell;
              float* vq = V32 + (size_t)q * ell;
              const float x = vp[lane], y = vq[lane];
              vp[lane] = c * x - sn * y;
              vq[lane] = sn * x + c * y;
            }
          }
        }
      }
      __syncthreads();
    }
    if (!(rotated & 2)) break;
    __syncthreads();                     // everyone has read `rotated` before it is reset
  }
  // Newton-Schulz in FP64: X <- 1.5 X - 0.5 X (X^T X), twice
  for (int e = tid; e < ell * ell; e += kJ32T) X[e] = (double)V32[e];
  __syncthreads();
  for (int it = 0; it < 2; ++it) {
    for (int e = tid; e < ell * ell; e += kJ32T) {          // W = X^T X, (a, b) at b * ell + a
      const int a = e % ell, b = e / ell;
      const double* xa = X + (size_t)a * ell;
      const double* xb = X + (size_t)b * ell;
      double s0 = 0.0, s1 = 0.0;
      int k = 0;
      for (; k + 1 < ell; k += 2) {
        s0 = fma(xa[k], xb[k], s0);
        s1 = fma(xa[k + 1], xb[k + 1], s1);
      }
      if (k < ell) s0 = fma(xa[k], xb[k], s0);
      W[e] = s0 + s1;
    }
    __syncthreads();
    double nx[2] = {0.0, 0.0};
    for (int e = tid, u = 0; e < ell * ell; e += kJ32T, ++u) {  // (X W)(i, j) at j * ell + i
      const int i = e % ell, j = e / ell;
      const double* wj = W + (size_t)j * ell;
      double s0 = 0.0, s1 = 0.0;
      int k = 0;
      for (; k + 1 < ell; k += 2) {
        s0 = fma(X[(size_t)k * ell + i], wj[k], s0);
        s1 = fma(X[(size_t)(k + 1) * ell + i], wj[k + 1], s1);
      }
      if (k < ell) s0 = fma(X[(size_t)k * ell + i], wj[k], s0);
      nx[u] = fma(-0.5, s0 + s1, 1.5 * X[e]);
    }
    __syncthreads();
    for (int e = tid, u = 0; e < ell * ell; e += kJ32T, ++u) X[e] = nx[u];
    __syncthreads();
  }
  for (int e = tid; e < ell * ell; e += kJ32T) V[e] = X[e];
}

// FP64 cleanup after the FP32 start, on the Gram matrix instead of on B2:
// B2 = B V0 has nearly orthogonal columns (cosines at the FP32 start's
// tolerance), so G = B2^T B2 = S A S with S = diag of the column norms and A
// within ~1e-5 of the identity.  Two-sided cyclic Jacobi on such a matrix
// keeps the high relative accuracy of one-sided Jacobi on B2: it depends on
// the condition of A (about 1), and forming G in FP64 perturbs A by ~m eps.
// The rotations are those of the one-sided iteration (the same pair order,
// the same (c, s) from (g_pp, g_qq, g_pq) as from the squared norms and the
// inner product, the same stopping rule), so B2 V1 with V1 the accumulated
// rotations is what the FP64 one-sided sweeps on B2 would converge to.  The
// matrix is ell x ell (ell <= 32): the whole iteration runs in one CTA, no
// inner products over the m rows and no cluster barriers; the ceil(ell/2)
// rotations of a round are computed side by side by the lanes of one warp.
// G's upper triangle is read (the lower one mirrored); V1 is written.
constexpr int kJG = 512;

__global__ void __launch_bounds__(kJG) k_jacobi_gram(int ell, const double* __restrict__ G, double* __restrict__ V,
                                                   double tol, int max_sweeps, const int* err, int* sweeps_out) {
  constexpr int ld = 33;                 // padded column stride
  __shared__ double Gs[32 * ld], Vs[32 * ld];
  __shared__ double rc[2][16], rs[2][16];   // rotations of a round, double-buffered by round parity
  __shared__ int rp[2][16], rq[2][16], on[2][16];
  __shared__ unsigned char bk1[136], bk2[136];   // pair blocks (k1 <= k2) of the symmetric update
  __shared__ int level;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (*err) return;
  for (int e = tid; e < ell * ell; e += kJG) {
    const int i = e % ell, j = e / ell;
    Gs[j * ld + i] = i <= j ? G[(size_t)j * ell + i] : G[(size_t)i * ell + j];
    Vs[j * ld + i] = i == j ? 1.0 : 0.0;
  }
  const int lp = ell + (ell & 1);
  const int npairs = lp / 2;
  const int nblk = npairs * (npairs + 1) / 2;
  const int L = lp - 1;
  if (tid == 0) {
    int e = 0;
    for (int k1 = 0; k1 < npairs; ++k1)
      for (int k2 = k1; k2 < npairs; ++k2) { bk1[e] = (unsigned char)k1; bk2[e] = (unsigned char)k2; ++e; }
  }
  // V <- V J for the rotations in buffer b (threads from `first` on)
  auto v_update = [&](int b, int first, int stride) {
    for (int e = tid - first; e >= 0 && e < npairs * ell; e += stride) {
      const int k = e / ell, i = e - k * ell;
      if (!on[b][k]) continue;
      const int p = rp[b][k], q = rq[b][k];
      const double c = rc[b][k], sn = rs[b][k];
      const double x = Vs[p * ld + i], y = Vs[q * ld + i];
      Vs[p * ld + i] = c * x - sn * y;
      Vs[q * ld + i] = sn * x + c * y;
    }
  };
  int sweep = 0, buf = 0;
  bool pending = false;                  // the V update of the last round is still to do
  for (; sweep < max_sweeps; ++sweep) {
    if (tid == 0) level = 0;
    __syncthreads();
    for (int r = 0; r < L; ++r) {
      if (wid == 0) {
        if (lane < npairs) {
          int p, q;
          rr_pair(lane, r, lp, p, q);
          int rot = 0;
          double c = 1.0, sn = 0.0;
          if (q < ell) {
            const double a = Gs[p * ld + p], bb = Gs[q * ld + q], g = Gs[q * ld + p];
            if (jacobi_needs_rotation(a, bb, g, tol)) {
              jacobi_rotation(a, bb, g, c, sn);
              rot = 1;
              atomicOr(&level, jacobi_rotation_level(a, bb, g));
            }
          }
          rp[buf][lane] = p;
          rq[buf][lane] = q;
          rc[buf][lane] = c;
          rs[buf][lane] = sn;
          on[buf][lane] = rot;
        }
      } else if (pending) {
        // the previous round's rotations of V, while warp 0 forms this round's
        v_update(buf ^ 1, 32, kJG - 32);
      }
      __syncthreads();
      // G <- J^T G J, one 2 x 2 block (rows of pair k1, columns of pair k2,
      // k1 <= k2) per thread, mirrored below the diagonal
      for (int e = tid; e < nblk; e += kJG) {
        const int k1 = bk1[e], k2 = bk2[e];
        if (!on[buf][k1] && !on[buf][k2]) continue;
        const int a0 = rp[buf][k1], a1 = rq[buf][k1], b0 = rp[buf][k2], b1 = rq[buf][k2];
        const double c1 = rc[buf][k1], s1 = rs[buf][k1], c2 = rc[buf][k2], s2 = rs[buf][k2];
        const bool ra = a1 < ell, rb = b1 < ell;    // the second index of a pair may be the dummy
        const double g00 = Gs[b0 * ld + a0];
        const double g01 = rb ? Gs[b1 * ld + a0] : 0.0;
        const double g10 = ra ? Gs[b0 * ld + a1] : 0.0;
        const double g11 = (ra && rb) ? Gs[b1 * ld + a1] : 0.0;
        // X = G J2 (columns), then J1^T X (rows)
        const double x00 = c2 * g00 - s2 * g01, x01 = s2 * g00 + c2 * g01;
        const double x10 = c2 * g10 - s2 * g11, x11 = s2 * g10 + c2 * g11;
        const double y00 = c1 * x00 - s1 * x10, y10 = s1 * x00 + c1 * x10;
        const double y01 = c1 * x01 - s1 * x11, y11 = s1 * x01 + c1 * x11;
        Gs[b0 * ld + a0] = y00;
        Gs[a0 * ld + b0] = y00;
        if (rb) { Gs[b1 * ld + a0] = y01; Gs[a0 * ld + b1] = y01; }
        if (ra) { Gs[b0 * ld + a1] = y10; Gs[a1 * ld + b0] = y10; }
        if (ra && rb) { Gs[b1 * ld + a1] = y11; Gs[a1 * ld + b1] = y11; }
      }
      pending = true;
      buf ^= 1;
      __syncthreads();
    }
    if (!(level & 2)) break;
    __syncthreads();                     // everyone has read `level` before it is reset
  }
  if (pending) {
    v_update(buf ^ 1, 0, kJG);
    __syncthreads();
  }
  for (int e = tid; e < ell * ell; e += kJG) {
    const int i = e % ell, j = e / ell;
    V[(size_t)j * ell + i] = Vs[j * ld + i];
  }
  if (tid == 0) *sweeps_out = sweep < max_sweeps ? sweep + 1 : max_sweeps + 1;
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

// Cholesky of the ell x ell core (shared memory when it fits).
cudaError_t launch_chol(cudaStream_t st, int ell, double* G, int* err) {
  count_launches(1);
  if (ell <= kCholSmemMax) {
    const size_t sm = sizeof(double) * (size_t)ell * ell;
    cudaError_t e = cudaFuncSetAttribute(k_chol_smem, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(sizeof(double) * kCholSmemMax * kCholSmemMax));
    if (e != cudaSuccess) return e;
    k_chol_smem<<<1, kNT, sm, st>>>(ell, G, err);
  } else {
    k_chol<<<1, kNT, 0, st>>>(ell, G, err);
  }
  return cudaGetLastError();
}

// B = B C^{-1} for an m x ell B (column-major, ld) and upper-triangular C.
cudaError_t launch_trsm(cudaStream_t st, int m, int ell, double* B, int ld, const double* C, int* err) {
  count_launches(1);
  if (ell <= kTrsmSmemMax) {
    const size_t sm = sizeof(double) * ((size_t)ell * kTrsmRows + ell);
    cudaError_t e = cudaFuncSetAttribute(k_trsm_smem, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(sizeof(double) * ((size_t)kTrsmSmemMax * kTrsmRows + kTrsmSmemMax)));
    if (e != cudaSuccess) return e;
    k_trsm_smem<<<(m + kTrsmRows - 1) / kTrsmRows, kTrsmRows, sm, st>>>(m, ell, B, ld, C, err);
  } else {
    k_trsm_rows<<<(m + kNT - 1) / kNT, kNT, 0, st>>>(m, ell, B, ld, C, err);
  }
  return cudaGetLastError();
}

}  // namespace

bool nystrom_core_capturable(int m, int ell) {
  // the direct route (no Cholesky QR copies) with the cluster or one-CTA Jacobi
  const bool direct = (ell <= kJacobiClusterMaxEll && ell >= 2 && m <= kJacobiClusterMaxRows) ||
                      (m <= 2 * ell && (long long)m * ell <= kJacobiSmemElems);
  if (!direct) return false;
  return (ell <= kJacobiClusterMaxEll && ell >= 2 && m <= kJacobiClusterMaxRows) ||
         (long long)m * ell <= kJacobiSmemElems;
}

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
  e = launch_chol(st, ell, cw.G, err);
  if (e != cudaSuccess) return e;
  e = launch_trsm(st, m, ell, cw.Ynu, ld, cw.G, err);
  if (e != cudaSuccess) return e;
  double* Bsv = cw.Ynu;           // matrix whose column norms / directions give U and Sigma
  int jm = m, jld = ld;           // Jacobi problem: rows and leading dimension
  double* Jmat = cw.Ynu;
  // direct on B when the cluster Jacobi takes it (ell <= 32, one CTA per
  // pair), or when B is nearly square; otherwise through a QR of B
  const bool direct = (ell <= kJacobiClusterMaxEll && ell >= 2 && m <= kJacobiClusterMaxRows) ||
                      (m <= 2 * ell && (long long)m * ell <= kJacobiSmemElems);
  if (!direct) {
    // B = Q R by a shifted three-pass Cholesky QR (the first pass
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
      e = launch_chol(st, ell, cw.G, err);
      if (e != cudaSuccess) return e;
      e = launch_trsm(st, m, ell, cw.Ynu, ld, cw.G, err);
      if (e != cudaSuccess) return e;
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
  const bool f32 =
      direct && cw.f32_start && ell >= 2 && ell <= kJacobiClusterMaxEll && (long long)m * ell <= kJ32MaxElems;
  if (f32) {
    // FP32 Jacobi start: V (orthogonal to FP64 precision) in cw.R, then the
    // FP64 Jacobi runs on B2 = B V
    const size_t sm = sizeof(float) * ((size_t)m * ell + (size_t)ell * ell);
    e = cudaFuncSetAttribute(k_jacobi_f32_start, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(float) * (kJ32MaxElems + 32 * 32)));
    if (e != cudaSuccess) return e;
    count_launches(1);
    k_jacobi_f32_start<<<1, kJ32T, sm, st>>>(m, ell, cw.Ynu, ld, cw.R, 8, err);
    e = gemm_f64(st, m, ell, ell, cw.Ynu, 1, ld, cw.R, 1, ell, nullptr, cw.B2, 1, ld, cw.split_buf,
                 cw.split_cap);
    if (e != cudaSuccess) return e;
    Jmat = cw.B2;
    Bsv = cw.B2;
  }
  double tol = sqrt((double)jm) * 0x1.0p-53;
  if (tol < 0x1.0p-52) tol = 0x1.0p-52;
  if (f32 && cw.gram) {
    // FP64 sweeps on G2 = B2^T B2 (one CTA), then B3 = B2 V1 into Ynu
    e = gemm_f64(st, ell, ell, m, cw.B2, ld, 1, cw.B2, 1, ld, nullptr, cw.G, 1, ell, cw.split_buf, cw.split_cap);
    if (e != cudaSuccess) return e;
    count_launches(1);
    k_jacobi_gram<<<1, kJG, 0, st>>>(ell, cw.G, cw.Rt, tol, CoreWork::kMaxSweeps, err, si + SI_SWEEPS);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = gemm_f64(st, m, ell, ell, cw.B2, 1, ld, cw.Rt, 1, ell, nullptr, cw.Ynu, 1, ld, cw.split_buf,
                 cw.split_cap);
    Bsv = cw.Ynu;
  } else if (ell <= kJacobiClusterMaxEll && ell >= 2 && jm <= kJacobiClusterMaxRows) {
    // one CTA per column pair of a round, in one thread-block cluster
    const int C = (ell + 1) / 2;
    const size_t sm = sizeof(double) * (4 * (size_t)jm + C);
    e = cudaFuncSetAttribute(k_jacobi_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(double) * (4 * (size_t)kJacobiClusterMaxRows + 16)));
    if (e != cudaSuccess) return e;
    if (C > 8) {
      e = cudaFuncSetAttribute(k_jacobi_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)C);
    cfg.blockDim = dim3(kJC);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    count_launches(1);
    e = cudaLaunchKernelEx(&cfg, k_jacobi_cluster, jm, ell, Jmat, jld, tol, (int)CoreWork::kMaxSweeps,
                           (const int*)err, si + SI_SWEEPS);
  } else if ((long long)jm * ell <= kJacobiSmemElems) {
    // one-sided Jacobi in one CTA's shared memory
    const size_t sm = sizeof(double) * (size_t)jm * ell;
    // the attribute is set to the kernel's maximum, never lowered: handles on
    // other host threads may be launching it concurrently
    e = cudaFuncSetAttribute(k_jacobi_smem, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(double) * kJacobiSmemElems));
    if (e != cudaSuccess) return e;
    count_launches(1);
    k_jacobi_smem<<<1, kJT, sm, st>>>(jm, ell, Jmat, jld, tol, CoreWork::kMaxSweeps, err, si + SI_SWEEPS);
  } else {
    // one-sided Jacobi (cooperative)
    cudaMemsetAsync(cw.sweep_flags, 0, sizeof(int) * CoreWork::kMaxSweeps, st);
    cudaMemsetAsync(cw.bar, 0, 2 * sizeof(unsigned), st);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jacobi, kNT, 0);
    int grid = (ell + 1) / 2;
    const int cap = per_sm * num_sms;
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    int mm = jm, ee = ell, ldd = jld, ms = CoreWork::kMaxSweeps;
    double* Bp = Jmat;
    int* flags = cw.sweep_flags;
    unsigned* bar = cw.bar;
    int* sweeps = si + SI_SWEEPS;
    void* args[] = {&mm, &ee, &Bp, &ldd, &tol, &flags, &ms, &bar, &err, &sweeps};
    count_launches(1);
    e = cudaLaunchCooperativeKernel((const void*)k_jacobi, dim3(grid), dim3(kNT), args, 0, st);
  }
  if (e != cudaSuccess) return e;
  if (!direct) {
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
