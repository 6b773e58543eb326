// Whole Nystrom-PCG solves inside one thread-block cluster, for small QPs.
//
// A PCG iteration of a small system (A of a few hundred KB) is far too little
// work for the whole GPU: issued as kernels it is bound by launch latency, and
// in a grid-wide cooperative kernel by grid-barrier latency.  Here one
// cluster of C CTAs (C <= 16, on C SMs of one GPC) runs the whole CG loop.
// The CTAs synchronise through the cluster's hardware barrier and exchange
// partial sums through distributed shared memory, so no step of an iteration
// touches global memory except the reads of A when A does not fit on chip.
//
// Partition: CTA k owns the column band [j0, j1) of A (for t = D .* A^T p,
// which then needs no cross-CTA sum) and the row band [i0, i1) of every
// m-vector (x, r, w, z and the rows of U).  Its slice A[:, j0:j1] is kept in
// shared memory when it fits (kAS), else read from global memory (L2).  Every
// CTA holds the full search direction p.  One iteration (Algorithm 2 / the
// textbook PCG recurrences of the multi-kernel path):
//
//   p = z + beta p                      all rows, every CTA (z is replicated)
//   t = D_k .* (A_k^T p)                own columns
//   q_k = A_k t                         all rows: partial of A t over own columns
//   -- cluster barrier 1
//   w = delta p + sum_k q_k             own rows (fixed order over k); partial p^T w
//   -- cluster barrier 2                -> alpha = r^T z / p^T w
//   x += alpha p, r -= alpha w          own rows; partials of U^T r and r^T r
//   -- cluster barrier 3                -> s = U^T r, ||r||^2, stop test
//   z = r + U (wts .* s)                own rows, pushed into every CTA's copy; partial r^T z
//   -- cluster barrier 4                -> beta
//
// Every cross-CTA sum is taken by every CTA over the same partials in the same
// order, so all CTAs reach bit-identical scalars and take the same branches:
// the number of cluster barriers each CTA passes is the same by construction,
// and there is no spin-wait.  The stop rule is the multi-kernel path's
// (relative residual tested after each update, forced counts, max_iter).
#include <cooperative_groups.h>

#include "common.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

namespace nys {

namespace {

constexpr int kCT = 256;
constexpr int kCW = kCT / 32;
constexpr int kChunk = 128;             // columns per pass of the A^T p loop (4 per lane)
constexpr int kMaxC = 16;
constexpr size_t kSmemCap = 226 * 1024; // dynamic shared memory per CTA (static use is < 1 KB)

// Shared-memory layout of one CTA, in doubles.  Computed identically on the
// host (to size the launch) and on the device.
struct Layout {
  int rb, cbw, ncp;
  size_t oA, oP, oZ, oT, oDl, oX, oR, oW, oU, oWs, oWss, oQin, oUtIn, oPwIn, oRzIn, oRed, oBc, total;
};

__host__ __device__ inline Layout make_layout(int m, int n, int ell, int C, bool a_smem) {
  Layout L;
  L.rb = (m + C - 1) / C;
  L.cbw = (n + C - 1) / C;
  L.ncp = L.cbw | 1;                    // odd row stride: row-parallel reads hit distinct banks
  size_t o = 0;
  L.oA = o; o += a_smem ? (size_t)m * L.ncp : 0;
  L.oP = o; o += m;                     // search direction, all rows
  L.oZ = o; o += m;                     // preconditioned residual, all rows (pushed by owners)
  L.oT = o; o += L.cbw;                 // t = D .* A^T p, own columns
  L.oDl = o; o += L.cbw;                // D, own columns
  L.oX = o; o += L.rb;                  // x, r, w: own rows
  L.oR = o; o += L.rb;
  L.oW = o; o += L.rb;
  L.oU = o; o += (size_t)L.rb * ell;   // own rows of U, column-major (ld = rb)
  L.oWs = o; o += ell;                  // (lam_ell + delta) / (lam + delta) - 1
  L.oWss = o; o += ell;                 // ws .* (U^T r)
  L.oQin = o; o += (size_t)C * L.rb;   // [k][row]: CTA k's partial of A t on own rows
  L.oUtIn = o; o += (size_t)C * (ell + 1);  // [k][c]: CTA k's partials of U^T r, ||r||^2
  L.oPwIn = o; o += C;                  // [k]: partials of p^T w
  L.oRzIn = o; o += C;                  // [k]: partials of r^T z
  L.oRed = o; o += (size_t)kCW * kChunk;
  L.oBc = o; o += 8;                    // scalars broadcast inside the CTA
  L.total = o;
  return L;
}

// Fixed pairwise tree over C (<= 16) values: every CTA that sums the same
// values gets the same bits.
__device__ __forceinline__ double tree_sum(const double* v, int C, size_t stride = 1) {
  double a[kMaxC];
#pragma unroll
  for (int k = 0; k < kMaxC; ++k) a[k] = k < C ? v[(size_t)k * stride] : 0.0;
#pragma unroll
  for (int s = 1; s < kMaxC; s <<= 1)
#pragma unroll
    for (int k = 0; k + s < kMaxC; k += 2 * s) a[k] += a[k + s];
  return a[0];
}

// Partial sum of the values k in [4w, 4w + 4) (those below C) of a strided
// array, as ((v0 + v1) + (v2 + v3)): four warps each take one quarter, and
// (g0 + g1) + (g2 + g3) then reproduces tree_sum's order exactly.
__device__ __forceinline__ double quad_sum(const double* v, int C, size_t stride, int w) {
  double a[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int idx = 4 * w + k;
    a[k] = idx < C ? v[(size_t)idx * stride] : 0.0;
  }
  return (a[0] + a[1]) + (a[2] + a[3]);
}

// Sum of C (<= 16) values with one per lane (a fixed xor tree of four
// levels), broadcast from lane 0; called by a whole warp.
__device__ __forceinline__ double lane_sum(const double* v, int C, int lane) {
  double x = lane < C ? v[lane] : 0.0;
#pragma unroll
  for (int o = kMaxC / 2; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return __shfl_sync(0xffffffffu, x, 0);
}

// Push one value into slot `rank` of array `arr` in every CTA of the cluster
// (lanes 0..C-1 of the calling warp store lane 0's value, so every CTA
// receives the same bits: all CTAs must reach identical scalars, or their
// branch decisions, and with them their cluster-barrier counts, would differ).
__device__ __forceinline__ void push_all(cg::cluster_group& cl, double* arr, int rank, double v, int C, int lane) {
  v = __shfl_sync(0xffffffffu, v, 0);
  if (lane < C) *cl.map_shared_rank(arr + rank, lane) = v;
}

template <bool kAS>
__global__ void __launch_bounds__(kCT, kAS ? 1 : 3) k_pcg_cluster(ClusterPcgTask t0, const ClusterPcgTask* tasks) {
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const ClusterPcgTask T = tasks ? tasks[blockIdx.x / C] : t0;
  unsigned long long t_start = 0;
  if (T.t_ns && rank == 0 && threadIdx.x == 0) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_start));
  extern __shared__ double smem[];
  __shared__ double sh[kCW];
  const int m = T.m, n = T.n, ell = T.ell;
  const Layout L = make_layout(m, n, ell, C, kAS);
  double* As = smem + L.oA;
  double* P = smem + L.oP;
  double* Zf = smem + L.oZ;
  double* Ts = smem + L.oT;
  double* Dl = smem + L.oDl;
  double* Xb = smem + L.oX;
  double* Rb = smem + L.oR;
  double* Wb = smem + L.oW;
  double* Ub = smem + L.oU;
  double* ws = smem + L.oWs;
  double* wss = smem + L.oWss;
  double* Qin = smem + L.oQin;
  double* UtIn = smem + L.oUtIn;
  double* PwIn = smem + L.oPwIn;
  double* RzIn = smem + L.oRzIn;
  double* red = smem + L.oRed;
  double* bc = smem + L.oBc;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int rb = L.rb;
  const int i0 = min(m, rank * rb), i1 = min(m, i0 + rb), nr = i1 - i0;
  const int j0 = min(n, rank * L.cbw), j1 = min(n, j0 + L.cbw), nc = j1 - j0;
  const double delta = T.delta;
  // own-row work: warp 0 alone when the band has at most 32 rows
  const bool row_warp = rb <= 32;

  // Sum over this CTA's own rows of a per-row value (valid in warp 0).
  auto own_sum = [&](double v) -> double {
    if (row_warp) return wid == 0 ? warp_sum(v) : 0.0;
    v = warp_sum(v);
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) r = warp_sum(lane < kCW ? sh[lane] : 0.0);   // every lane of warp 0 gets the sum
    __syncthreads();
    return r;
  };
  const int row_stride = row_warp ? 32 : kCT;
  const bool row_thread = row_warp ? (wid == 0) : true;

  // ---- stage A's column band, D's, U's row band, the weights; r = xi, x = 0
  if (kAS) {
    for (long long e = tid; e < (long long)m * nc; e += kCT) {
      const int i = (int)(e / nc), jj = (int)(e % nc);
      As[(size_t)i * L.ncp + jj] = __ldg(T.A + (long long)i * T.lda + j0 + jj);
    }
  }
  for (int jj = tid; jj < nc; jj += kCT) Dl[jj] = __ldg(T.D + j0 + jj);
  for (int e = tid; e < nr * ell; e += kCT) {
    const int ii = e % nr, c = e / nr;
    Ub[(size_t)c * rb + ii] = __ldg(T.U + (size_t)c * T.ld + i0 + ii);
  }
  const double lam_ell = T.lam[ell - 1];
  for (int c = tid; c < ell; c += kCT) ws[c] = (lam_ell + delta) / (T.lam[c] + delta) - 1.0;
  for (int ii = tid; ii < nr; ii += kCT) { Rb[ii] = T.xi[i0 + ii]; Xb[ii] = 0.0; }
  cl.sync();   // every CTA has started and staged (distributed shared memory is live)

  // partials of U^T r and ||r||^2 over own rows, pushed into every CTA
  auto ut_push = [&]() {
    __syncthreads();
    if (row_warp) {
      // short bands: a thread per column walks the band (few FP64
      // instructions; a warp reduction per column would cost five)
      for (int c = tid; c < ell; c += kCT) {
        const double* u = Ub + (size_t)c * rb;
        double a0 = 0.0, a1 = 0.0;
        int ii = 0;
        for (; ii + 1 < nr; ii += 2) {
          a0 = fma(u[ii], Rb[ii], a0);
          a1 = fma(u[ii + 1], Rb[ii + 1], a1);
        }
        if (ii < nr) a0 = fma(u[ii], Rb[ii], a0);
        const double acc = a0 + a1;
        for (int k = 0; k < C; ++k) *cl.map_shared_rank(UtIn + (size_t)rank * (ell + 1) + c, k) = acc;
      }
    } else {
      for (int c = wid; c < ell; c += kCW) {
        const double* u = Ub + (size_t)c * rb;
        double a0 = 0.0, a1 = 0.0;
        int ii = lane;
        for (; ii + 32 < nr; ii += 64) {
          a0 = fma(u[ii], Rb[ii], a0);
          a1 = fma(u[ii + 32], Rb[ii + 32], a1);
        }
        if (ii < nr) a0 = fma(u[ii], Rb[ii], a0);
        const double acc = warp_sum(a0 + a1);
        push_all(cl, UtIn + (size_t)rank * (ell + 1), c, acc, C, lane);
      }
    }
    double v = 0.0;
    if (row_thread)
      for (int ii = tid; ii < nr; ii += row_stride) v = fma(Rb[ii], Rb[ii], v);
    v = own_sum(v);
    if (wid == 0) push_all(cl, UtIn + (size_t)rank * (ell + 1), ell, v, C, lane);
  };
  // s = U^T r (into wss as ws .* s) and ||r||^2 (returned) from the pushed partials
  auto ut_gather = [&]() -> double {
    if (4 * (ell + 1) <= kCW * kChunk) {
      // four warps (one per sub-partition) each add a quarter of the partials
      if (wid < 4)
        for (int e = lane; e <= ell; e += 32) red[wid * (ell + 1) + e] = quad_sum(UtIn + e, C, (size_t)(ell + 1), wid);
      __syncthreads();
      for (int e = tid; e <= ell; e += kCT) {
        const double s = (red[e] + red[(ell + 1) + e]) + (red[2 * (ell + 1) + e] + red[3 * (ell + 1) + e]);
        if (e < ell) wss[e] = ws[e] * s;
        else bc[0] = s;
      }
    } else {
      for (int e = tid; e <= ell; e += kCT) {
        const double s = tree_sum(UtIn + e, C, (size_t)(ell + 1));
        if (e < ell) wss[e] = ws[e] * s;
        else bc[0] = s;
      }
    }
    __syncthreads();
    return bc[0];
  };
  // z = r + U (ws .* s) on own rows, pushed into every CTA's Zf; partial r^T z pushed
  auto z_push = [&]() {
    double v = 0.0;
    if (row_warp) {
      // columns of U in four quarters, one per warp (sub-partition), then warp
      // 0 adds the quarters for its rows
      const int cq = (ell + 3) / 4;
      if (wid < 4 && lane < nr) {
        const int c0 = wid * cq, c1 = min(ell, c0 + cq);
        double a0 = 0.0, a1 = 0.0;
        int c = c0;
        for (; c + 1 < c1; c += 2) {
          a0 = fma(Ub[(size_t)c * rb + lane], wss[c], a0);
          a1 = fma(Ub[(size_t)(c + 1) * rb + lane], wss[c + 1], a1);
        }
        if (c < c1) a0 = fma(Ub[(size_t)c * rb + lane], wss[c], a0);
        red[wid * 32 + lane] = a0 + a1;
      }
      __syncthreads();
      if (wid == 0 && lane < nr) {
        const double zi = Rb[lane] + ((red[lane] + red[32 + lane]) + (red[64 + lane] + red[96 + lane]));
        for (int k = 0; k < C; ++k) *cl.map_shared_rank(Zf + i0 + lane, k) = zi;
        v = Rb[lane] * zi;
      }
    } else if (row_thread) {
      for (int ii = tid; ii < nr; ii += row_stride) {
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        int c = 0;
        for (; c + 4 <= ell; c += 4) {
          a0 = fma(Ub[(size_t)(c + 0) * rb + ii], wss[c + 0], a0);
          a1 = fma(Ub[(size_t)(c + 1) * rb + ii], wss[c + 1], a1);
          a2 = fma(Ub[(size_t)(c + 2) * rb + ii], wss[c + 2], a2);
          a3 = fma(Ub[(size_t)(c + 3) * rb + ii], wss[c + 3], a3);
        }
        for (; c < ell; ++c) a0 = fma(Ub[(size_t)c * rb + ii], wss[c], a0);
        const double zi = Rb[ii] + ((a0 + a1) + (a2 + a3));
        for (int k = 0; k < C; ++k) *cl.map_shared_rank(Zf + i0 + ii, k) = zi;
        v = fma(Rb[ii], zi, v);
      }
    }
    v = own_sum(v);
    if (wid == 0) push_all(cl, RzIn, rank, v, C, lane);
  };

  ut_push();
  cl.sync();
  double rr = ut_gather();
  const double bnorm2 = rr;
  const int limit = T.forced >= 0 ? T.forced : T.max_iter;
  int it = 0;
  bool done = (bnorm2 == 0.0) || (limit <= 0);
  double rz = 0.0, beta = 0.0;
  if (!done) {
    z_push();
    cl.sync();
    rz = tree_sum(RzIn, C);
  }
  int fail = 0;
  while (!done) {
    // p = z + beta p (all rows)
    for (int i = tid; i < m; i += kCT) P[i] = it == 0 ? Zf[i] : fma(beta, P[i], Zf[i]);
    __syncthreads();
    // t = D .* (A^T p) over own columns: lanes over 32 columns, warps over
    // rows (two interleaved accumulators each), then a tree over the warps.
    // One 32-column block at a time: a warp-uniform loop, so no FP64
    // instruction is issued for columns beyond the band (a predicated-off
    // FP64 instruction costs a full warp slot on this GPU).
    for (int c0 = 0; c0 < nc; c0 += kChunk) {
      const int nb = min(kChunk, nc - c0);
      if (!kAS && nb == kChunk) {
        // A from L2: four 32-column blocks per pass over the rows (longer
        // contiguous reads per row); every block is inside the band
        double a[4] = {0.0, 0.0, 0.0, 0.0}, b[4] = {0.0, 0.0, 0.0, 0.0};
        int i = wid;
        for (; i + kCW < m; i += 2 * kCW) {
          const double p0 = P[i], p1 = P[i + kCW];
          const double* r0p = T.A + (long long)i * T.lda + j0 + c0 + lane;
          const double* r1p = T.A + (long long)(i + kCW) * T.lda + j0 + c0 + lane;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            a[u] = fma(__ldg(r0p + u * 32), p0, a[u]);
            b[u] = fma(__ldg(r1p + u * 32), p1, b[u]);
          }
        }
        if (i < m) {
          const double p0 = P[i];
          const double* r0p = T.A + (long long)i * T.lda + j0 + c0 + lane;
#pragma unroll
          for (int u = 0; u < 4; ++u) a[u] = fma(__ldg(r0p + u * 32), p0, a[u]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) red[wid * kChunk + u * 32 + lane] = a[u] + b[u];
      } else
      for (int b0 = 0; b0 < nb; b0 += 32) {
        const int jj = c0 + b0 + lane;
        const bool on = b0 + lane < nb;
        double a = 0.0, b = 0.0;
        if (on) {
          int i = wid;
          for (; i + kCW < m; i += 2 * kCW) {
            const double x0 = kAS ? As[(size_t)i * L.ncp + jj] : __ldg(T.A + (long long)i * T.lda + j0 + jj);
            const double x1 = kAS ? As[(size_t)(i + kCW) * L.ncp + jj]
                                  : __ldg(T.A + (long long)(i + kCW) * T.lda + j0 + jj);
            a = fma(x0, P[i], a);
            b = fma(x1, P[i + kCW], b);
          }
          if (i < m) {
            const double x0 = kAS ? As[(size_t)i * L.ncp + jj] : __ldg(T.A + (long long)i * T.lda + j0 + jj);
            a = fma(x0, P[i], a);
          }
        }
        red[wid * kChunk + b0 + lane] = a + b;
      }
      __syncthreads();
      for (int c = tid; c < nb; c += kCT) {
        double w8[kCW];
#pragma unroll
        for (int w = 0; w < kCW; ++w) w8[w] = red[w * kChunk + c];
#pragma unroll
        for (int st = 1; st < kCW; st <<= 1)
#pragma unroll
          for (int w = 0; w + st < kCW; w += 2 * st) w8[w] += w8[w + st];
        Ts[c0 + c] = Dl[c0 + c] * w8[0];
      }
      __syncthreads();
    }
    // q = A_k t over all rows, each row's partial pushed to the CTA owning it
    if (kAS) {
      for (int i = tid; i < m; i += kCT) {
        const double* a = As + (size_t)i * L.ncp;
        double q0 = 0.0, q1 = 0.0, q2 = 0.0, q3 = 0.0;
        int jj = 0;
        for (; jj + 4 <= nc; jj += 4) {
          q0 = fma(a[jj + 0], Ts[jj + 0], q0);
          q1 = fma(a[jj + 1], Ts[jj + 1], q1);
          q2 = fma(a[jj + 2], Ts[jj + 2], q2);
          q3 = fma(a[jj + 3], Ts[jj + 3], q3);
        }
        for (; jj < nc; ++jj) q0 = fma(a[jj], Ts[jj], q0);
        const int o = i / rb;
        *cl.map_shared_rank(Qin + (size_t)rank * rb + (i - o * rb), o) = (q0 + q1) + (q2 + q3);
      }
    } else {
      for (int i = wid; i < m; i += kCW) {
        const double* a = T.A + (long long)i * T.lda + j0;
        double a0 = 0.0, a1 = 0.0;
        int jj = lane;
        for (; jj + 32 < nc; jj += 64) {
          a0 = fma(__ldg(a + jj), Ts[jj], a0);
          a1 = fma(__ldg(a + jj + 32), Ts[jj + 32], a1);
        }
        if (jj < nc) a0 = fma(__ldg(a + jj), Ts[jj], a0);
        const double acc = warp_sum(a0 + a1);
        const int o = i / rb;
        if (lane == 0) *cl.map_shared_rank(Qin + (size_t)rank * rb + (i - o * rb), o) = acc;
      }
    }
    cl.sync();                                                     // 1
    // w = delta p + sum_k q_k on own rows; partial p^T w pushed
    {
      double v = 0.0;
      if (row_warp) {
        // four warps each add a quarter of the C partials of the band's rows
        if (wid < 4 && lane < nr) red[wid * 32 + lane] = quad_sum(Qin + lane, C, (size_t)rb, wid);
        __syncthreads();
        if (wid == 0 && lane < nr) {
          const double s = (red[lane] + red[32 + lane]) + (red[64 + lane] + red[96 + lane]);
          const double wi = fma(delta, P[i0 + lane], s);
          Wb[lane] = wi;
          v = P[i0 + lane] * wi;
        }
      } else {
        for (int ii = tid; ii < nr; ii += row_stride) {
          const double wi = fma(delta, P[i0 + ii], tree_sum(Qin + ii, C, (size_t)rb));
          Wb[ii] = wi;
          v = fma(P[i0 + ii], wi, v);
        }
      }
      v = own_sum(v);
      if (wid == 0) push_all(cl, PwIn, rank, v, C, lane);
    }
    cl.sync();                                                     // 2
    if (wid == 0) {
      const double pw = lane_sum(PwIn, C, lane);
      const bool bad = !(pw > 0.0) || !isfinite(pw);
      if (lane == 0) { bc[1] = bad ? 0.0 : rz / pw; bc[2] = bad ? 1.0 : 0.0; }
    }
    __syncthreads();
    if (bc[2] != 0.0) { fail = 1; break; }
    const double alpha = bc[1];
    if (row_thread)
      for (int ii = tid; ii < nr; ii += row_stride) {
        Xb[ii] = fma(alpha, P[i0 + ii], Xb[ii]);
        Rb[ii] = fma(-alpha, Wb[ii], Rb[ii]);
      }
    ut_push();
    cl.sync();                                                     // 3
    rr = ut_gather();
    ++it;
    if (!isfinite(rr)) { fail = 1; break; }
    if (T.forced >= 0 ? (it >= T.forced) : (rr <= T.eta2 * bnorm2 || it >= T.max_iter)) break;
    z_push();
    cl.sync();                                                     // 4
    if (wid == 0) {
      const double rz_new = lane_sum(RzIn, C, lane);
      const int st = (!(rz_new > 0.0) || !isfinite(rz_new)) ? (rz_new != 0.0 ? 2 : 1) : 0;
      if (lane == 0) { bc[3] = rz_new; bc[4] = st == 0 ? rz_new / rz : 0.0; bc[5] = (double)st; }
    }
    __syncthreads();
    if (bc[5] != 0.0) {
      if (bc[5] == 2.0) fail = 1;
      break;
    }
    beta = bc[4];
    rz = bc[3];
  }
  for (int ii = tid; ii < nr; ii += kCT) T.x[i0 + ii] = Xb[ii];
  if (rank == 0 && tid == 0) {
    if (fail) set_error(T.err, kErrNumeric);
    *T.iters = it;
    T.sd[SD_RR] = rr;
    T.sd[SD_BNORM2] = bnorm2;
    T.sd[SD_ETA2] = T.eta2;
    if (T.t_ns) {
      unsigned long long t_end;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_end));
      atomicAdd(T.t_ns, t_end - t_start);
    }
  }
  cl.sync();   // no CTA leaves while a peer may still read its shared memory
}

// Whether the device can make a cluster of C CTAs resident with this much
// shared memory per CTA (a cluster must fit in one GPC).
bool launchable(int C, size_t smem_bytes, bool a_smem) {
  const void* fn = a_smem ? (const void*)k_pcg_cluster<true> : (const void*)k_pcg_cluster<false>;
  // attributes are set to the kernel's maxima, never lowered: handles on other
  // host threads may be launching it concurrently
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap) != cudaSuccess ||
      (C > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)) {
    cudaGetLastError();
    return false;
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)C);
  cfg.blockDim = dim3(kCT);
  cfg.dynamicSmemBytes = smem_bytes;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, fn, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return clusters >= 1;
}

}  // namespace

bool pcg_cluster_plan(int m, int n, int ell, int policy, ClusterPlan* plan) {
  if (m <= 0 || n <= 0 || ell <= 0) return false;
  // latency (one system at a time): 16 or 8 SMs with A on chip; a larger A
  // is faster on the cooperative grid.  Throughput (many systems side by
  // side): 8 or 4 SMs per system, A on chip or read from L2, since the FP64
  // work of an SM is used best by small clusters.
  struct Cand { int C, as; };
  static const Cand lat[] = {{kMaxC, 1}, {8, 1}};
  static const Cand thr[] = {{8, 1}, {4, 1}, {8, 0}, {4, 0}};
  const Cand* lists[2] = {lat, thr};
  const int lens[2] = {2, 4};
  for (int li = 0; li < 2; ++li) {
    if ((li == 0 && policy == 1) || (li == 1 && policy == 0)) continue;
    for (int k = 0; k < lens[li]; ++k) {
      const int C = lists[li][k].C, as = lists[li][k].as;
      const Layout L = make_layout(m, n, ell, C, as != 0);
      const size_t bytes = L.total * sizeof(double);
      if (bytes > kSmemCap) continue;
      if (!launchable(C, bytes, as != 0)) continue;
      plan->C = C;
      plan->a_smem = as;
      plan->smem_bytes = bytes;
      return true;
    }
  }
  return false;
}

int pcg_cluster_candidates(int m, int n, int ell, ClusterPlan* out, int cap) {
  if (m <= 0 || n <= 0 || ell <= 0) return 0;
  static const int Cs[3] = {kMaxC, 8, 4};
  int k = 0;
  for (int as = 1; as >= 0; --as)
    for (int ci = 0; ci < 3 && k < cap; ++ci) {
      if (as == 0 && Cs[ci] == kMaxC) continue;   // A from L2 runs on 8 or 4 CTAs only
      const Layout L = make_layout(m, n, ell, Cs[ci], as != 0);
      const size_t bytes = L.total * sizeof(double);
      if (bytes > kSmemCap || !launchable(Cs[ci], bytes, as != 0)) continue;
      out[k].C = Cs[ci];
      out[k].a_smem = as;
      out[k].smem_bytes = bytes;
      ++k;
    }
  return k;
}

bool pcg_cluster_plan_for(int m, int n, int ell, int C, int a_smem, ClusterPlan* plan) {
  if (m <= 0 || n <= 0 || ell <= 0 || (C != 4 && C != 8 && C != kMaxC)) return false;
  const Layout L = make_layout(m, n, ell, C, a_smem != 0);
  const size_t bytes = L.total * sizeof(double);
  if (bytes > kSmemCap || !launchable(C, bytes, a_smem != 0)) return false;
  plan->C = C;
  plan->a_smem = a_smem;
  plan->smem_bytes = bytes;
  return true;
}

cudaError_t pcg_cluster_f64(cudaStream_t st, const ClusterPlan& plan, const ClusterPcgTask& task,
                            const ClusterPcgTask* tasks, int count) {
  const void* fn = plan.a_smem ? (const void*)k_pcg_cluster<true> : (const void*)k_pcg_cluster<false>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap);
  if (e != cudaSuccess) return e;
  if (plan.C > 8) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)plan.C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)(plan.C * (tasks ? count : 1)));
  cfg.blockDim = dim3(kCT);
  cfg.dynamicSmemBytes = plan.smem_bytes;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  count_launches(1);
  if (plan.a_smem) return cudaLaunchKernelEx(&cfg, k_pcg_cluster<true>, task, tasks);
  return cudaLaunchKernelEx(&cfg, k_pcg_cluster<false>, task, tasks);
}

}  // namespace nys
