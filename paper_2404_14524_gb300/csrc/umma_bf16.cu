// tcgen05 (5th-generation tensor core) BF16 GEMM for the Nystrom sketch of
// the precision form (Algorithm 1, second step, Y = A (D .* (A^T Omega))).
//
//   P[z][c][r] = sum_{k in split z} A[r, k] * B[c, k]     (FP32 accumulate)
//
// Both operands are K-major BF16 matrices in global memory (row r of A and
// row c of B are contiguous over k).  One CTA computes a 128-row stripe of
// the output for all N <= 512 columns (the whole sketch width), so each
// operand element of A is loaded from HBM exactly once per split.
//
//   warp 0 lane 0 : TMA producer (cp.async.bulk.tensor.2d, 128B swizzle)
//   warp 1 lane 0 : MMA issuer (tcgen05.mma.cta_group::1.kind::f16, M = 128)
//   warp 2        : TMEM allocator (tcgen05.alloc / dealloc, 512 columns)
//   warps 0-3     : epilogue (tcgen05.ld 32x32b, FP32 partials to global)
//
// Shared memory holds `kStages` stages of {A tile 128 x 64, B tile Npad x 64}
// guarded by full/empty mbarriers; the MMA warp releases a stage through
// tcgen05.commit.  Every mbarrier wait is bounded: on expiry the kernel
// records kErrTimeout, skips the remaining work, still deallocates TMEM and
// returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdlib>
#include <map>
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace nys {

namespace {

constexpr int kBM = 128;        // rows per CTA (UMMA M)
constexpr int kBK = 64;         // K per stage: 64 BF16 = 128 bytes = one swizzle atom row
constexpr int kMaxDynSmem = 227 * 1024;   // opt-in shared memory per CTA
constexpr int kUmmaK = 16;      // K per tcgen05.mma for kind::f16
constexpr int kThreads = 128;
constexpr unsigned kTmemCols = 512;
constexpr unsigned long long kSpinLimit = 1ull << 22;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: false (and the error word set) when the limit expires.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, int* err) {
  unsigned long long spins = 0;
  while (!mbar_try_wait(bar, parity)) {
    if (++spins > kSpinLimit) { set_error(err, kErrTimeout); return false; }
    if (*(volatile int*)err) return false;
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, unsigned long long* bar,
                                            int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<unsigned long long>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// Shared-memory matrix descriptor for a K-major, 128B-swizzled tile whose
// rows are 128 bytes and whose 8-row groups are 1024 bytes apart.
__device__ __forceinline__ unsigned long long sw128_desc(const void* base) {
  const unsigned long long addr = smem_u32(base);
  unsigned long long d = 0;
  d |= (addr & 0x3FFFFull) >> 4;              // start address
  d |= (unsigned long long)(16 >> 4) << 16;   // leading byte offset (unused for swizzled K-major)
  d |= (unsigned long long)(1024 >> 4) << 32; // stride byte offset: next 8-row group
  d |= 1ull << 46;                            // descriptor version for tcgen05
  d |= 2ull << 61;                            // 128-byte swizzle
  return d;
}

// Instruction descriptor: BF16 x BF16 -> FP32, both K-major, M = 128, N = n.
__host__ __device__ constexpr unsigned idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(n >> 3) << 17) | ((unsigned)(kBM >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(unsigned tmem_d, unsigned long long a, unsigned long long b,
                                          unsigned idesc, unsigned accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(tmem_d), "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(unsigned long long* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               ::"r"(smem_u32(bar)) : "memory");
}

template <int kStages>
struct Smem {
  alignas(1024) unsigned char a[kStages][kBM * kBK * 2];
  unsigned long long full[kStages];
  unsigned long long empty[kStages];
  unsigned long long done;
  unsigned tmem_base;
  int issued, consumed;
};

// B tiles live after the Smem header in dynamic shared memory (1024-aligned).
template <int kStages>
__global__ void __launch_bounds__(kThreads, 1)
    k_umma_gemm(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                int M, int npad, int box_rows, int K, int kblocks_per_split, float* __restrict__ part,
                int* err) {
  extern __shared__ __align__(1024) unsigned char dyn[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(dyn) + 1023) & ~uintptr_t(1023));
  Smem<kStages>& s = *reinterpret_cast<Smem<kStages>*>(base);
  unsigned char* btiles = base + ((sizeof(Smem<kStages>) + 1023) & ~size_t(1023));
  const int nboxes = (npad + box_rows - 1) / box_rows;
  const size_t b_stage_bytes = (size_t)nboxes * box_rows * kBK * 2;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kBM;
  const int z = blockIdx.y;
  const int kb_total = (K + kBK - 1) / kBK;
  const int kb0 = z * kblocks_per_split;
  const int kb1 = min(kb_total, kb0 + kblocks_per_split);
  const int nkb = kb1 - kb0;

  if (threadIdx.x == 0) {
    s.issued = 0;
    s.consumed = 0;
    for (int i = 0; i < kStages; ++i) { mbar_init(&s.full[i], 1); mbar_init(&s.empty[i], 1); }
    mbar_init(&s.done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(&s.tmem_base)), "r"(kTmemCols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = s.tmem_base;

  const unsigned a_bytes = kBM * kBK * 2;
  const unsigned tx_bytes = a_bytes + (unsigned)b_stage_bytes;   // full boxes, zero-filled past the edges

  if (warp == 0 && lane == 0 && nkb > 0) {
    // producer
    for (int i = 0; i < nkb; ++i) {
      const int st = i % kStages;
      const unsigned ph = (unsigned)(i / kStages) & 1u;
      if (i >= kStages && !mbar_wait(&s.empty[st], ph ^ 1u, err)) break;
      mbar_expect_tx(&s.full[st], tx_bytes);
      const int kx = (kb0 + i) * kBK;
      tma_load_2d(s.a[st], &mapA, &s.full[st], kx, m0);
      unsigned char* bt = btiles + st * b_stage_bytes;
      for (int bx = 0; bx < nboxes; ++bx)
        tma_load_2d(bt + (size_t)bx * box_rows * kBK * 2, &mapB, &s.full[st], kx, bx * box_rows);
      s.issued = i + 1;
    }
  } else if (warp == 1 && lane == 0 && nkb > 0) {
    // MMA issuer
    for (int i = 0; i < nkb; ++i) {
      const int st = i % kStages;
      const unsigned ph = (unsigned)(i / kStages) & 1u;
      if (!mbar_wait(&s.full[st], ph, err)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const unsigned long long da = sw128_desc(s.a[st]);
      unsigned char* bt = btiles + st * b_stage_bytes;
      for (int kk = 0; kk < kBK / kUmmaK; ++kk) {
        const unsigned long long koff = (unsigned long long)((kk * kUmmaK * 2) >> 4);
        for (int c0 = 0; c0 < npad; c0 += 256) {
          const int nn = min(256, npad - c0);
          const unsigned long long db = sw128_desc(bt + (size_t)c0 * kBK * 2);
          umma_bf16(tmem + (unsigned)c0, da + koff, db + koff, idesc_bf16(nn), (i > 0 || kk > 0) ? 1u : 0u);
        }
      }
      umma_commit(&s.empty[st]);
      s.consumed = i + 1;
    }
    umma_commit(&s.done);
  }
  __syncthreads();
  // After a timeout, wait (bounded) for TMA copies that were issued but not
  // consumed, so that no bulk copy targets this CTA's shared memory at exit.
  if (threadIdx.x == 0) {
    for (int i = s.consumed; i < s.issued; ++i) {
      unsigned long long spins = 0;
      while (!mbar_try_wait(&s.full[i % kStages], (unsigned)(i / kStages) & 1u) && ++spins < kSpinLimit) {}
    }
  }

  // epilogue: every warp reads its 32 TMEM lanes (rows)
  bool ok = (nkb > 0) ? mbar_wait(&s.done, 0u, err) : true;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int row = m0 + warp * 32 + lane;
  float* out = part + (size_t)z * npad * M;
  if (ok) {
    for (int c0 = 0; c0 < npad; c0 += 8) {
      unsigned v[8];
      const unsigned taddr = tmem + ((unsigned)(warp * 32) << 16) + (unsigned)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < M) {
#pragma unroll
        for (int j = 0; j < 8; ++j) out[(size_t)(c0 + j) * M + row] = nkb > 0 ? __uint_as_float(v[j]) : 0.0f;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 2) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// out[c * ldo + r] = op(sum_z part[z][c][r]) for r < M, c < N (fixed order).
//   mode 0: FP32 store;  mode 1: scale by D[r], store BF16.
__global__ void k_splitk_reduce_f32(int M, int N, int npad, int S, const float* __restrict__ part,
                                    int mode, const double* __restrict__ D, void* out, long long ldo) {
  const long long idx = (long long)blockIdx.x * kNT + threadIdx.x;
  if (idx >= (long long)M * N) return;
  const int r = (int)(idx % M), c = (int)(idx / M);
  float s = 0.0f;
  for (int zz = 0; zz < S; ++zz) s += part[((size_t)zz * npad + c) * M + r];
  if (mode == 0) static_cast<float*>(out)[(size_t)c * ldo + r] = s;
  else static_cast<__nv_bfloat16*>(out)[(size_t)c * ldo + r] = __float2bfloat16_rn((float)(D[r] * (double)s));
}

// ---------------------------------------------------------------- CTA-pair kernel
//
// tcgen05.mma.cta_group::2 with M = 256: a cluster of two CTAs (one per SM)
// computes a 256-row stripe of the output.  Each CTA stages its own 128 rows
// of A and one half of every B chunk (an MMA of N columns reads columns
// [0, N/2) from the even CTA's shared memory and [N/2, N) from the odd
// one's), so a stage costs 16 KB + Npad x 64 B per SM instead of
// 16 KB + Npad x 128 B: five stages fit at Npad = 416 where the one-SM kernel
// holds three, and B crosses L2 half as often.  Npad is N rounded up to 32
// so that every MMA chunk (at most 256 columns) is a multiple of 32 wide.
//
// Work split (stream-K): the tiles x kb (256-row tile, 64-wide k-block)
// units, tile-major, are cut into equal contiguous ranges, one per pair of a
// grid of co-resident pairs.  A pair walks its range as segments, one per
// tile it touches; a segment that covers a whole tile is written straight to
// the output (with the output mode applied), any other one as an FP32
// partial into slot (tile + pair) of the workspace, and k_pair_reduce sums
// the partials of a tile in pair order (deterministic).  Slots never
// collide: pair ranges increase with the pair index.
//
// The TMA loads carry L2 eviction hints: A streams through once (evict
// first), B is re-read by every pair (evict last); measured +4 % at
// M = 8000, K = 40000.  An L2 prefetch of A a few k-blocks ahead of the
// stages gained nothing, and one of A and B twelve k-blocks ahead evicted
// tiles before their loads (DRAM reads 761 -> 1084 MB) and was slower.
//
// Roles per CTA (6 warps): warp 0 lane 0 is the TMA producer in both CTAs
// (the copies of both land on the even CTA's full barrier, which expects
// both CTAs' bytes); warp 1 lane 0 of the even CTA issues the MMAs and
// commits to the barriers of both CTAs; warps 2-5 drain TMEM (warp w reads
// lanes 32 (w mod 4) .. +31) and arrive on the even CTA's tmem_empty barrier
// once per segment; warp 2 also allocates TMEM together with the peer's
// warp 2.  Every wait is bounded in time (kPairWaitNs): on expiry the kernel
// records kErrTimeout and every role stops at its next wait; the epilogue
// warps decide together whether to go on (a barrier reduction), and the MMA
// thread still commits a drain barrier so that no tensor-core operation is
// in flight when TMEM is freed.
constexpr int kPairThreads = 192;
constexpr bool kPairHints = true;    // L2 eviction hints on the TMA loads
constexpr int kPairMaxStages = 8;
constexpr unsigned kAStage = kBM * kBK * 2;                  // 16 KB: 128 rows x 128 B
constexpr size_t kPairHdr = 1024;
constexpr unsigned long long kPairWaitNs = 2000000000ull;    // 2 s
constexpr unsigned long long kPairDrainNs = 20000000ull;     // 20 ms (only after an abort)

struct PairSmem {
  unsigned long long full[kPairMaxStages];
  unsigned long long empty[kPairMaxStages];
  unsigned long long tmem_full, tmem_empty, drain;
  unsigned tmem_base;
  int issued, consumed;
};
static_assert(sizeof(PairSmem) <= kPairHdr, "pair header");

struct PairArgs {
  int M, N, npad, tiles, kb, per, U, stages, nchunk;
  float* part;
  int mode;
  const double* D;
  void* out;
  long long ldo;
  int* err;
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Shared::cluster address of the same shared variable in CTA `rank`.
__device__ __forceinline__ unsigned map_rank(const void* p, unsigned rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}

__device__ __forceinline__ bool mbar_try_wait_cl(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded in time: false (error word set on expiry) when the limit passes or
// another role has already recorded an error.
__device__ __forceinline__ bool mbar_wait_pair(unsigned long long* bar, unsigned parity, int* err) {
  if (mbar_try_wait_cl(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (unsigned it = 1;; ++it) {
    if (mbar_try_wait_cl(bar, parity)) return true;
    if ((it & 63u) == 0) {
      if (*(volatile int*)err) return false;
      if (global_ns() - t0 > kPairWaitNs) { set_error(err, kErrTimeout); return false; }
    }
  }
}

// Drain waits after an abort: bounded by a short time, no error recorded.
__device__ __forceinline__ void mbar_drain_wait(unsigned long long* bar, unsigned parity) {
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait_cl(bar, parity) && global_ns() - t0 < kPairDrainNs) {}
}

// TMA 2D load into this CTA's shared memory, completion counted on the
// mbarrier at shared::cluster address `bar` (the even CTA's).
__device__ __forceinline__ void tma_load_2d_pair(void* dst, const CUtensorMap* map, unsigned bar, int x, int y,
                                                 unsigned long long pol) {
  if (kPairHints)
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%3, %4}], [%2], %5;"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<unsigned long long>(map)), "r"(bar), "r"(x), "r"(y), "l"(pol)
        : "memory");
  else
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<unsigned long long>(map)), "r"(bar), "r"(x), "r"(y)
        : "memory");
}

// L2 eviction policies: A streams through once (evict first), B is re-read
// by every pair (evict last).
__device__ __forceinline__ unsigned long long l2_policy(bool evict_last) {
  unsigned long long pol;
  if (evict_last) asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  else asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

// Instruction descriptor: BF16 x BF16 -> FP32, both K-major, M = 256, N = n.
__host__ __device__ constexpr unsigned idesc_pair(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(n >> 3) << 17) | ((unsigned)(256 >> 4) << 24);
}

__device__ __forceinline__ void umma_pair(unsigned tmem_d, unsigned long long a, unsigned long long b,
                                          unsigned idesc, unsigned accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(tmem_d), "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

// Arrive on the barrier at the same offset in both CTAs of the pair once the
// tensor-core operations issued so far have completed.
__device__ __forceinline__ void umma_commit_pair(unsigned long long* bar) {
  const unsigned short mask = 3;
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;"
      ::"r"(smem_u32(bar)), "h"(mask) : "memory");
}

__device__ __forceinline__ void tmem_ld32(unsigned taddr, unsigned* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
}

// AND of v over the 128 epilogue threads (named barrier 1).
__device__ __forceinline__ bool epilogue_all(bool v) {
  unsigned r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, 1, 128, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((unsigned)v)
      : "memory");
  return r != 0;
}

// Is tile t covered by one pair's range (written straight to the output)?
__host__ __device__ __forceinline__ bool pair_whole_tile(int t, int kb, int per) {
  return (long long)t * kb / per == ((long long)(t + 1) * kb - 1) / per;
}

// 32 columns [c0, c0 + 32) of one TMEM row to the output or to a partial slot.
__device__ __forceinline__ void pair_store32(const PairArgs& p, const unsigned* v, int c0, bool whole, int row,
                                             double drow, float* slot) {
  if (whole) {
    if (row >= p.M) return;
    if (p.mode == 0) {
      float* o = static_cast<float*>(p.out);
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (c0 + j < p.N) o[(size_t)(c0 + j) * p.ldo + row] = __uint_as_float(v[j]);
    } else {
      __nv_bfloat16* o = static_cast<__nv_bfloat16*>(p.out);
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (c0 + j < p.N)
          o[(size_t)(c0 + j) * p.ldo + row] = __float2bfloat16_rn((float)(drow * (double)__uint_as_float(v[j])));
    }
  } else if (row < p.M) {
#pragma unroll
    for (int j = 0; j < 32; ++j) slot[(size_t)(c0 + j) * 256] = __uint_as_float(v[j]);
  }
}

__global__ void __launch_bounds__(kPairThreads, 1)
    k_umma_gemm_pair(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB0,
                     const __grid_constant__ CUtensorMap mapB1, const PairArgs p) {
  extern __shared__ __align__(1024) unsigned char dyn[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(dyn) + 1023) & ~uintptr_t(1023));
  PairSmem& s = *reinterpret_cast<PairSmem*>(base);
  unsigned char* atiles = base + kPairHdr;
  unsigned char* btiles = atiles + (size_t)p.stages * kAStage;
  const size_t b_stage = (size_t)p.npad * 64;    // npad / 2 rows of 128 B
  const unsigned rank = cluster_rank();
  const int pair = blockIdx.x >> 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int u_begin = pair * p.per;
  const int u_end = min(p.U, u_begin + p.per);

  if (threadIdx.x == 0) {
    for (int i = 0; i < p.stages; ++i) { mbar_init(&s.full[i], 1); mbar_init(&s.empty[i], 1); }
    mbar_init(&s.tmem_full, 1);
    mbar_init(&s.tmem_empty, 2);   // one arrival from each CTA's epilogue
    mbar_init(&s.drain, 1);
    s.issued = 0;
    s.consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(&s.tmem_base)), "r"(kTmemCols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  cluster_sync_all();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = s.tmem_base;

  if (warp == 0) {
    if (lane == 0) {
      // producer (both CTAs)
      const unsigned stage_tx = 2u * (kAStage + (unsigned)b_stage);
      const unsigned long long pol_a = l2_policy(false), pol_b = l2_policy(true);
      int st = 0, i = 0;
      unsigned ph = 0;
      for (int u = u_begin; u < u_end; ++u, ++i) {
        const int t = u / p.kb;
        const int kx = (u - t * p.kb) * kBK;
        if (i >= p.stages && !mbar_wait_pair(&s.empty[st], ph ^ 1u, p.err)) break;
        if (rank == 0) mbar_expect_tx(&s.full[st], stage_tx);
        const unsigned fb = map_rank(&s.full[st], 0);
        tma_load_2d_pair(atiles + (size_t)st * kAStage, &mapA, fb, kx, t * 256 + (int)rank * kBM, pol_a);
        unsigned char* bt = btiles + (size_t)st * b_stage;
        for (int c = 0; c < p.nchunk; ++c) {
          const int c0 = c * 256, nc = min(256, p.npad - c0), hc = nc / 2;
          tma_load_2d_pair(bt + (size_t)c * 128 * 128, nc == 256 ? &mapB0 : &mapB1, fb, kx, c0 + (int)rank * hc,
                           pol_b);
        }
        s.issued = i + 1;
        if (++st == p.stages) { st = 0; ph ^= 1u; }
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && rank == 0) {
      // MMA issuer (even CTA)
      int st = 0, i = 0, j = 0;
      unsigned ph = 0;
      bool ok = true;
      for (int u = u_begin; ok && u < u_end; ++j) {
        const int t = u / p.kb;
        const int seg_end = min(u_end, (t + 1) * p.kb);
        if (j > 0 && !mbar_wait_pair(&s.tmem_empty, (unsigned)(j - 1) & 1u, p.err)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        for (int v = u; v < seg_end; ++v, ++i) {
          if (!mbar_wait_pair(&s.full[st], ph, p.err)) { ok = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const unsigned long long da = sw128_desc(atiles + (size_t)st * kAStage);
          unsigned char* bt = btiles + (size_t)st * b_stage;
#pragma unroll
          for (int kk = 0; kk < kBK / kUmmaK; ++kk) {
            const unsigned long long koff = (unsigned long long)((kk * kUmmaK * 2) >> 4);
            for (int c = 0; c < p.nchunk; ++c) {
              const int c0 = c * 256, nc = min(256, p.npad - c0);
              const unsigned long long db = sw128_desc(bt + (size_t)c * 128 * 128);
              umma_pair(tmem + (unsigned)c0, da + koff, db + koff, idesc_pair(nc), (v > u || kk > 0) ? 1u : 0u);
            }
          }
          umma_commit_pair(&s.empty[st]);
          s.consumed = i + 1;
          if (++st == p.stages) { st = 0; ph ^= 1u; }
        }
        if (!ok) break;
        umma_commit_pair(&s.tmem_full);
        u = seg_end;
      }
      umma_commit_pair(&s.drain);
    }
  } else {
    // epilogue (warps 2-5, both CTAs)
    const int lg = warp & 3;
    const int rl = (int)rank * kBM + lg * 32 + lane;
    const unsigned trow = tmem + ((unsigned)(lg * 32) << 16);
    int j = 0;
    for (int u = u_begin; u < u_end; ++j) {
      const int t = u / p.kb;
      const int seg_end = min(u_end, (t + 1) * p.kb);
      // the four epilogue warps leave together (each pass ends at named barrier 1)
      const bool got = mbar_wait_pair(&s.tmem_full, (unsigned)j & 1u, p.err);
      __syncwarp();
      if (!epilogue_all(got)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const bool whole = pair_whole_tile(t, p.kb, p.per);
      const int row = t * 256 + rl;
      const double drow = (whole && p.mode == 1 && row < p.M) ? p.D[row] : 0.0;
      float* slot = p.part + (size_t)(t + pair) * p.npad * 256 + rl;
      for (int c0 = 0; c0 < p.npad; c0 += 64) {
        const bool two = c0 + 32 < p.npad;
        unsigned v0[32], v1[32];
        tmem_ld32(trow + (unsigned)c0, v0);
        if (two) tmem_ld32(trow + (unsigned)(c0 + 32), v1);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        pair_store32(p, v0, c0, whole, row, drow, slot);
        if (two) pair_store32(p, v1, c0 + 32, whole, row, drow, slot);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (warp == 2 && lane == 0)
        asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];"
                     ::"r"(map_rank(&s.tmem_empty, 0)) : "memory");
      u = seg_end;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // no tensor-core operation in flight once the drain commit has arrived
    mbar_drain_wait(&s.drain, 0u);
    if (rank == 0) {
      // after an abort: copies issued by either CTA and not consumed still
      // signal this CTA's full barriers; wait for them (bounded)
      int peer_issued;
      asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(peer_issued) : "r"(map_rank(&s.issued, 1)) : "memory");
      const int hi = max(s.issued, peer_issued);
      for (int i = s.consumed; i < hi; ++i)
        mbar_drain_wait(&s.full[i % p.stages], (unsigned)(i / p.stages) & 1u);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  cluster_sync_all();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 2) {
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// out[c * ldo + r] for rows of tiles split across pairs: the partial slots
// (t + q), q = first .. last pair touching tile t, summed in that order.
__global__ void k_pair_reduce(int M, int N, int npad, int kb, int per, const float* __restrict__ part, int mode,
                              const double* __restrict__ D, void* out, long long ldo) {
  const long long idx = (long long)blockIdx.x * kNT + threadIdx.x;
  if (idx >= (long long)M * N) return;
  const int r = (int)(idx % M), c = (int)(idx / M);
  const int t = r / 256, rl = r - t * 256;
  if (pair_whole_tile(t, kb, per)) return;
  const int q0 = (int)((long long)t * kb / per), q1 = (int)(((long long)(t + 1) * kb - 1) / per);
  float s = 0.0f;
  for (int q = q0; q <= q1; ++q) s += part[((size_t)(t + q) * npad + c) * 256 + rl];
  if (mode == 0) static_cast<float*>(out)[(size_t)c * ldo + r] = s;
  else static_cast<__nv_bfloat16*>(out)[(size_t)c * ldo + r] = __float2bfloat16_rn((float)(D[r] * (double)s));
}

typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
  static EncodeTiled fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  }
  return fn;
}

// 2D BF16 tensor map over a row-major rows x cols matrix (leading dimension
// ld elements), box kBK (cols) x box_rows, 128-byte swizzle, zero fill.
bool make_map(CUtensorMap* map, const void* ptr, long long rows, long long cols, long long ld, int box_rows) {
  EncodeTiled enc = encoder();
  if (!enc) return false;
  if ((reinterpret_cast<uintptr_t>(ptr) & 15u) || ((ld * 2) % 16)) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// B is loaded in ceil(npad / 256) boxes of equal height (a multiple of 8 rows,
// so every box starts on a 1024-byte swizzle group).
int b_box_rows(int npad) {
  const int nb = (npad + 255) / 256;
  return ((npad + nb - 1) / nb + 7) / 8 * 8;
}

template <int kStages>
size_t smem_bytes(int npad) {
  const int br = b_box_rows(npad);
  const int nb = (npad + br - 1) / br;
  return 1024 + ((sizeof(Smem<kStages>) + 1023) & ~size_t(1023)) + (size_t)kStages * nb * br * kBK * 2;
}

// Number of K splits, from a simple time model in units of one k-block of
// MMAs on one SM: waves(S) * (ceil(kb / S) + 16), where a wave is one CTA per
// SM and 16 k-blocks is the cost of writing and re-reading one 128 x N FP32
// partial tile at the per-SM share of HBM bandwidth (both scale with N).
int pick_splits(int M, int N, int K, int num_sms) {
  (void)N;
  const int tiles = (M + kBM - 1) / kBM;
  const int kb = (K + kBK - 1) / kBK;
  int best = 1;
  long long best_t = -1;
  for (int S = 1; S <= 64 && S <= kb; ++S) {
    const long long units = (long long)tiles * S;
    const long long waves = (units + num_sms - 1) / num_sms;
    const long long t = waves * ((kb + S - 1) / S + (S > 1 ? 16 : 0));
    if (best_t < 0 || t < best_t) { best_t = t; best = S; }
  }
  return best;
}

// ---- CTA-pair plan
constexpr int kPairMinUnits = 8;      // shortest range a pair is given (k-blocks), unless K is shorter

int pair_npad(int N) { return (N + 31) / 32 * 32; }

int pair_stages(int npad) {
  const size_t per_stage = kAStage + (size_t)npad * 64;
  return (int)std::min<size_t>(kPairMaxStages, (kMaxDynSmem - 1024 - kPairHdr) / per_stage);
}

size_t pair_smem(int npad, int stages) { return 1024 + kPairHdr + (size_t)stages * (kAStage + (size_t)npad * 64); }

struct PairPlan {
  int npad, stages, tiles, kb, U, per, pairs, nchunk;
  size_t smem;
  bool any_split;
};

PairPlan pair_plan(int M, int N, int K, int max_pairs) {
  PairPlan q;
  q.npad = pair_npad(N);
  q.stages = pair_stages(q.npad);
  q.smem = pair_smem(q.npad, q.stages);
  q.tiles = (M + 255) / 256;
  q.kb = (K + kBK - 1) / kBK;
  q.U = q.tiles * q.kb;
  q.per = std::max((q.U + max_pairs - 1) / max_pairs, std::min(q.kb, kPairMinUnits));
  q.pairs = (q.U + q.per - 1) / q.per;
  q.nchunk = (q.npad + 255) / 256;
  q.any_split = false;
  for (int t = 0; t < q.tiles && !q.any_split; ++t) q.any_split = !pair_whole_tile(t, q.kb, q.per);
  return q;
}

size_t pair_part_elems(const PairPlan& q) {
  return q.any_split ? (size_t)(q.tiles + q.pairs) * q.npad * 256 : 0;
}

// Pairs of the kernel that can be resident at once for this shared-memory
// size (0 when clusters of two cannot be launched).
int pair_max_resident(size_t smem) {
  static std::mutex mu;
  static std::map<size_t, int> cache;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(smem);
  if (it != cache.end()) return it->second;
  int n = 0;
  if (cudaFuncSetAttribute(k_umma_gemm_pair, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem) ==
      cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(2, 1, 1);
    cfg.blockDim = dim3(kPairThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (cudaOccupancyMaxActiveClusters(&n, k_umma_gemm_pair, &cfg) != cudaSuccess) n = 0;
  }
  cudaGetLastError();
  cache[smem] = n;
  return n;
}

// NYS_UMMA_PAIR: "0" the one-SM kernel only, "1" the CTA-pair kernel only
// (an error when it cannot run), unset: the pair kernel where it can run.
int pair_policy() {
  const char* e = std::getenv("NYS_UMMA_PAIR");
  if (!e || !*e) return -1;
  return e[0] == '0' ? 0 : 1;
}

cudaError_t launch_pair(cudaStream_t st, const PairPlan& q, int M, int N, int K, const void* A, long long lda,
                        const void* B, long long ldb, float* part, int mode, const double* D, void* out,
                        long long ldo, int* err) {
  CUtensorMap ma, mb0, mb1;
  const int hc_last = (q.npad - (q.nchunk - 1) * 256) / 2;
  if (!make_map(&ma, A, M, K, lda, kBM) || !make_map(&mb0, B, N, K, ldb, 128) ||
      !make_map(&mb1, B, N, K, ldb, hc_last))
    return cudaErrorInvalidValue;
  PairArgs a;
  a.M = M;
  a.N = N;
  a.npad = q.npad;
  a.tiles = q.tiles;
  a.kb = q.kb;
  a.per = q.per;
  a.U = q.U;
  a.stages = q.stages;
  a.nchunk = q.nchunk;
  a.part = part;
  a.mode = mode;
  a.D = D;
  a.out = out;
  a.ldo = ldo;
  a.err = err;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(2 * q.pairs, 1, 1);
  cfg.blockDim = dim3(kPairThreads, 1, 1);
  cfg.dynamicSmemBytes = q.smem;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  count_launches(1);
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_umma_gemm_pair, ma, mb0, mb1, a);
  if (e != cudaSuccess) return e;
  if (q.any_split) {
    const long long total = (long long)M * N;
    count_launches(1);
    k_pair_reduce<<<(unsigned)((total + kNT - 1) / kNT), kNT, 0, st>>>(M, N, q.npad, q.kb, q.per, part, mode, D,
                                                                      out, ldo);
  }
  return cudaGetLastError();
}

cudaError_t launch_one_sm(cudaStream_t st, int M, int N, int K, const void* A, long long lda, const void* B,
                          long long ldb, float* part, size_t part_cap, int num_sms, int mode, const double* D,
                          void* out, long long ldo, int* err) {
  const int npad = (N + 15) / 16 * 16;
  if ((size_t)npad * M > part_cap) return cudaErrorInvalidValue;
  CUtensorMap ma, mb;
  if (!make_map(&ma, A, M, K, lda, kBM)) return cudaErrorInvalidValue;
  const int br = b_box_rows(npad);
  if (!make_map(&mb, B, N, K, ldb, br)) return cudaErrorInvalidValue;
  const int tiles = (M + kBM - 1) / kBM;
  const int kb = (K + kBK - 1) / kBK;
  int S = pick_splits(M, N, K, num_sms);
  while (S > 1 && (size_t)S * npad * M > part_cap) --S;
  const int per = (kb + S - 1) / S;
  S = (kb + per - 1) / per;
  dim3 grid(tiles, S);
  cudaError_t e;
  if (npad <= 128) {
    const size_t sm = smem_bytes<6>(npad);
    e = cudaFuncSetAttribute(k_umma_gemm<6>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kMaxDynSmem);   // never lowered: other host threads may launch it
    if (e != cudaSuccess) return e;
    count_launches(1);
    k_umma_gemm<6><<<grid, kThreads, sm, st>>>(ma, mb, M, npad, br, K, per, part, err);
  } else if (npad <= 256) {
    const size_t sm = smem_bytes<4>(npad);
    e = cudaFuncSetAttribute(k_umma_gemm<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kMaxDynSmem);   // never lowered: other host threads may launch it
    if (e != cudaSuccess) return e;
    count_launches(1);
    k_umma_gemm<4><<<grid, kThreads, sm, st>>>(ma, mb, M, npad, br, K, per, part, err);
  } else if (smem_bytes<3>(npad) <= (size_t)kMaxDynSmem) {
    const size_t sm = smem_bytes<3>(npad);
    e = cudaFuncSetAttribute(k_umma_gemm<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kMaxDynSmem);   // never lowered: other host threads may launch it
    if (e != cudaSuccess) return e;
    count_launches(1);
    k_umma_gemm<3><<<grid, kThreads, sm, st>>>(ma, mb, M, npad, br, K, per, part, err);
  } else {
    // N above 448: three stages of {A, B} no longer fit in shared memory
    const size_t sm = smem_bytes<2>(npad);
    e = cudaFuncSetAttribute(k_umma_gemm<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kMaxDynSmem);   // never lowered: other host threads may launch it
    if (e != cudaSuccess) return e;
    count_launches(1);
    k_umma_gemm<2><<<grid, kThreads, sm, st>>>(ma, mb, M, npad, br, K, per, part, err);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long total = (long long)M * N;
  count_launches(1);
  k_splitk_reduce_f32<<<(unsigned)((total + kNT - 1) / kNT), kNT, 0, st>>>(M, N, npad, S, part, mode, D, out, ldo);
  return cudaGetLastError();
}

}  // namespace

size_t umma_part_elems(int M, int N, int K, int num_sms) {
  const int npad = (N + 15) / 16 * 16;
  const size_t one_sm = (size_t)pick_splits(M, N, K, num_sms) * npad * M;
  return std::max(one_sm, pair_part_elems(pair_plan(M, N, K, std::max(1, num_sms / 2))));
}

cudaError_t umma_gemm_bf16(cudaStream_t st, int M, int N, int K, const void* A, long long lda, const void* B,
                           long long ldb, float* part, size_t part_cap, int num_sms, int mode, const double* D,
                           void* out, long long ldo, int* err, int* kernel_used) {
  if (M <= 0 || N <= 0 || N > 512 || K <= 0 || (mode == 1 && !D)) return cudaErrorInvalidValue;
  const int policy = pair_policy();
  if (policy != 0) {
    const int maxp = pair_max_resident(pair_smem(pair_npad(N), pair_stages(pair_npad(N))));
    if (maxp > 0) {
      const PairPlan q = pair_plan(M, N, K, maxp);
      if (pair_part_elems(q) <= part_cap) {
        if (kernel_used) *kernel_used = 2;
        return launch_pair(st, q, M, N, K, A, lda, B, ldb, part, mode, D, out, ldo, err);
      }
    }
    if (policy == 1) return cudaErrorInvalidValue;
  }
  if (kernel_used) *kernel_used = 1;
  return launch_one_sm(st, M, N, K, A, lda, B, ldb, part, part_cap, num_sms, mode, D, out, ldo, err);
}

}  // namespace nys
