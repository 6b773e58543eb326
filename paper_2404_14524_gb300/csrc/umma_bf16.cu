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

}  // namespace

size_t umma_part_elems(int M, int N, int K, int num_sms) {
  const int npad = (N + 15) / 16 * 16;
  return (size_t)pick_splits(M, N, K, num_sms) * npad * M;
}

cudaError_t umma_gemm_bf16(cudaStream_t st, int M, int N, int K, const void* A, long long lda,
                           const void* B, long long ldb, float* part, size_t part_cap, int num_sms,
                           int* S_out, int* err) {
  if (M <= 0 || N <= 0 || N > 512 || K <= 0) return cudaErrorInvalidValue;
  const int npad = (N + 15) / 16 * 16;
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
  *S_out = S;
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
  } else {
    const size_t sm = smem_bytes<3>(npad);
    e = cudaFuncSetAttribute(k_umma_gemm<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kMaxDynSmem);   // never lowered: other host threads may launch it
    if (e != cudaSuccess) return e;
    count_launches(1);
    k_umma_gemm<3><<<grid, kThreads, sm, st>>>(ma, mb, M, npad, br, K, per, part, err);
  }
  return cudaGetLastError();
}

cudaError_t umma_reduce(cudaStream_t st, int M, int N, int S, const float* part, int mode,
                        const double* D, void* out, long long ldo) {
  const int npad = (N + 15) / 16 * 16;
  const long long total = (long long)M * N;
  count_launches(1);
  k_splitk_reduce_f32<<<(unsigned)((total + kNT - 1) / kNT), kNT, 0, st>>>(M, N, npad, S, part, mode, D, out, ldo);
  return cudaGetLastError();
}

}  // namespace nys
