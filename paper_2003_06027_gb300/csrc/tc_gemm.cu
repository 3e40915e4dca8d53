// tc_gemm.cu - BF16 x BF16 -> FP32 GEMM on the 5th-generation tensor cores
// (tcgen05.mma, accumulator in tensor memory), operands staged by TMA.
//
// One CTA computes a 128 x BN tile of D = A . B^T (BN <= 256, a multiple of 16)
// over its run of K:
//   * warp 0 allocates BN (rounded up to a power of two, >= 32) TMEM columns;
//   * one thread of warp 0 is the producer: per 64-wide k-block it loads the
//     128 x 64 tile of A and the BN x 64 tile of B into one of STAGES shared
//     memory slots with cp.async.bulk.tensor (128-byte swizzle, zero fill beyond
//     the matrix edges), completing on the slot's "full" mbarrier;
//   * one thread of warp 1 issues the MMAs: 4 x tcgen05.mma (K = 16 each) per
//     k-block into the TMEM accumulator, then tcgen05.commit onto the slot's
//     "empty" mbarrier, which frees the slot for the producer once the MMAs
//     that read it have completed; a last commit signals "accumulator ready";
//   * all four warps drain the accumulator: warp w reads TMEM lanes 32w..32w+31
//     (tile rows m) with tcgen05.ld, adds the bias, applies the ReLU and writes
//     out[n][m]: for each column n the 32 lanes of a warp store 32 consecutive
//     m, so the transposed write is coalesced.
// Every mbarrier wait is bounded (2^24 polls or 1 s); a wait that gives up
// records a timeout in the status word, the tile is written as NaN, and the
// CTA frees its TMEM and exits.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "fwi_internal.cuh"
#include "tc_gemm.h"
#include "tma.cuh"

namespace fwi {
namespace {

constexpr int TC_BM = 128;
constexpr int TC_BK = 64;  // one 128-byte swizzle row of BF16
constexpr int TC_STAGES = 4;
constexpr int TC_THREADS = 128;
constexpr int A_STAGE = TC_BM * TC_BK * 2;  // 16 KB

struct TcArgs {
  long long M;
  int N, BN, nkb, kbps;
  float* out;
  long long ldo, split_stride;
  const float* bias;
  int relu;
  int* status;
  uint32_t idesc;
  uint32_t tmem_cols;
};

// Shared-memory matrix descriptor of a K-major operand tile written by TMA with
// the 128-byte swizzle: rows of 128 bytes, 8-row groups 1024 bytes apart.
//   bits  0-13 start address >> 4      bits 16-29 leading byte offset >> 4 (unused here)
//   bits 32-45 stride byte offset >> 4 bits 46-47 descriptor version (1)
//   bits 61-63 layout: 2 = 128-byte swizzle
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t r[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__global__ void __launch_bounds__(TC_THREADS, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, const TcArgs a) {
  extern __shared__ unsigned char tc_smem_raw[];
  __shared__ uint64_t full[TC_STAGES], empty[TC_STAGES], accb;
  __shared__ uint32_t tmem_slot;
  __shared__ int err;
  // the swizzled tiles need 1024-byte alignment
  const uint32_t raw = smem_u32(tc_smem_raw);
  unsigned char* smA = tc_smem_raw + ((1024u - (raw & 1023u)) & 1023u);
  const int B_STAGE = a.BN * TC_BK * 2;
  unsigned char* smB = smA + TC_STAGES * A_STAGE;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long m0 = (long long)blockIdx.x * TC_BM;
  const int n0 = blockIdx.y * a.BN;
  const int kb0 = blockIdx.z * a.kbps;
  const int nk = min(a.nkb - kb0, a.kbps);

  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; s++) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&accb, 1);
    err = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(a.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == 0 && lane == 0) {
    // producer
    for (int i = 0; i < nk; i++) {
      const int s = i % TC_STAGES;
      const uint32_t ph = (uint32_t)(i / TC_STAGES) & 1u;
      if (!mbar_wait(&empty[s], ph ^ 1u)) {
        err = 1;
        break;
      }
      mbar_expect_tx(&full[s], (uint32_t)(A_STAGE + B_STAGE));
      tma_2d(smA + s * A_STAGE, &ta, (kb0 + i) * TC_BK, (int)m0, &full[s]);
      tma_2d(smB + s * B_STAGE, &tb, (kb0 + i) * TC_BK, n0, &full[s]);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    for (int i = 0; i < nk; i++) {
      const int s = i % TC_STAGES;
      const uint32_t ph = (uint32_t)(i / TC_STAGES) & 1u;
      if (!mbar_wait(&full[s], ph)) {
        err = 1;
        break;
      }
      tc_fence_after();
      const uint64_t ad = sdesc_sw128(smem_u32(smA + s * A_STAGE));
      const uint64_t bd = sdesc_sw128(smem_u32(smB + s * B_STAGE));
#pragma unroll
      for (int kk = 0; kk < TC_BK / 16; kk++)  // +32 bytes along K per MMA
        tc_mma(tmem, ad + 2 * kk, bd + 2 * kk, a.idesc, (uint32_t)(i | kk));
      tc_commit(&empty[s]);
    }
    tc_commit(&accb);
  }
  __syncwarp();

  // epilogue: TMEM lane = tile row m, column = n
  const bool ok = mbar_wait(&accb, 0);
  tc_fence_after();
  __syncwarp();
  if (!ok && lane == 0) atomicOr(a.status, ST_TIMEOUT);
  const int row = warp * 32 + lane;
  const long long m = m0 + row;
  float* outp = a.out + (long long)blockIdx.z * a.split_stride;
  const bool bad = !ok || err;
  for (int c0 = 0; c0 < a.BN; c0 += 16) {
    uint32_t r[16];
    tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
    if (m < a.M) {
#pragma unroll
      for (int j = 0; j < 16; j++) {
        const int n = n0 + c0 + j;
        if (n < a.N) {
          float v = bad ? __int_as_float(0x7fc00000) : __uint_as_float(r[j]);
          if (a.bias) v += a.bias[n];
          if (a.relu) v = fmaxf(v, 0.f);
          outp[(long long)n * a.ldo + m] = v;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (err && threadIdx.x == 0) atomicOr(a.status, ST_TIMEOUT);
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
}

bool encode_bf16_sw128(CUtensorMap* map, const void* base, long long inner, long long rows, long long ld_elems,
                       int box_rows) {
  tma_host::EncodeTiled fn = tma_host::encoder();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld_elems * 2};
  const cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows};
  const cuuint32_t es[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

int tc_split_count(long long K, int want) {
  const long long nkb = tc_kblocks(K);
  if (want < 1) want = 1;
  const long long kbps = (nkb + want - 1) / want;
  return (int)((nkb + kbps - 1) / kbps);
}

cudaError_t tc_gemm(const TcGemm& g, cudaStream_t st) {
  if (!g.A || !g.B || !g.out || !g.status || g.M < 1 || g.N < 1 || g.K < 1 || g.splits < 1) return cudaErrorInvalidValue;
  if (g.lda % 8 || g.ldb % 8 || g.lda < g.K || g.ldb < g.K) return cudaErrorInvalidValue;
  if (((uintptr_t)g.A & 15) || ((uintptr_t)g.B & 15)) return cudaErrorInvalidValue;
  if (g.M > 0x7fffff00LL || g.N > 0x7fffff00) return cudaErrorInvalidValue;
  const int BN = std::min(256, (g.N + 15) / 16 * 16);
  const long long nkb = tc_kblocks(g.K);
  const long long kbps = (nkb + g.splits - 1) / g.splits;
  const int splits = (int)((nkb + kbps - 1) / kbps);
  uint32_t cols = 32;
  while ((int)cols < BN) cols <<= 1;
  TcArgs a;
  a.M = g.M;
  a.N = g.N;
  a.BN = BN;
  a.nkb = (int)nkb;
  a.kbps = (int)kbps;
  a.out = g.out;
  a.ldo = g.ldo;
  a.split_stride = g.split_stride;
  a.bias = g.bias;
  a.relu = g.relu;
  a.status = g.status;
  // instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
  // (bits 7-9 = 1, 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
  a.idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(TC_BM >> 4) << 24);
  a.tmem_cols = cols;
  CUtensorMap ta, tb;
  if (!encode_bf16_sw128(&ta, g.A, g.K, g.M, g.lda, TC_BM) || !encode_bf16_sw128(&tb, g.B, g.K, g.N, g.ldb, BN))
    return cudaErrorInvalidValue;
  const int smem = TC_STAGES * (A_STAGE + BN * TC_BK * 2) + 1024;
  cudaError_t e = cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)((g.M + TC_BM - 1) / TC_BM), (unsigned)((g.N + BN - 1) / BN), (unsigned)splits);
  k_tc_gemm<<<grid, TC_THREADS, smem, st>>>(ta, tb, a);
  return cudaGetLastError();
}

}  // namespace fwi
