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
// The convolution variant (CONV) gathers A instead of loading it: 256 threads
// build each 128 x 64 A stage from the FP32 activations of a 3x3 layer in the
// same swizzled layout, fence their shared-memory writes for the tensor core
// and arrive on the stage's second "full" barrier, which the MMA thread also
// waits for; warp 8 loads B by TMA, warp 9 issues the MMAs.
// Every mbarrier wait is bounded (2^24 polls or 1 s); a wait that gives up
// records a timeout in the status word, the tile is written as NaN, and the
// CTA frees its TMEM and exits.
#include <cuda.h>
#include <cuda_bf16.h>
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

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ uint32_t mulhi_div(uint32_t n, unsigned long long m, uint32_t s) {
  return (uint32_t)(((unsigned long long)n * m) >> s);
}

// The threads of a CTA: 128 (warp 0: TMEM and the TMA producer, warp 1: the
// MMA issuer, all four: the epilogue); with a gathered A operand (CONV) 320:
// warps 0-7 gather A (two threads per tile row, 32 taps each; warps 0-3 also
// run the epilogue), warp 8 loads B by TMA, warp 9 issues the MMAs. Up to two
// CONV CTAs share an SM, so that one's gather covers the other's load latency.
template <bool CONV>
struct TcRoles {
  static constexpr int THREADS = CONV ? 320 : TC_THREADS;
  static constexpr int GATHER = 2 * TC_BM;  // gathering threads (CONV)
  static constexpr int B_WARP = CONV ? 8 : 0;
  static constexpr int MMA_WARP = CONV ? 9 : 1;
  static constexpr int CTAS = CONV ? 2 : 1;
};

// Gathered A rows (CONV): threads r and r + 128 build row r of every 128 x 64
// stage tile, pixel m0 + r, each 32 of its taps (half h: k0 + 32 h .. k0 + 32 h
// + 31), read from x (zero outside the image and beyond 9 C), rounded to BF16 as
// the im2col kernels round them, and stored as four 16-byte chunks in the
// layout TMA's 128-byte swizzle gives a K-major tile (chunk c of row r at
// 16 (c ^ (r % 8)) within its 128-byte row).
struct GatherRow {
  long long base;  // x offset of (b, r0, s0) relative to channel 0, if m is a pixel
  uint32_t mask;   // bit 3p + q: tap (p, q) inside the image (0 if m is not a pixel)
};
__device__ __forceinline__ GatherRow gather_row(const TcConvA& c, long long m, long long M) {
  GatherRow g{0, 0u};
  if (m >= M) return g;
  const uint32_t bi = mulhi_div((uint32_t)m, c.wo_m, c.wo_s);
  const int j = (int)((uint32_t)m - bi * (uint32_t)c.Wo);
  const uint32_t b = mulhi_div(bi, c.ho_m, c.ho_s);
  const int i = (int)(bi - b * (uint32_t)c.Ho);
  const int r0 = c.sh * i - 1, s0 = c.sw * j - 1;
  g.base = ((long long)b * c.H + r0) * c.W + s0;
#pragma unroll
  for (int p = 0; p < 3; p++)
#pragma unroll
    for (int q = 0; q < 3; q++)
      if (r0 + p >= 0 && r0 + p < c.H && s0 + q >= 0 && s0 + q < c.W) g.mask |= 1u << (3 * p + q);
  return g;
}
constexpr int GATHER_K = TC_BK / 2;  // taps of a row built by one gathering thread per stage
// Tap table of a CONV CTA (shared memory, built once, one entry per tap of every
// k-block): for tap k < 9 C the x offset of (channel c, tap row p, tap column q)
// relative to a pixel's base, c B H W + p W + q, and the mask bit of its tap,
// 1 << (3 p + q); beyond 9 C, offset 0 and bit 1 << 9 (a bit no mask has).
// Loads (into registers) the GATHER_K taps of half `half` of k-block kb for the thread's row.
__device__ __forceinline__ void gather_load(const TcConvA& c, const GatherRow& g, const int2* tab, int kb, int half,
                                            float v[GATHER_K]) {
  const int2* t = tab + kb * TC_BK + GATHER_K * half;
  const float* xb = c.x + g.base;
#pragma unroll
  for (int kk = 0; kk < GATHER_K; kk++) {
    const int2 e = t[kk];
    v[kk] = (g.mask & (uint32_t)e.y) ? __ldg(xb + e.x) : 0.f;
  }
}
// Rounds them to BF16 and stores them as chunks 4 half .. 4 half + 3 of the row.
__device__ __forceinline__ void gather_store(const float v[GATHER_K], int row, int half, unsigned char* dst) {
  unsigned char* rowp = dst + row * 128;
#pragma unroll
  for (int cl = 0; cl < 4; cl++) {
    const int cc = 4 * half + cl;  // 16-byte chunk of the row
    uint32_t w[4];
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const __nv_bfloat162 h = __floats2bfloat162_rn(v[8 * cl + 2 * u], v[8 * cl + 2 * u + 1]);
      w[u] = *reinterpret_cast<const uint32_t*>(&h);
    }
    *reinterpret_cast<uint4*>(rowp + ((cc ^ (row & 7)) << 4)) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

template <bool CONV>
__global__ void __launch_bounds__(TcRoles<CONV>::THREADS, TcRoles<CONV>::CTAS)
    k_tc_gemm(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, const TcArgs a,
              const TcConvA conv) {
  using R = TcRoles<CONV>;
  extern __shared__ unsigned char tc_smem_raw[];
  __shared__ uint64_t full[TC_STAGES], empty[TC_STAGES], fulla[TC_STAGES], accb;
  __shared__ uint32_t tmem_slot;
  __shared__ int err;
  // the swizzled tiles need 1024-byte alignment
  const uint32_t raw = smem_u32(tc_smem_raw);
  unsigned char* smA = tc_smem_raw + ((1024u - (raw & 1023u)) & 1023u);
  const int B_STAGE = a.BN * TC_BK * 2;
  unsigned char* smB = smA + TC_STAGES * A_STAGE;
  int2* tab = nullptr;
  if (CONV) {  // after the stages: a.nkb k-blocks of (offset, tap bit) entries
    const int K9 = 9 * conv.C, len = a.nkb * TC_BK;
    tab = reinterpret_cast<int2*>(smB + TC_STAGES * a.BN * TC_BK * 2);
    const int plane = conv.B * conv.H * conv.W;
    for (int k = threadIdx.x; k < len; k += blockDim.x) {
      const int ch = k / 9, t = k - 9 * ch, p = t / 3, q = t - 3 * p;
      tab[k] = k < K9 ? make_int2(ch * plane + p * conv.W + q, 1 << t) : make_int2(0, 1 << 9);
    }
  }

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long m0 = (long long)blockIdx.x * TC_BM;
  const int n0 = blockIdx.y * a.BN;
  const int kb0 = blockIdx.z * a.kbps;
  const int nk = min(a.nkb - kb0, a.kbps);

  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; s++) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
      mbar_init(&fulla[s], R::GATHER);  // CONV: one arrival per gathering thread
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

  if (warp == R::B_WARP && lane == 0) {
    // TMA producer: A and B, or B alone when A is gathered
    for (int i = 0; i < nk; i++) {
      const int s = i % TC_STAGES;
      const uint32_t ph = (uint32_t)(i / TC_STAGES) & 1u;
      if (!mbar_wait(&empty[s], ph ^ 1u)) {
        err = 1;
        break;
      }
      mbar_expect_tx(&full[s], (uint32_t)((CONV ? 0 : A_STAGE) + B_STAGE));
      if (!CONV) tma_2d(smA + s * A_STAGE, &ta, (kb0 + i) * TC_BK, (int)m0, &full[s]);
      tma_2d(smB + s * B_STAGE, &tb, (kb0 + i) * TC_BK, n0, &full[s]);
    }
  } else if (warp == R::MMA_WARP && lane == 0) {
    // MMA issuer
    for (int i = 0; i < nk; i++) {
      const int s = i % TC_STAGES;
      const uint32_t ph = (uint32_t)(i / TC_STAGES) & 1u;
      if (!mbar_wait(&full[s], ph) || (CONV && !mbar_wait(&fulla[s], ph))) {
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
  } else if (CONV && (int)threadIdx.x < R::GATHER) {
    // A gatherers: half threadIdx.x / 128 of row threadIdx.x % 128 of every stage tile
    const int row = threadIdx.x % TC_BM, half = threadIdx.x / TC_BM;
    const GatherRow g = gather_row(conv, m0 + row, a.M);
    // the loads of k-block i + 1 are issued before block i is converted and stored
    float vn[GATHER_K];
    if (nk > 0) gather_load(conv, g, tab, kb0, half, vn);
    for (int i = 0; i < nk; i++) {
      const int s = i % TC_STAGES;
      const uint32_t ph = (uint32_t)(i / TC_STAGES) & 1u;
      float v[GATHER_K];
#pragma unroll
      for (int kk = 0; kk < GATHER_K; kk++) v[kk] = vn[kk];
      if (i + 1 < nk) gather_load(conv, g, tab, kb0 + i + 1, half, vn);
      if (!mbar_wait(&empty[s], ph ^ 1u)) {
        err = 1;
        break;
      }
      gather_store(v, row, half, smA + s * A_STAGE);
      fence_proxy_async();  // the generic-proxy writes before the tensor core reads them
      mbar_arrive(&fulla[s]);
    }
  }
  __syncwarp();

  // epilogue (warps 0-3): TMEM lane = tile row m, column = n
  if (warp < 4) {
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

// Multiply-shift constants for floor(n / d), n < 2^31 (Granlund & Montgomery,
// "Division by invariant integers using multiplication", 1994): l = ceil(log2 d),
// m = ceil(2^(32+l) / d), floor(n / d) = (n m) >> (32 + l).
static void div_consts(uint32_t d, unsigned long long* m, uint32_t* s) {
  uint32_t l = 0;
  while ((1ull << l) < d) l++;
  *s = 32 + l;
  *m = ((1ull << *s) + d - 1) / d;
}

TcConvA tc_conv_a(const float* x, int C, int B, int H, int W, int sh, int sw) {
  TcConvA c;
  c.x = x;
  c.C = C;
  c.B = B;
  c.H = H;
  c.W = W;
  c.sh = sh;
  c.sw = sw;
  c.Ho = (H - 1) / sh + 1;
  c.Wo = (W - 1) / sw + 1;
  div_consts((uint32_t)c.Wo, &c.wo_m, &c.wo_s);
  div_consts((uint32_t)c.Ho, &c.ho_m, &c.ho_s);
  return c;
}

int tc_split_count(long long K, int want) {
  const long long nkb = tc_kblocks(K);
  if (want < 1) want = 1;
  const long long kbps = (nkb + want - 1) / want;
  return (int)((nkb + kbps - 1) / kbps);
}

cudaError_t tc_gemm(const TcGemm& g, cudaStream_t st) {
  const bool conv = g.conv != nullptr;
  if ((!conv && !g.A) || !g.B || !g.out || !g.status || g.M < 1 || g.N < 1 || g.K < 1 || g.splits < 1)
    return cudaErrorInvalidValue;
  if (g.ldb % 8 || g.ldb < g.K || ((uintptr_t)g.B & 15)) return cudaErrorInvalidValue;
  if (!conv && (g.lda % 8 || g.lda < g.K || ((uintptr_t)g.A & 15))) return cudaErrorInvalidValue;
  if (conv) {  // the gathered operand must be the one the sizes describe
    const TcConvA& c = *g.conv;
    if (!c.x || (long long)c.B * c.Ho * c.Wo != g.M || 9LL * c.C != g.K) return cudaErrorInvalidValue;
  }
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
  if (!encode_bf16_sw128(&tb, g.B, g.K, g.N, g.ldb, BN)) return cudaErrorInvalidValue;
  if (conv) ta = tb;  // unused: A is gathered
  else if (!encode_bf16_sw128(&ta, g.A, g.K, g.M, g.lda, TC_BM)) return cudaErrorInvalidValue;
  const int smem = TC_STAGES * (A_STAGE + BN * TC_BK * 2) + 1024 + (conv ? (int)nkb * TC_BK * 8 : 0);
  const dim3 grid((unsigned)((g.M + TC_BM - 1) / TC_BM), (unsigned)((g.N + BN - 1) / BN), (unsigned)splits);
  TcConvA c{};
  if (conv) c = *g.conv;
  auto kern = conv ? k_tc_gemm<true> : k_tc_gemm<false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, conv ? TcRoles<true>::THREADS : TcRoles<false>::THREADS, smem, st>>>(ta, tb, a, c);
  return cudaGetLastError();
}

}  // namespace fwi
