// cnn.cu - layers of the learned start-model network (sm_103a).
//
// The one dense contraction of the project: 3x3 convolutions written as GEMMs
// over the whole batch, run on the tcgen05 tensor cores by tc_gemm.cu (BF16
// operands, FP32 accumulation in tensor memory). Activations are channel-major
// [C][B][H][W]; with Npix = B*Ho*Wo output pixels and K9 = 9C taps:
//   forward   y[o][pix]   = act(sum_k colT[pix][k] W[o][k] + bias[o])
//             A = colT [Npix][K9] (im2col, pixel-major), B = W [O][K9];
//             the epilogue adds the bias, applies the ReLU and writes y
//             channel-major directly from the accumulator;
//   data grad dcol[k][pix] = sum_o dyT[pix][o] W[o][k]
//             A = dyT [Npix][O], B = W^T [K9][O]; col2im gathers dx;
//   weight gr dw[o][k]    = sum_pix col[k][pix] dy[o][pix]
//             A = col [K9][Npix] (im2col, tap-major), B = dy [O][Npix],
//             split over pixel runs into FP32 partials summed in a fixed order.
// The data movement around the GEMMs (im2col in both layouts with the FP32 ->
// BF16 rounding, col2im as a deterministic gather, ReLU backward, bias
// gradient, transposes, upsampling, loss, Adam) is in the kernels below. No
// floating-point atomics: every reduction has a fixed order.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "fwi_cnn.h"
#include "fwi_host.h"
#include "fwi_internal.cuh"
#include "tc_gemm.h"

namespace fwi {
namespace {

__device__ __forceinline__ uint16_t to_bf16_bits(float f) {
  const __nv_bfloat16 b = __float2bfloat16_rn(f);
  return *reinterpret_cast<const uint16_t*>(&b);
}

__host__ __device__ __forceinline__ int conv_out(int n, int s) { return (n - 1) / s + 1; }
__host__ __device__ __forceinline__ long long round8(long long v) { return (v + 7) / 8 * 8; }

// Division by a loop-invariant divisor d >= 1 for dividends n < 2^31, as a
// multiply and a shift (Granlund & Montgomery, "Division by invariant integers
// using multiplication", 1994): with l = ceil(log2 d) and m = ceil(2^(32+l) / d),
// floor(n / d) = floor(n m / 2^(32+l)) exactly, since the error of m adds less
// than 2^(-1-l) <= 1/(2d) to n/d, whose fractional part is at most (d-1)/d.
struct FastDiv {
  uint32_t d = 1, s = 32;
  unsigned long long m = 1ull;
  FastDiv() = default;
  explicit FastDiv(uint32_t dv) : d(dv) {
    uint32_t l = 0;
    while ((1ull << l) < dv) l++;
    s = 32 + l;
    m = ((1ull << s) + dv - 1) / dv;
  }
  __device__ __forceinline__ uint32_t div(uint32_t n) const { return (uint32_t)(((unsigned long long)n * m) >> s); }
  __device__ __forceinline__ uint32_t mod(uint32_t n, uint32_t q) const { return n - q * d; }
};

struct ConvDims {
  int C, B, H, W, sh, sw, Ho, Wo;
  int K9, Npix;
  FastDiv fWo, fHo;  // pixel n = (b * Ho + i) * Wo + j
  FastDiv fW, fH, fB;  // input element e = ((c * B + b) * H + r) * W + s
};

// colT[pix][k] (row stride ldk, BF16): 64 pixels x 64 taps per block, read
// along pixels (coalesced in x), transposed through shared memory, written as
// 16-byte runs of taps. Taps k >= K9 up to ldk are written as zeros.
__global__ void __launch_bounds__(256) k_im2col_t(const float* __restrict__ x, const ConvDims d, int ldk,
                                                  uint16_t* __restrict__ colT) {
  __shared__ uint16_t tile[64][66];
  const int t = threadIdx.x;
  const int n0 = blockIdx.x * 64, k0 = blockIdx.y * 64;
  const int nl = t & 63, n = n0 + nl;
  int b = 0, i = 0, j = 0;
  const bool nok = n < d.Npix;
  if (nok) {
    const uint32_t bi = d.fWo.div((uint32_t)n);
    j = (int)d.fWo.mod((uint32_t)n, bi);
    b = (int)d.fHo.div(bi);
    i = (int)d.fHo.mod(bi, (uint32_t)b);
  }
  const long long plane = (long long)d.B * d.H * d.W;
  const float* xb = x + (long long)b * d.H * d.W;
  const int r0 = d.sh * i - 1, s0 = d.sw * j - 1;
  float v[16];
#pragma unroll
  for (int u = 0; u < 16; u++) {  // all 16 loads in flight before the first use
    const int k = k0 + (t >> 6) + 4 * u;
    const int c = k / 9, pq = k - 9 * c, p = pq / 3, q = pq - 3 * p;
    const int r = r0 + p, s = s0 + q;
    v[u] = (nok && k < d.K9 && r >= 0 && r < d.H && s >= 0 && s < d.W) ? __ldg(xb + c * plane + (long long)r * d.W + s)
                                                                       : 0.f;
  }
#pragma unroll
  for (int u = 0; u < 16; u++) tile[(t >> 6) + 4 * u][nl] = to_bf16_bits(v[u]);
  __syncthreads();
#pragma unroll
  for (int pass = 0; pass < 2; pass++) {
    const int nl2 = pass * 32 + (t >> 3), kg = t & 7;
    const int n2 = n0 + nl2, kk = k0 + 8 * kg;
    if (n2 < d.Npix && kk < ldk) {
      uint32_t w[4];
#pragma unroll
      for (int u = 0; u < 4; u++)
        w[u] = (uint32_t)tile[8 * kg + 2 * u][nl2] | ((uint32_t)tile[8 * kg + 2 * u + 1][nl2] << 16);
      *reinterpret_cast<uint4*>(colT + (long long)n2 * ldk + kk) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

// colT[pix][k] (row stride ldk, BF16), row-staged: a block takes one output
// row (b, i), a run of 64 output columns and 16 input channels. It stages the 3
// input rows each channel's taps read (64 sw + 2 columns, zero outside the
// image) in shared memory, reading every input value once, then writes each
// pixel's 144 taps of the chunk as 18 runs of 16 bytes (288 bytes, whole
// 32-byte sectors when the row stride is a multiple of 288 bytes, as for 16
// channels or a multiple: no sector is shared between two blocks' writes).
// Thread (run v, pixel group g) of the 288 writes run v of pixels g, g+16,
// g+32, g+48: the 8 taps of its run, and so their shared-memory offsets, are
// the same for all four, computed once. Taps in [K9, ldk) are written as zeros
// (their staged channels are zero). Dynamic shared memory: IM_CC * 3 * (64 sw +
// 2) floats.
constexpr int IM_CC = 16;   // channels per block
constexpr int IM_VPP = IM_CC * 9 / 8;  // 16-byte runs per pixel
constexpr int IM_PIX = 64;  // output columns per block
constexpr int IM_GRP = 16;  // pixel groups: IM_VPP x IM_GRP threads
constexpr int IM_T_THREADS = IM_VPP * IM_GRP;
__global__ void __launch_bounds__(IM_T_THREADS) k_im2col_rows_t(const float* __restrict__ x, const ConvDims d, int ldk,
                                                                uint16_t* __restrict__ colT) {
  extern __shared__ float xs[];  // [IM_CC][3][JW]
  const int row = blockIdx.x;    // b * Ho + i
  const int j0 = blockIdx.y * IM_PIX, c0 = blockIdx.z * IM_CC;
  const uint32_t b = d.fHo.div((uint32_t)row);
  const int i = row - (int)b * d.Ho;
  const int JW = IM_PIX * d.sw + 2, s0 = d.sw * j0 - 1;
  const long long plane = (long long)d.B * d.H * d.W;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int cp = warp; cp < IM_CC * 3; cp += IM_T_THREADS / 32) {  // staged row (channel, tap row)
    const int cc = cp / 3, p = cp - 3 * cc, c = c0 + cc, r = d.sh * i + p - 1;
    const bool rok = c < d.C && r >= 0 && r < d.H;
    const float* src = rok ? x + c * plane + ((long long)b * d.H + r) * d.W : x;
    for (int col = lane; col < JW; col += 32) {
      const int sc = s0 + col;
      xs[cp * JW + col] = (rok && sc >= 0 && sc < d.W) ? __ldg(src + sc) : 0.f;
    }
  }
  __syncthreads();
  const int vv = threadIdx.x % IM_VPP, grp = threadIdx.x / IM_VPP;
  const int k0 = c0 * 9 + 8 * vv;
  if (k0 >= ldk) return;
  int off[8];
#pragma unroll
  for (int u = 0; u < 8; u++) {
    const int t = 8 * vv + u;  // tap within the chunk: (cc, p, q)
    const int cc = t / 9, pq = t - 9 * cc, p = pq / 3, q = pq - 3 * p;
    off[u] = (3 * cc + p) * JW + q;
  }
  const long long pix0 = (long long)row * d.Wo;
#pragma unroll
  for (int k = 0; k < IM_PIX / IM_GRP; k++) {
    const int jl = grp + IM_GRP * k, j = j0 + jl;
    if (j >= d.Wo) break;
    const float* xl = xs + d.sw * jl;
    uint32_t w[4];
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const __nv_bfloat162 h = __floats2bfloat162_rn(xl[off[2 * u]], xl[off[2 * u + 1]]);
      w[u] = *reinterpret_cast<const uint32_t*>(&h);
    }
    *reinterpret_cast<uint4*>(colT + (pix0 + j) * ldk + k0) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// col[k][pix] (row stride ldn, BF16), row-staged: a block takes one input
// channel c and R consecutive output rows; it stages the 3 input rows of each
// output row (sw Wo + 2 columns) in shared memory and writes the 9 tap rows
// k = 9c .. 9c+8 over those pixels, 4 pixels (8 bytes) per store where the
// pixel index allows. Dynamic shared memory: R * 3 * (sw Wo + 2) floats.
__global__ void __launch_bounds__(256) k_im2col_rows_n(const float* __restrict__ x, const ConvDims d, int R,
                                                       long long ldn, uint16_t* __restrict__ col) {
  extern __shared__ float xs[];  // [R][3][JW]
  const int c = blockIdx.y, row0 = blockIdx.x * R;
  const int nrows = min(R, d.B * d.Ho - row0);
  const int JW = d.sw * d.Wo + 2;
  const float* xc = x + (long long)c * d.B * d.H * d.W;
  for (int e = threadIdx.x; e < nrows * 3 * JW; e += 256) {  // all staging loads independent
    const int rp = e / JW, colx = e - rp * JW;
    const int rl = rp / 3, p = rp - 3 * rl, row = row0 + rl;
    const uint32_t b = d.fHo.div((uint32_t)row);
    const int i = row - (int)b * d.Ho, r = d.sh * i + p - 1, s = colx - 1;
    xs[e] = (r >= 0 && r < d.H && s >= 0 && s < d.W) ? __ldg(xc + ((long long)b * d.H + r) * d.W + s) : 0.f;
  }
  __syncthreads();
  const int q4 = (d.Wo + 3) / 4;  // 4-pixel groups per output row
  const bool vec = (d.Wo & 3) == 0;
  for (int e = threadIdx.x; e < nrows * 9 * q4; e += 256) {
    const int jq = e % q4, t = e / q4, kk = t % 9, rl = t / 9;
    const int p = kk / 3, q = kk - 3 * p;
    const float* xr = xs + (3 * rl + p) * JW;
    const long long n0 = (long long)(row0 + rl) * d.Wo + 4 * jq;
    uint16_t* dst = col + (long long)(9 * c + kk) * ldn + n0;
    uint16_t v[4];
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const int j = 4 * jq + u;
      v[u] = to_bf16_bits(j < d.Wo ? xr[d.sw * j + q] : 0.f);
    }
    if (vec) {
      *reinterpret_cast<uint2*>(dst) = make_uint2((uint32_t)v[0] | ((uint32_t)v[1] << 16),
                                                  (uint32_t)v[2] | ((uint32_t)v[3] << 16));
    } else {
      for (int u = 0; u < 4 && 4 * jq + u < d.Wo; u++) dst[u] = v[u];
    }
  }
}

// The row-staged tap-major im2col for output rows of a multiple of 8 pixels
// (Wo = 8 W8): the staging of k_im2col_rows_n, then item e = (row rl, tap kk,
// 8-pixel group j8) with j8 fastest, decoded by multiply-shift, writes 8
// pixels of one tap row as one 16-byte store (consecutive threads, consecutive
// 16-byte runs of the row). A staged row is kept in 8 column classes: column
// col at (col mod 8) JW8 + col / 8 (JW8 odd), so that the threads of a warp,
// reading the same tap of consecutive 8-pixel groups, read consecutive words.
// Dynamic shared memory: R * 3 * 8 * JW8 floats (im2col_n8_row).
__host__ __device__ __forceinline__ int im2col_n8_row(int JW) { return 8 * (((JW + 7) / 8) | 1); }
__global__ void __launch_bounds__(256) k_im2col_rows_n8(const float* __restrict__ x, const ConvDims d, int R,
                                                        long long ldn, FastDiv fW8, uint16_t* __restrict__ col) {
  extern __shared__ float xs[];  // [R][3][8][JW8]
  const int c = blockIdx.y, row0 = blockIdx.x * R;
  const int nrows = min(R, d.B * d.Ho - row0);
  const int JW = d.sw * d.Wo + 2, JWT = im2col_n8_row(JW), JW8 = JWT / 8;
  const float* xc = x + (long long)c * d.B * d.H * d.W;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int rp = warp; rp < nrows * 3; rp += 8) {  // staged row (output row, tap row)
    const int rl = rp / 3, p = rp - 3 * rl, row = row0 + rl;
    const uint32_t b = d.fHo.div((uint32_t)row);
    const int i = row - (int)b * d.Ho, r = d.sh * i + p - 1;
    const bool rok = r >= 0 && r < d.H;
    const float* src = rok ? xc + ((long long)b * d.H + r) * d.W : xc;
    for (int colx = lane; colx < JW; colx += 32) {
      const int sc = colx - 1;
      xs[rp * JWT + (colx & 7) * JW8 + (colx >> 3)] = (rok && sc >= 0 && sc < d.W) ? __ldg(src + sc) : 0.f;
    }
  }
  __syncthreads();
  const int W8 = (int)fW8.d;
  for (int e = threadIdx.x; e < nrows * 9 * W8; e += 256) {
    const uint32_t t = fW8.div((uint32_t)e);
    const int j8 = e - (int)t * W8, rl = (int)t / 9, kk = (int)t - 9 * rl;
    const int p = kk / 3, q = kk - 3 * p;
    const float* xr = xs + (3 * rl + p) * JWT;
    const int c0 = q + 8 * d.sw * j8;  // staged column of the group's first pixel
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; u++) {
      const int cu = c0 + d.sw * u;
      v[u] = xr[(cu & 7) * JW8 + (cu >> 3)];
    }
    uint32_t w[4];
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * u], v[2 * u + 1]);
      w[u] = *reinterpret_cast<const uint32_t*>(&h);
    }
    const long long n0 = (long long)(row0 + rl) * d.Wo + 8 * j8;
    *reinterpret_cast<uint4*>(col + (long long)(9 * c + kk) * ldn + n0) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// col[k][pix] (row stride ldn, BF16): one tap row per blockIdx.y, 4 pixels per
// thread; the first pixel's (b, i, j) is decoded once and the next ones step
// along the row.
__global__ void __launch_bounds__(256) k_im2col_n(const float* __restrict__ x, const ConvDims d, long long ldn,
                                                  uint16_t* __restrict__ col) {
  const int k = blockIdx.y;
  const int nb = (blockIdx.x * 256 + threadIdx.x) * 4;
  if (nb >= d.Npix) return;
  const int c = k / 9, pq = k - 9 * c, p = pq / 3, q = pq - 3 * p;
  const float* xc = x + (long long)c * d.B * d.H * d.W;
  uint32_t bi = d.fWo.div((uint32_t)nb);
  int j = (int)d.fWo.mod((uint32_t)nb, bi);
  uint32_t b = d.fHo.div(bi);
  int i = (int)d.fHo.mod(bi, b);
  float f[4];
#pragma unroll
  for (int u = 0; u < 4; u++) {
    if (j == d.Wo) {  // next pixel row (next image after its last row)
      j = 0;
      if (++i == d.Ho) {
        i = 0;
        b++;
      }
    }
    const int r = d.sh * i + p - 1, s = d.sw * j + q - 1;
    f[u] = (nb + u < d.Npix && r >= 0 && r < d.H && s >= 0 && s < d.W)
               ? __ldg(xc + ((long long)b * d.H + r) * d.W + s)
               : 0.f;
    j++;
  }
  uint16_t v[4];
#pragma unroll
  for (int u = 0; u < 4; u++) v[u] = to_bf16_bits(f[u]);
  uint16_t* dst = col + (long long)k * ldn + nb;
  if (nb + 3 < d.Npix) {
    *reinterpret_cast<uint2*>(dst) = make_uint2((uint32_t)v[0] | ((uint32_t)v[1] << 16),
                                                (uint32_t)v[2] | ((uint32_t)v[3] << 16));
  } else {
    for (int u = 0; u < 4 && nb + u < d.Npix; u++) dst[u] = v[u];
  }
}

// dx[c][b][r][s] = sum over the taps (p, q) that read (r, s): dcol[c*9+p*3+q][(b*Ho+i)*Wo+j]
// with r = sh i + p - 1, s = sw j + q - 1 (a gather: each output written once, fixed order).
__global__ void __launch_bounds__(256) k_col2im(const float* __restrict__ dcol, const ConvDims d,
                                                float* __restrict__ dx) {
  const int total = d.C * d.B * d.H * d.W;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const uint32_t t1 = d.fW.div((uint32_t)e), t2 = d.fH.div(t1), c = d.fB.div(t2);
    const int s = (int)d.fW.mod((uint32_t)e, t1), r = (int)d.fH.mod(t1, t2), b = (int)d.fB.mod(t2, c);
    float acc = 0.f;
#pragma unroll
    for (int p = 0; p < 3; p++) {
      const int ri = r + 1 - p;
      if (ri < 0 || ri % d.sh != 0) continue;
      const int i = ri / d.sh;
      if (i >= d.Ho) continue;
#pragma unroll
      for (int q = 0; q < 3; q++) {
        const int sj = s + 1 - q;
        if (sj < 0 || sj % d.sw != 0) continue;
        const int j = sj / d.sw;
        if (j >= d.Wo) continue;
        acc += __ldg(dcol + (long long)(c * 9 + p * 3 + q) * d.Npix + (b * d.Ho + i) * d.Wo + j);
      }
    }
    dx[e] = acc;
  }
}

// ReLU backward and the BF16 copy of the pre-activation gradient:
// dy *= (y > 0) if relu (in place, [O][Npix]); dyb[o][pix] = bf16(dy) (row stride ldn);
// part[o][chunk] = sum of the chunk's dy (fixed tree), summed by k_db.
constexpr int ACT_CHUNK = 4096;
__global__ void __launch_bounds__(256) k_act_back(float* __restrict__ dy, const float* __restrict__ y, int Npix,
                                                  long long ldn, int relu, uint16_t* __restrict__ dyb,
                                                  float* __restrict__ part) {
  __shared__ float red[8];
  const int o = blockIdx.y, chunk = blockIdx.x;
  const long long row = (long long)o * Npix;
  float acc = 0.f;
  const int e0 = chunk * ACT_CHUNK, e1 = min(Npix, e0 + ACT_CHUNK);
  for (int n = e0 + threadIdx.x; n < e1; n += 256) {
    float g = dy[row + n];
    if (relu && !(y[row + n] > 0.f)) g = 0.f;
    dy[row + n] = g;
    dyb[(long long)o * ldn + n] = to_bf16_bits(g);
    acc += g;
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int w = 0; w < 8; w++) s += red[w];
    part[(long long)o * gridDim.x + chunk] = s;
  }
}
// db[o] = sum of the chunk partials in chunk order (one thread per channel)
__global__ void k_db(const float* __restrict__ part, int O, int nchunk, float* __restrict__ db) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= O) return;
  float s = 0.f;
  for (int c = 0; c < nchunk; c++) s += part[(long long)o * nchunk + c];
  db[o] = s;
}

// dyT[pix][o] (row stride ldo) = dyb[o][pix] (row stride ldn): 32 x 32 tiles through shared memory
__global__ void k_dy_transpose(const uint16_t* __restrict__ dyb, int O, int Npix, long long ldn, int ldo,
                               uint16_t* __restrict__ dyT) {
  __shared__ uint16_t tile[32][34];
  const int n0 = blockIdx.x * 32, o0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int o = o0 + r, n = n0 + threadIdx.x;
    tile[r][threadIdx.x] = (o < O && n < Npix) ? dyb[(long long)o * ldn + n] : (uint16_t)0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int n = n0 + r, o = o0 + threadIdx.x;
    if (n < Npix && o < ldo) dyT[(long long)n * ldo + o] = tile[threadIdx.x][r];
  }
}

// Weights as GEMM operands: Wp[o][k] (row stride ldk, 16-byte aligned rows) and Wt[k][o] (row stride ldo)
__global__ void k_wprep(const uint16_t* __restrict__ w, int O, int K9, int ldk, int ldo, uint16_t* __restrict__ Wp,
                        uint16_t* __restrict__ Wt) {
  const int total = O * K9;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int o = e / K9, k = e - o * K9;
    const uint16_t v = w[e];
    if (Wp) Wp[(long long)o * ldk + k] = v;
    if (Wt) Wt[(long long)k * ldo + o] = v;
  }
}

// Flipped, transposed weights of a stride-1 layer's data gradient:
// Wf[c][o*9 + p*3 + q] = w[o][c][2-p][2-q] (row stride ldf).
__global__ void k_wflip(const uint16_t* __restrict__ w, int O, int C, int ldf, uint16_t* __restrict__ Wf) {
  const int total = O * C * 9;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int o = e / (C * 9), r = e - o * C * 9, c = r / 9, pq = r - 9 * c;  // e = (o, c, p, q)
    Wf[(long long)c * ldf + o * 9 + (8 - pq)] = w[e];
  }
}

// out[e] = sum over splits s (in order) of part[s * n + e]
__global__ void k_split_sum(const float* __restrict__ part, int splits, long long n, float* __restrict__ out) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int k = 0; k < splits; k++) s += part[(long long)k * n + e];
    out[e] = s;
  }
}

// Input row `row` (= cb H + r) of x feeds output rows 2 row and 2 row + 1 of y
// (cb 2H + 2r = 2 row): blocks walk the input rows, threads the columns, and
// each thread writes its value's 2 x 2 copies as two 8-byte stores (y 8-byte
// aligned; the launcher checks).
__global__ void k_upsample2(const float* __restrict__ x, int CB, int H, int W, float* __restrict__ y) {
  const long long rows = (long long)CB * H, W2 = 2LL * W;
  for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
    const float* xr = x + row * W;
    float2* y0 = reinterpret_cast<float2*>(y + 2 * row * W2);
    float2* y1 = reinterpret_cast<float2*>(y + (2 * row + 1) * W2);
    for (int s = threadIdx.x; s < W; s += blockDim.x) {
      const float v = __ldg(xr + s);
      y0[s] = make_float2(v, v);
      y1[s] = make_float2(v, v);
    }
  }
}

// dx[row][s] = (dy[2 row][2s] + dy[2 row][2s + 1]) + (dy[2 row + 1][2s] + dy[2 row + 1][2s + 1]),
// blocks walking the rows and threads the columns (8-byte loads; dy 8-byte aligned).
__global__ void k_upsample2_back(const float* __restrict__ dy, int CB, int H, int W, float* __restrict__ dx) {
  const long long rows = (long long)CB * H, W2 = 2LL * W;
  for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
    const float2* d0 = reinterpret_cast<const float2*>(dy + 2 * row * W2);
    const float2* d1 = reinterpret_cast<const float2*>(dy + (2 * row + 1) * W2);
    for (int s = threadIdx.x; s < W; s += blockDim.x) {
      const float2 a = __ldg(d0 + s), b = __ldg(d1 + s);
      dx[row * W + s] = (a.x + a.y) + (b.x + b.y);
    }
  }
}

// loss = 1/(2n) sum (p - t)^2 in FP64, dp = (p - t)/n: each block sums a fixed
// slice of the elements (fixed tree) into part[block]; k_mse_final adds the
// block partials in block order. MSE_BLOCKS is fixed, so the order is too.
constexpr int MSE_BLOCKS = 304;
__global__ void __launch_bounds__(256) k_mse(const float* __restrict__ p, const float* __restrict__ t, long long n,
                                             double* __restrict__ part, float* __restrict__ dp) {
  __shared__ double red[8];
  double acc = 0.0;
  const float inv = (float)(1.0 / (double)n);
  for (long long e = blockIdx.x * 256LL + threadIdx.x; e < n; e += (long long)MSE_BLOCKS * 256) {
    const float r = p[e] - t[e];
    dp[e] = r * inv;
    acc += (double)r * (double)r;
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; w++) s += red[w];
    part[blockIdx.x] = s;
  }
}
__global__ void k_mse_final(const double* __restrict__ part, long long n, double* loss) {
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < MSE_BLOCKS; k++) s += part[k];
    *loss = 0.5 * s / (double)n;
  }
}

__global__ void k_adam(float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1,
                       float c2, uint16_t* __restrict__ thb) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const float gi = g[e];
    const float mi = b1 * m[e] + (1.f - b1) * gi;
    const float vi = b2 * v[e] + (1.f - b2) * gi * gi;
    m[e] = mi;
    v[e] = vi;
    const float t = th[e] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    th[e] = t;
    if (thb) thb[e] = to_bf16_bits(t);
  }
}

__global__ void k_to_bf16(const float* __restrict__ x, uint16_t* __restrict__ y, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    y[e] = to_bf16_bits(x[e]);
}

int blocks_for(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152 * 16)); }

}  // namespace
}  // namespace fwi

// ---------------------------------------------------------------------------
// C ABI
struct fwi_cnn {
  int device = 0;
  void* ws = nullptr;     // workspace of the layer calls (grows to the largest layer)
  size_t ws_bytes = 0;
  int* status = nullptr;  // device status word of the GEMMs (timeout bit)
  double* red = nullptr;  // block partials of the loss reduction
  bool gather = true;     // forward / stride-1 data-gradient GEMMs gather their tap operand (no im2col matrix)
};

namespace {

using fwi::blocks_for;

fwi_status cuda_fail(cudaError_t e, const char* what) {
  return fwi::host_fail(FWI_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CNN_CK(call, what)                              \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, what);  \
  } while (0)

bool bad_dims(int C, int B, int H, int W) { return C < 1 || B < 1 || H < 1 || W < 1; }

// Carves 256-byte aligned pieces out of the handle's workspace.
struct Carve {
  size_t off = 0;
  size_t take(size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) / 256 * 256;
    return o;
  }
};

// Grow the workspace to `bytes` (cudaFree synchronises the device, so no call
// still in flight uses the old buffer).
fwi_status ws_reserve(fwi_cnn* h, size_t bytes) {
  if (bytes <= h->ws_bytes) return FWI_OK;
  if (h->ws) CNN_CK(cudaFree(h->ws), "cudaFree");
  h->ws = nullptr;
  h->ws_bytes = 0;
  const size_t want = bytes + bytes / 4;
  CNN_CK(cudaMalloc(&h->ws, want), "cudaMalloc (cnn workspace)");
  h->ws_bytes = want;
  return FWI_OK;
}

fwi_status dims_of(int C, int B, int H, int W, int sh, int sw, fwi::ConvDims* d) {
  d->C = C; d->B = B; d->H = H; d->W = W; d->sh = sh; d->sw = sw;
  d->Ho = fwi::conv_out(H, sh);
  d->Wo = fwi::conv_out(W, sw);
  const long long npix = (long long)B * d->Ho * d->Wo, k9 = 9LL * C;
  if (npix > 0x7fffff00LL || k9 > 65535 || (long long)C * B * H * W > 0x7fffff00LL)
    return fwi::host_fail(FWI_EINVAL, "layer too large");
  d->K9 = (int)k9;
  d->Npix = (int)npix;
  d->fWo = fwi::FastDiv((uint32_t)d->Wo);
  d->fHo = fwi::FastDiv((uint32_t)d->Ho);
  d->fW = fwi::FastDiv((uint32_t)W);
  d->fH = fwi::FastDiv((uint32_t)H);
  d->fB = fwi::FastDiv((uint32_t)B);
  return FWI_OK;
}

// The row-staged im2col kernels where their staging fits in shared memory
// (every layer of the network does), else the per-element ones.
cudaError_t im2col_t(const float* x, const fwi::ConvDims& d, int ldk, uint16_t* colT, cudaStream_t st) {
  const size_t smem = (size_t)fwi::IM_CC * 3 * (fwi::IM_PIX * d.sw + 2) * sizeof(float);
  const int rows = d.B * d.Ho;
  if (smem <= 48 * 1024 && d.C <= 65535 * fwi::IM_CC) {
    const dim3 grid((unsigned)rows, (unsigned)((d.Wo + fwi::IM_PIX - 1) / fwi::IM_PIX),
                    (unsigned)((d.C + fwi::IM_CC - 1) / fwi::IM_CC));
    fwi::k_im2col_rows_t<<<grid, fwi::IM_T_THREADS, smem, st>>>(x, d, ldk, colT);
  } else {
    fwi::k_im2col_t<<<dim3((d.Npix + 63) / 64, (ldk + 63) / 64), 256, 0, st>>>(x, d, ldk, colT);
  }
  return cudaGetLastError();
}
cudaError_t im2col_n(const float* x, const fwi::ConvDims& d, long long ldn, uint16_t* col, cudaStream_t st) {
  const int R = std::max(1, std::min(16, 1024 / std::max(1, d.Wo)));
  const size_t smem = (size_t)R * 3 * (d.sw * d.Wo + 2) * sizeof(float);
  const size_t smem8 = (size_t)R * 3 * fwi::im2col_n8_row(d.sw * d.Wo + 2) * sizeof(float);
  const int rows = d.B * d.Ho;
  if (smem8 <= 48 * 1024 && d.C <= 65535 && d.Wo % 8 == 0) {
    fwi::k_im2col_rows_n8<<<dim3((unsigned)((rows + R - 1) / R), (unsigned)d.C), 256, smem8, st>>>(
        x, d, R, ldn, fwi::FastDiv((uint32_t)(d.Wo / 8)), col);
  } else if (smem <= 48 * 1024 && d.C <= 65535) {
    fwi::k_im2col_rows_n<<<dim3((unsigned)((rows + R - 1) / R), (unsigned)d.C), 256, smem, st>>>(x, d, R, ldn, col);
  } else {
    fwi::k_im2col_n<<<dim3((d.Npix + 1023) / 1024, d.K9), 256, 0, st>>>(x, d, ldn, col);
  }
  return cudaGetLastError();
}

int gemm_blocks(long long tiles_per_split) {
  // splits so that about two waves of CTAs cover the GPU's 152 SMs
  return (int)std::max<long long>(1, (2 * 152 + tiles_per_split - 1) / tiles_per_split);
}

}  // namespace

extern "C" {

fwi_status fwi_cnn_create(fwi_cnn** h, int device) {
  if (!h) return fwi::host_fail(FWI_EINVAL, "h must not be NULL");
  CNN_CK(cudaSetDevice(device), "cudaSetDevice");
  fwi_cnn* c = new fwi_cnn;
  c->device = device;
  cudaError_t e = cudaMalloc(&c->status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(c->status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&c->red, fwi::MSE_BLOCKS * sizeof(double));
  if (e != cudaSuccess) {
    if (c->status) cudaFree(c->status);
    if (c->red) cudaFree(c->red);
    delete c;
    return cuda_fail(e, "cudaMalloc (status)");
  }
  *h = c;
  return FWI_OK;
}

fwi_status fwi_cnn_destroy(fwi_cnn* h) {
  if (!h) return FWI_OK;
  cudaSetDevice(h->device);
  if (h->ws) cudaFree(h->ws);
  if (h->status) cudaFree(h->status);
  if (h->red) cudaFree(h->red);
  delete h;
  return FWI_OK;
}

fwi_status fwi_cnn_check(fwi_cnn* h, void* stream) {
  if (!h) return fwi::host_fail(FWI_EINVAL, "h must not be NULL");
  CNN_CK(cudaSetDevice(h->device), "cudaSetDevice");
  int st = 0;
  CNN_CK(cudaMemcpyAsync(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream), "status read");
  CNN_CK(cudaStreamSynchronize((cudaStream_t)stream), "cudaStreamSynchronize");
  if (st) {
    CNN_CK(cudaMemset(h->status, 0, sizeof(int)), "status clear");
    return fwi::host_fail(FWI_ETIMEOUT, "a tensor-core GEMM wait timed out; its output holds NaN");
  }
  return FWI_OK;
}

fwi_status fwi_cnn_set_conv_gather(fwi_cnn* h, int32_t on) {
  if (!h) return fwi::host_fail(FWI_EINVAL, "h must not be NULL");
  h->gather = on != 0;
  return FWI_OK;
}

fwi_status fwi_cnn_gemm_bt(fwi_cnn* h, const uint16_t* A, int64_t lda, const uint16_t* B, int64_t ldb, int64_t M,
                           int32_t N, int64_t K, float* out, int64_t ldo, const float* bias, int32_t relu,
                           int32_t splits, void* stream) {
  if (!h || !A || !B || !out) return fwi::host_fail(FWI_EINVAL, "NULL pointer");
  if (M < 1 || N < 1 || K < 1 || splits < 1 || ldo < M || lda < K || ldb < K || lda % 8 || ldb % 8)
    return fwi::host_fail(FWI_EINVAL, "bad sizes or leading dimensions (lda, ldb: multiples of 8, >= K; ldo >= M)");
  if (((uintptr_t)A & 15) || ((uintptr_t)B & 15)) return fwi::host_fail(FWI_EINVAL, "A and B must be 16-byte aligned");
  CNN_CK(cudaSetDevice(h->device), "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)stream;
  const int S = fwi::tc_split_count(K, splits);
  float* dst = out;
  if (S > 1) {
    const fwi_status v = ws_reserve(h, (size_t)S * N * ldo * sizeof(float));
    if (v != FWI_OK) return v;
    dst = (float*)h->ws;
  }
  fwi::TcGemm g{A, lda, B, ldb, M, N, K, dst, ldo, (long long)N * ldo, S > 1 ? nullptr : bias, S > 1 ? 0 : relu, S,
                h->status};
  CNN_CK(fwi::tc_gemm(g, st), "tcgen05 GEMM");
  if (S > 1) {
    if (bias || relu) return fwi::host_fail(FWI_EINVAL, "bias / relu need splits == 1");
    fwi::k_split_sum<<<blocks_for((long long)N * ldo), 256, 0, st>>>(dst, S, (long long)N * ldo, out);
    CNN_CK(cudaGetLastError(), "split sum");
  }
  return FWI_OK;
}

fwi_status fwi_cnn_conv_forward(fwi_cnn* h, const float* x, int32_t C, int32_t B, int32_t H, int32_t W,
                                const uint16_t* w_bf16, const float* bias, int32_t O, int32_t sh, int32_t sw,
                                int32_t relu, float* y, void* stream) {
  if (!h || !x || !w_bf16 || !bias || !y) return fwi::host_fail(FWI_EINVAL, "NULL pointer");
  if (bad_dims(C, B, H, W) || O < 1 || sh < 1 || sw < 1) return fwi::host_fail(FWI_EINVAL, "bad sizes");
  fwi::ConvDims d;
  fwi_status v = dims_of(C, B, H, W, sh, sw, &d);
  if (v != FWI_OK) return v;
  CNN_CK(cudaSetDevice(h->device), "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)stream;
  const int ldk = (int)fwi::round8(d.K9);
  const bool gather = h->gather;
  Carve cv;
  const size_t o_col = cv.take(gather ? 0 : (size_t)d.Npix * ldk * 2), o_wp = cv.take((size_t)O * ldk * 2);
  if ((v = ws_reserve(h, cv.off)) != FWI_OK) return v;
  char* ws = (char*)h->ws;
  uint16_t* colT = (uint16_t*)(ws + o_col);
  uint16_t* Wp = (uint16_t*)(ws + o_wp);
  fwi::k_wprep<<<blocks_for((long long)O * d.K9), 256, 0, st>>>(w_bf16, O, d.K9, ldk, 0, Wp, nullptr);
  CNN_CK(cudaGetLastError(), "weight layout");
  const fwi::TcConvA ca = fwi::tc_conv_a(x, C, B, H, W, sh, sw);
  if (!gather) CNN_CK(im2col_t(x, d, ldk, colT, st), "im2col");
  fwi::TcGemm g{gather ? nullptr : colT, ldk, Wp, ldk, d.Npix, O, d.K9, y, d.Npix, 0, bias, relu, 1, h->status,
                gather ? &ca : nullptr};
  CNN_CK(fwi::tc_gemm(g, st), "conv forward GEMM");
  return FWI_OK;
}

fwi_status fwi_cnn_conv_backward(fwi_cnn* h, const float* x, int32_t C, int32_t B, int32_t H, int32_t W,
                                 const uint16_t* w_bf16, int32_t O, int32_t sh, int32_t sw, int32_t relu,
                                 const float* y, float* dy, float* dx, float* dw, float* db, void* stream) {
  if (!h || !x || !w_bf16 || !y || !dy || !dw || !db) return fwi::host_fail(FWI_EINVAL, "NULL pointer");
  if (bad_dims(C, B, H, W) || O < 1 || sh < 1 || sw < 1) return fwi::host_fail(FWI_EINVAL, "bad sizes");
  fwi::ConvDims d;
  fwi_status v = dims_of(C, B, H, W, sh, sw, &d);
  if (v != FWI_OK) return v;
  CNN_CK(cudaSetDevice(h->device), "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)stream;
  const long long ldn = fwi::round8(d.Npix);
  const int ldo = (int)fwi::round8(O);
  const int nchunk = (d.Npix + fwi::ACT_CHUNK - 1) / fwi::ACT_CHUNK;
  // weight gradient split over pixel runs: about two waves of CTAs
  const long long mt = (d.K9 + 127) / 128, nt = (O + 255) / 256;
  const int S = fwi::tc_split_count(d.Npix, gemm_blocks(mt * nt));
  // stride-1 data gradient: dy seen as a [O][B][H][W] activation, convolved with the flipped weights
  fwi::ConvDims dd = d;
  dd.C = O;
  dd.K9 = 9 * O;
  dd.Npix = B * H * W;  // = d.Npix at stride 1
  const int ldf = (int)fwi::round8(dd.K9);
  const bool s1 = sh == 1 && sw == 1;
  Carve cv;
  const size_t o_dyb = cv.take((size_t)O * ldn * 2), o_bp = cv.take((size_t)O * nchunk * 4);
  size_t colb_elems = (size_t)d.K9 * ldn;
  if (dx) colb_elems = std::max(colb_elems, s1 ? (h->gather ? 0 : (size_t)dd.Npix * ldf) : (size_t)d.Npix * ldo);
  const size_t o_col = cv.take(colb_elems * 2);
  const size_t o_wt = cv.take(dx ? (size_t)(s1 ? C * ldf : d.K9 * ldo) * 2 : 0);
  const size_t o_dcol = cv.take(dx && !s1 ? (size_t)d.K9 * d.Npix * 4 : 0);
  const size_t o_part = cv.take(S > 1 ? (size_t)S * O * d.K9 * 4 : 0);
  if ((v = ws_reserve(h, cv.off)) != FWI_OK) return v;
  char* ws = (char*)h->ws;
  uint16_t* dyb = (uint16_t*)(ws + o_dyb);
  float* bpart = (float*)(ws + o_bp);
  uint16_t* colb = (uint16_t*)(ws + o_col);
  uint16_t* Wt = (uint16_t*)(ws + o_wt);
  uint16_t* Wf = Wt;  // stride 1: the flipped weights in the same slot
  float* dcol = (float*)(ws + o_dcol);
  float* part = (float*)(ws + o_part);

  fwi::k_act_back<<<dim3(nchunk, O), 256, 0, st>>>(dy, y, d.Npix, ldn, relu, dyb, bpart);
  CNN_CK(cudaGetLastError(), "activation backward");
  fwi::k_db<<<(O + 127) / 128, 128, 0, st>>>(bpart, O, nchunk, db);
  CNN_CK(cudaGetLastError(), "bias gradient");
  if (dx && s1) {
    // stride 1: dx is the convolution of the pre-activation gradient with the
    // flipped, transposed weights, dx[c][pix] = sum_{o,p,q} dy[o][pix shifted by (1-p, 1-q)] w[o][c][p][q]:
    // im2col of dy (BF16, the same rounding as dyb) and one GEMM, no dcol / col2im
    fwi::k_wflip<<<blocks_for(9LL * O * C), 256, 0, st>>>(w_bf16, O, C, ldf, Wf);
    CNN_CK(cudaGetLastError(), "weight flip");
    const fwi::TcConvA ca = fwi::tc_conv_a(dy, O, B, H, W, 1, 1);
    if (!h->gather) CNN_CK(im2col_t(dy, dd, ldf, colb, st), "im2col of dy");
    fwi::TcGemm g{h->gather ? nullptr : colb, ldf, Wf, ldf, dd.Npix, C, dd.K9, dx, dd.Npix, 0, nullptr, 0, 1,
                  h->status, h->gather ? &ca : nullptr};
    CNN_CK(fwi::tc_gemm(g, st), "conv data-gradient GEMM");
  } else if (dx) {
    // dcol[k][pix] = sum_o dyT[pix][o] W[o][k], then the col2im gather
    fwi::k_dy_transpose<<<dim3((d.Npix + 31) / 32, (ldo + 31) / 32), dim3(32, 8), 0, st>>>(dyb, O, d.Npix, ldn, ldo,
                                                                                          colb);
    CNN_CK(cudaGetLastError(), "dy transpose");
    fwi::k_wprep<<<blocks_for((long long)O * d.K9), 256, 0, st>>>(w_bf16, O, d.K9, 0, ldo, nullptr, Wt);
    CNN_CK(cudaGetLastError(), "weight layout");
    fwi::TcGemm g{colb, ldo, Wt, ldo, d.Npix, d.K9, O, dcol, d.Npix, 0, nullptr, 0, 1, h->status};
    CNN_CK(fwi::tc_gemm(g, st), "conv data-gradient GEMM");
    fwi::k_col2im<<<blocks_for((long long)C * B * H * W), 256, 0, st>>>(dcol, d, dx);
    CNN_CK(cudaGetLastError(), "col2im");
  }
  // dw[o][k] = sum_pix col[k][pix] dy[o][pix]
  CNN_CK(im2col_n(x, d, ldn, colb, st), "im2col");
  fwi::TcGemm g{colb, ldn, dyb, ldn, d.K9, O, d.Npix, S > 1 ? part : dw, d.K9, (long long)O * d.K9, nullptr, 0, S,
                h->status};
  CNN_CK(fwi::tc_gemm(g, st), "conv weight-gradient GEMM");
  if (S > 1) {
    fwi::k_split_sum<<<blocks_for((long long)O * d.K9), 256, 0, st>>>(part, S, (long long)O * d.K9, dw);
    CNN_CK(cudaGetLastError(), "split sum");
  }
  return FWI_OK;
}

fwi_status fwi_cnn_upsample2(const float* x, int32_t C, int32_t B, int32_t H, int32_t W, float* y, void* stream) {
  if (!x || !y) return fwi::host_fail(FWI_EINVAL, "NULL pointer");
  if (bad_dims(C, B, H, W)) return fwi::host_fail(FWI_EINVAL, "bad sizes");
  if ((long long)C * B * 4 * H * W > 0x7fffff00LL) return fwi::host_fail(FWI_EINVAL, "tensor too large");
  if ((uintptr_t)y & 7) return fwi::host_fail(FWI_EINVAL, "y must be 8-byte aligned");
  const int CB = C * B;
  const long long rows = (long long)CB * H;
  fwi::k_upsample2<<<(unsigned)std::min<long long>(rows, 65535LL * 16), W >= 256 ? 256 : 128, 0,
                     (cudaStream_t)stream>>>(x, CB, H, W, y);
  CNN_CK(cudaGetLastError(), "upsample");
  return FWI_OK;
}

fwi_status fwi_cnn_upsample2_backward(const float* dy, int32_t C, int32_t B, int32_t H, int32_t W, float* dx,
                                      void* stream) {
  if (!dy || !dx) return fwi::host_fail(FWI_EINVAL, "NULL pointer");
  if (bad_dims(C, B, H, W)) return fwi::host_fail(FWI_EINVAL, "bad sizes");
  if ((long long)C * B * 4 * H * W > 0x7fffff00LL) return fwi::host_fail(FWI_EINVAL, "tensor too large");
  if ((uintptr_t)dy & 7) return fwi::host_fail(FWI_EINVAL, "dy must be 8-byte aligned");
  const int CB = C * B;
  const long long rows = (long long)CB * H;
  fwi::k_upsample2_back<<<(unsigned)std::min<long long>(rows, 65535LL * 16), W >= 256 ? 256 : 128, 0,
                          (cudaStream_t)stream>>>(dy, CB, H, W, dx);
  CNN_CK(cudaGetLastError(), "upsample backward");
  return FWI_OK;
}

fwi_status fwi_cnn_mse(fwi_cnn* h, const float* p, const float* t, int64_t n, double* loss, float* dp,
                       void* stream) {
  if (!h || !p || !t || !loss || !dp) return fwi::host_fail(FWI_EINVAL, "NULL pointer");
  if (n < 1) return fwi::host_fail(FWI_EINVAL, "n must be >= 1");
  CNN_CK(cudaSetDevice(h->device), "cudaSetDevice");
  fwi::k_mse<<<fwi::MSE_BLOCKS, 256, 0, (cudaStream_t)stream>>>(p, t, n, h->red, dp);
  CNN_CK(cudaGetLastError(), "mse");
  fwi::k_mse_final<<<1, 32, 0, (cudaStream_t)stream>>>(h->red, n, loss);
  CNN_CK(cudaGetLastError(), "mse");
  return FWI_OK;
}

fwi_status fwi_cnn_adam(float* theta, const float* g, float* m, float* v, int64_t n, int32_t step, float lr,
                        float beta1, float beta2, float eps, uint16_t* theta_bf16, void* stream) {
  if (!theta || !g || !m || !v) return fwi::host_fail(FWI_EINVAL, "NULL pointer");
  if (n < 1 || step < 1) return fwi::host_fail(FWI_EINVAL, "n and step must be >= 1");
  const float c1 = (float)(1.0 - std::pow((double)beta1, step)), c2 = (float)(1.0 - std::pow((double)beta2, step));
  fwi::k_adam<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(theta, g, m, v, n, lr, beta1, beta2, eps, c1, c2,
                                                               theta_bf16);
  CNN_CK(cudaGetLastError(), "adam");
  return FWI_OK;
}

fwi_status fwi_cnn_to_bf16(const float* x, uint16_t* y, int64_t n, void* stream) {
  if (!x || !y) return fwi::host_fail(FWI_EINVAL, "NULL pointer");
  if (n < 1) return fwi::host_fail(FWI_EINVAL, "n must be >= 1");
  fwi::k_to_bf16<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(x, y, n);
  CNN_CK(cudaGetLastError(), "to_bf16");
  return FWI_OK;
}

}  // extern "C"
