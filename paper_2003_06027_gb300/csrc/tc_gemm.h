// tc_gemm.h - BF16 tensor-core GEMM of libfwi (tcgen05 + TMA + TMEM, sm_103a).
// Internal to the library: the convolution layers of the start-model network
// call it (cnn.cu); fwi_cnn_gemm_bt exposes it through the C ABI.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace fwi {

// out[split][n][m] = act(sum_{k in split} A[m][k] * B[n][k] + bias[n])
//
//   A: M rows of K BF16 values, row stride lda elements (K-major; lda % 8 == 0)
//   B: N rows of K BF16 values, row stride ldb elements (K-major; ldb % 8 == 0)
//   out: FP32, element (n, m) of split s at out[s * split_stride + n * ldo + m]
//        (the product is written transposed: m is the contiguous index)
//   bias: [N] FP32 or nullptr; relu: max(., 0) after the bias
//   splits: the K range is cut into `splits` contiguous runs of 64-wide
//           k-blocks; each run writes its own partial (no atomics)
//   status: device int; a bounded wait that gives up ORs 32 (timeout) into it
// Returns cudaSuccess, or the launch / tensor-map error (cudaErrorInvalidValue
// for sizes or alignments the kernel does not take).
// The A operand of a 3x3 convolution (padding 1, strides sh, sw) gathered
// on the fly instead of read from an im2col matrix: A[m][k] = BF16(x[c][b][r][s])
// for output pixel m = (b * Ho + i) * Wo + j and tap k = 9 c + 3 p + q, with
// r = sh i + p - 1, s = sw j + q - 1, and 0 outside the image or for k >= 9 C.
// x is FP32, channel-major [C][B][H][W]. The divisions by Wo and Ho use the
// multiply-shift constants filled in by tc_conv_a().
struct TcConvA {
  const float* x;
  int C, B, H, W, Ho, Wo, sh, sw;
  unsigned long long wo_m, ho_m;
  uint32_t wo_s, ho_s;
};
TcConvA tc_conv_a(const float* x, int C, int B, int H, int W, int sh, int sw);

struct TcGemm {
  const uint16_t* A;
  long long lda;
  const uint16_t* B;
  long long ldb;
  long long M;
  int N;
  long long K;
  float* out;
  long long ldo;
  long long split_stride;
  const float* bias;
  int relu;
  int splits;
  int* status;
  // if not null, A (and lda) are ignored and A is gathered from conv->x
  // (M = B Ho Wo pixels, K = 9 C taps); the results equal those of the
  // im2col matrix of the same layer bit for bit
  const TcConvA* conv = nullptr;
};

cudaError_t tc_gemm(const TcGemm& g, cudaStream_t st);

// Number of 64-wide k-blocks of a K-long contraction, and the number of
// partials tc_gemm writes when asked for `want` splits (at most want; every
// partial covers at least one k-block).
inline long long tc_kblocks(long long K) { return (K + 63) / 64; }
int tc_split_count(long long K, int want);

}  // namespace fwi
