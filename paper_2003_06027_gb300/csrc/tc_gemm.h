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
};

cudaError_t tc_gemm(const TcGemm& g, cudaStream_t st);

// Number of 64-wide k-blocks of a K-long contraction, and the number of
// partials tc_gemm writes when asked for `want` splits (at most want; every
// partial covers at least one k-block).
inline long long tc_kblocks(long long K) { return (K + 63) / 64; }
int tc_split_count(long long K, int want);

}  // namespace fwi
