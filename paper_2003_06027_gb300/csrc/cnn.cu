// cnn.cu - layers of the learned start-model network (sm_103a).
//
// The one dense contraction of the project: 3x3 convolutions written as GEMMs
// over the whole batch (activations are channel-major [C][B][H][W], so the
// im2col matrix of a layer is [C*9][B*Ho*Wo] and y = W col is a single
// [O][C*9] x [C*9][B*Ho*Wo] product). The GEMMs run on the tensor cores through
// cuBLAS with BF16 operands and FP32 accumulation; the data movement around
// them (im2col with the FP32 -> BF16 rounding, col2im as a deterministic gather,
// bias + ReLU epilogue, bias gradient, upsampling, loss, Adam) is in the kernels
// below. No floating-point atomics: every reduction has a fixed order.
#include <cublas_v2.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "fwi_cnn.h"
#include "fwi_host.h"

namespace fwi {
namespace {

__device__ __forceinline__ uint16_t to_bf16_bits(float f) {
  const __nv_bfloat16 b = __float2bfloat16_rn(f);
  return *reinterpret_cast<const uint16_t*>(&b);
}

__host__ __device__ __forceinline__ int conv_out(int n, int s) { return (n - 1) / s + 1; }

// col[k][n], k = c*9 + p*3 + q, n = (b*Ho + i)*Wo + j  <-  x[c][b][sh i + p - 1][sw j + q - 1] (0 outside)
__global__ void k_im2col(const float* __restrict__ x, int C, int B, int H, int W, int sh, int sw, int Ho, int Wo,
                         uint16_t* __restrict__ col) {
  const long long N = (long long)B * Ho * Wo, total = (long long)C * 9 * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long k = e / N, n = e - k * N;
    const int c = (int)(k / 9), pq = (int)(k - (long long)c * 9), p = pq / 3, q = pq - 3 * p;
    const int j = (int)(n % Wo);
    const long long bi = n / Wo;
    const int i = (int)(bi % Ho), b = (int)(bi / Ho);
    const int r = sh * i + p - 1, s = sw * j + q - 1;
    float v = 0.f;
    if (r >= 0 && r < H && s >= 0 && s < W) v = x[(((long long)c * B + b) * H + r) * W + s];
    col[e] = to_bf16_bits(v);
  }
}

// dx[c][b][r][s] = sum over the taps (p, q) that read (r, s): dcol[c*9+p*3+q][(b*Ho+i)*Wo+j]
// with r = sh i + p - 1, s = sw j + q - 1 (a gather: each output written once, fixed order).
__global__ void k_col2im(const float* __restrict__ dcol, int C, int B, int H, int W, int sh, int sw, int Ho, int Wo,
                         float* __restrict__ dx) {
  const long long N = (long long)B * Ho * Wo, total = (long long)C * B * H * W;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(e % W);
    const long long t1 = e / W;
    const int r = (int)(t1 % H);
    const long long t2 = t1 / H;
    const int b = (int)(t2 % B), c = (int)(t2 / B);
    float acc = 0.f;
    for (int p = 0; p < 3; p++) {
      const int ri = r + 1 - p;
      if (ri < 0 || ri % sh != 0) continue;
      const int i = ri / sh;
      if (i >= Ho) continue;
      for (int q = 0; q < 3; q++) {
        const int sj = s + 1 - q;
        if (sj < 0 || sj % sw != 0) continue;
        const int j = sj / sw;
        if (j >= Wo) continue;
        acc += dcol[(long long)(c * 9 + p * 3 + q) * N + ((long long)b * Ho + i) * Wo + j];
      }
    }
    dx[e] = acc;
  }
}

// y[o][n] += bias[o]; optional ReLU
__global__ void k_bias_act(float* __restrict__ y, const float* __restrict__ bias, long long N, int O, int relu) {
  const long long total = (long long)O * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    float v = y[e] + bias[e / N];
    y[e] = relu ? fmaxf(v, 0.f) : v;
  }
}

// dy *= (y > 0) if relu; dy_bf16 = bf16(dy); db[o] = sum_n dy[o][n] (one block per channel, fixed tree)
__global__ void k_act_back(float* __restrict__ dy, const float* __restrict__ y, long long N, int relu,
                           uint16_t* __restrict__ dyb, float* __restrict__ db) {
  __shared__ float red[32];
  const int o = blockIdx.x;
  float acc = 0.f;
  for (long long n = threadIdx.x; n < N; n += blockDim.x) {
    const long long e = (long long)o * N + n;
    float g = dy[e];
    if (relu && !(y[e] > 0.f)) g = 0.f;
    dy[e] = g;
    dyb[e] = to_bf16_bits(g);
    acc += g;
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += red[w];
    db[o] = s;
  }
}

__global__ void k_upsample2(const float* __restrict__ x, long long CB, int H, int W, float* __restrict__ y) {
  const long long total = CB * 4 * H * W;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(e % (2 * W));
    const long long t = e / (2 * W);
    const int r = (int)(t % (2 * H));
    const long long cb = t / (2 * H);
    y[e] = x[(cb * H + r / 2) * W + s / 2];
  }
}

__global__ void k_upsample2_back(const float* __restrict__ dy, long long CB, int H, int W, float* __restrict__ dx) {
  const long long total = CB * H * W;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(e % W);
    const long long t = e / W;
    const int r = (int)(t % H);
    const long long cb = t / H;
    const float* d = dy + (cb * 2 * H + 2 * r) * (2 * W) + 2 * s;
    dx[e] = (d[0] + d[1]) + (d[2 * W] + d[2 * W + 1]);
  }
}

// loss = 1/(2n) sum (p - t)^2 in FP64 (one block, fixed order), dp = (p - t)/n
__global__ void k_mse(const float* __restrict__ p, const float* __restrict__ t, long long n, double* loss,
                      float* __restrict__ dp) {
  __shared__ double red[32];
  double acc = 0.0;
  const float inv = (float)(1.0 / (double)n);
  for (long long e = threadIdx.x; e < n; e += blockDim.x) {
    const float r = p[e] - t[e];
    dp[e] = r * inv;
    acc += (double)r * (double)r;
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += red[w];
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
  cublasHandle_t blas = nullptr;
};

namespace {

using fwi::blocks_for;

fwi_status cuda_fail(cudaError_t e, const char* what) {
  return fwi::host_fail(FWI_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
fwi_status blas_fail(cublasStatus_t s, const char* what) {
  return fwi::host_fail(FWI_ECUDA, std::string(what) + ": cuBLAS status " + std::to_string((int)s));
}

#define CNN_CK(call, what)                              \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, what);  \
  } while (0)
#define CNN_BLAS(call, what)                                        \
  do {                                                              \
    cublasStatus_t s_ = (call);                                     \
    if (s_ != CUBLAS_STATUS_SUCCESS) return blas_fail(s_, what);    \
  } while (0)

// Row-major C[M][N] = A[M][K] . B[K][N] with BF16 A, B and FP32 C, as the
// column-major product C^T = B^T A^T (cuBLAS is column-major). ta / tb say
// whether the row-major operand is stored transposed ([K][M] / [N][K]).
fwi_status gemm_rm(cublasHandle_t h, bool ta, bool tb, int M, int N, int K, const uint16_t* A, const uint16_t* B,
                   float* C, const char* what) {
  const float one = 1.f, zero = 0.f;
  const int lda = ta ? M : K, ldb = tb ? K : N;
  CNN_BLAS(cublasGemmEx(h, tb ? CUBLAS_OP_T : CUBLAS_OP_N, ta ? CUBLAS_OP_T : CUBLAS_OP_N, N, M, K, &one, B,
                        CUDA_R_16BF, ldb, A, CUDA_R_16BF, lda, &zero, C, CUDA_R_32F, N, CUBLAS_COMPUTE_32F,
                        CUBLAS_GEMM_DEFAULT),
           what);
  return FWI_OK;
}

bool bad_dims(int C, int B, int H, int W) { return C < 1 || B < 1 || H < 1 || W < 1; }

}  // namespace

extern "C" {

fwi_status fwi_cnn_create(fwi_cnn** h, int device) {
  if (!h) return fwi::host_fail(FWI_EINVAL, "h must not be NULL");
  CNN_CK(cudaSetDevice(device), "cudaSetDevice");
  fwi_cnn* c = new fwi_cnn;
  c->device = device;
  cublasStatus_t s = cublasCreate(&c->blas);
  if (s != CUBLAS_STATUS_SUCCESS) {
    delete c;
    return blas_fail(s, "cublasCreate");
  }
  *h = c;
  return FWI_OK;
}

fwi_status fwi_cnn_destroy(fwi_cnn* h) {
  if (!h) return FWI_OK;
  cudaSetDevice(h->device);
  if (h->blas) cublasDestroy(h->blas);
  delete h;
  return FWI_OK;
}

fwi_status fwi_cnn_conv_forward(fwi_cnn* h, const float* x, int32_t C, int32_t B, int32_t H, int32_t W,
                                const uint16_t* w_bf16, const float* bias, int32_t O, int32_t sh, int32_t sw,
                                int32_t relu, uint16_t* col, float* y, void* stream) {
  if (!h || !x || !w_bf16 || !bias || !col || !y) return fwi::host_fail(FWI_EINVAL, "NULL pointer");
  if (bad_dims(C, B, H, W) || O < 1 || sh < 1 || sw < 1) return fwi::host_fail(FWI_EINVAL, "bad sizes");
  CNN_CK(cudaSetDevice(h->device), "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)stream;
  const int Ho = fwi::conv_out(H, sh), Wo = fwi::conv_out(W, sw);
  const long long N = (long long)B * Ho * Wo, K = 9LL * C;
  if (N > 0x7fffffffLL || K * N > (1LL << 40)) return fwi::host_fail(FWI_EINVAL, "layer too large for one GEMM");
  fwi::k_im2col<<<blocks_for(K * N), 256, 0, st>>>(x, C, B, H, W, sh, sw, Ho, Wo, col);
  CNN_CK(cudaGetLastError(), "im2col");
  CNN_BLAS(cublasSetStream(h->blas, st), "cublasSetStream");
  fwi_status v = gemm_rm(h->blas, false, false, O, (int)N, (int)K, w_bf16, col, y, "conv forward GEMM");
  if (v != FWI_OK) return v;
  fwi::k_bias_act<<<blocks_for((long long)O * N), 256, 0, st>>>(y, bias, N, O, relu);
  CNN_CK(cudaGetLastError(), "bias/activation");
  return FWI_OK;
}

fwi_status fwi_cnn_conv_backward(fwi_cnn* h, const float* x, int32_t C, int32_t B, int32_t H, int32_t W,
                                 const uint16_t* w_bf16, int32_t O, int32_t sh, int32_t sw, int32_t relu,
                                 const float* y, float* dy, uint16_t* col, uint16_t* dy_bf16, float* dcol, float* dx,
                                 float* dw, float* db, void* stream) {
  if (!h || !x || !w_bf16 || !y || !dy || !col || !dy_bf16 || !dw || !db || (dx && !dcol))
    return fwi::host_fail(FWI_EINVAL, "NULL pointer");
  if (bad_dims(C, B, H, W) || O < 1 || sh < 1 || sw < 1) return fwi::host_fail(FWI_EINVAL, "bad sizes");
  CNN_CK(cudaSetDevice(h->device), "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)stream;
  const int Ho = fwi::conv_out(H, sh), Wo = fwi::conv_out(W, sw);
  const long long N = (long long)B * Ho * Wo, K = 9LL * C;
  if (N > 0x7fffffffLL) return fwi::host_fail(FWI_EINVAL, "layer too large for one GEMM");
  fwi::k_act_back<<<O, 256, 0, st>>>(dy, y, N, relu, dy_bf16, db);
  CNN_CK(cudaGetLastError(), "activation backward");
  fwi::k_im2col<<<blocks_for(K * N), 256, 0, st>>>(x, C, B, H, W, sh, sw, Ho, Wo, col);
  CNN_CK(cudaGetLastError(), "im2col");
  CNN_BLAS(cublasSetStream(h->blas, st), "cublasSetStream");
  // dw[O][K] = dy[O][N] . col^T  (col stored [K][N])
  fwi_status v = gemm_rm(h->blas, false, true, O, (int)K, (int)N, dy_bf16, col, dw, "conv weight-gradient GEMM");
  if (v != FWI_OK) return v;
  if (dx) {
    // dcol[K][N] = w^T . dy  (w stored [O][K])
    v = gemm_rm(h->blas, true, false, (int)K, (int)N, O, w_bf16, dy_bf16, dcol, "conv data-gradient GEMM");
    if (v != FWI_OK) return v;
    fwi::k_col2im<<<blocks_for((long long)C * B * H * W), 256, 0, st>>>(dcol, C, B, H, W, sh, sw, Ho, Wo, dx);
    CNN_CK(cudaGetLastError(), "col2im");
  }
  return FWI_OK;
}

fwi_status fwi_cnn_upsample2(const float* x, int32_t C, int32_t B, int32_t H, int32_t W, float* y, void* stream) {
  if (!x || !y) return fwi::host_fail(FWI_EINVAL, "NULL pointer");
  if (bad_dims(C, B, H, W)) return fwi::host_fail(FWI_EINVAL, "bad sizes");
  const long long CB = (long long)C * B;
  fwi::k_upsample2<<<blocks_for(CB * 4 * H * W), 256, 0, (cudaStream_t)stream>>>(x, CB, H, W, y);
  CNN_CK(cudaGetLastError(), "upsample");
  return FWI_OK;
}

fwi_status fwi_cnn_upsample2_backward(const float* dy, int32_t C, int32_t B, int32_t H, int32_t W, float* dx,
                                      void* stream) {
  if (!dy || !dx) return fwi::host_fail(FWI_EINVAL, "NULL pointer");
  if (bad_dims(C, B, H, W)) return fwi::host_fail(FWI_EINVAL, "bad sizes");
  const long long CB = (long long)C * B;
  fwi::k_upsample2_back<<<blocks_for(CB * H * W), 256, 0, (cudaStream_t)stream>>>(dy, CB, H, W, dx);
  CNN_CK(cudaGetLastError(), "upsample backward");
  return FWI_OK;
}

fwi_status fwi_cnn_mse(const float* p, const float* t, int64_t n, double* loss, float* dp, void* stream) {
  if (!p || !t || !loss || !dp) return fwi::host_fail(FWI_EINVAL, "NULL pointer");
  if (n < 1) return fwi::host_fail(FWI_EINVAL, "n must be >= 1");
  fwi::k_mse<<<1, 1024, 0, (cudaStream_t)stream>>>(p, t, n, loss, dp);
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
