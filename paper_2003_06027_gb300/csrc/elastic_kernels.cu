// elastic_kernels.cu - sm_103a kernels of the elastic velocity-stress path.
//
// Forward: one time step of the velocity-stress system (Implementation,
// Eq. elastic, isotropic Hooke law) on the staggered grid, as the explicit
// recursion of Eq. forward: v^{n+1/2} from sigma^n (ela_vel_step), then
// sigma^{n+1} from v^{n+1/2} with the moment-tensor source (ela_str_step).
// Adjoint: the exact transpose of each half step in reverse order
// (Eq. adjoint-backward), fused with the gradient correlations of
// Eq. adjoint-gradient for lambda, mu (through mu at the shear nodes) and the
// buoyancies (ela_str_adj, ela_vel_adj).
//
// Every update is a first-order staggered stencil (memory bound, no tensor
// cores). Persistent CTAs walk the 64 x 32 tiles of all shots; the fields a
// tile needs with a halo are fetched by TMA (cp.async.bulk.tensor, one box per
// field). The forward kernels use two shared-memory buffers, so the next
// tile's fetch overlaps the current tile's work; the adjoint kernels, whose
// halo-item scratch is larger, use one buffer, refilled once stage 1 has read
// it. Bounded mbarrier waits report a timeout. Per-node operands without a
// halo are loaded before the wait. At 4th order every kernel runs 3 CTAs of
// 256 threads per SM (80 registers). Each thread updates 2 rows x 4 columns. CPML memory variables are node-local in the
// forward (updated in place) and double-buffered in the adjoint, where their
// values are needed at halo nodes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "fwi_internal.cuh"
#include "tma.cuh"

namespace fwi {

namespace {

constexpr int W72 = TILE_X + 8;   // 72: columns [x0-4, x0+68)
constexpr int H40 = TILE_Z + 8;   // 40: rows [z0-4, z0+36)

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float4 ldg4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ void f4a(const float4 v, float o[4]) {
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ float4 a4f(const float o[4]) { return make_float4(o[0], o[1], o[2], o[3]); }
__device__ __forceinline__ void seg12(const float* s, float v[12]) {
  f4a(ld4(s), v);
  f4a(ld4(s + 4), v + 4);
  f4a(ld4(s + 8), v + 8);
}
__device__ __forceinline__ bool any4(float4 a) { return a.x != 0.f || a.y != 0.f || a.z != 0.f || a.w != 0.f; }

// Stage ROWS x COLS floats whose top-left padded cell is (zt, xt) (xt a
// multiple of 4) into shared memory.
template <int ROWS, int COLS>
__device__ __forceinline__ void stage(float* dst, const float* __restrict__ src, int pitch, int zt, int xt) {
  constexpr int C4 = COLS / 4;
  for (int idx = threadIdx.x; idx < ROWS * C4; idx += NTHREADS) {
    const int r = idx / C4, c4 = idx - r * C4;
    st4(dst + r * COLS + 4 * c4, ldg4(src + (long long)(zt + r) * pitch + xt + 4 * c4));
  }
}

// Staggered stencils on a 12-wide row segment v[t] (t = 0..11):
//   plus(e)  = sum_k c_k (v[e+4+k] - v[e+5-k])   (integer -> half, or half -> integer shifted)
//   minus(e) = sum_k c_k (v[e+3+k] - v[e+4-k])
template <int N>
__device__ __forceinline__ float plus12(const float* c, const float v[12], int e) {
  float s = 0.f;
#pragma unroll
  for (int k = 1; k <= N; k++) s += c[k - 1] * (v[e + 4 + k] - v[e + 5 - k]);
  return s;
}
template <int N>
__device__ __forceinline__ float minus12(const float* c, const float v[12], int e) {
  float s = 0.f;
#pragma unroll
  for (int k = 1; k <= N; k++) s += c[k - 1] * (v[e + 3 + k] - v[e + 4 - k]);
  return s;
}
// The same along z on a (2N+1)-row window W[t] covering two output rows:
// out0 = sum c (W[k+N-1] - W[N-k]),  out1 = sum c (W[k+N] - W[N-k+1]).
template <int N>
__device__ __forceinline__ void zwin(const float* c, const float4* W, float o0[4], float o1[4]) {
  float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
#pragma unroll
  for (int k = 1; k <= N; k++) {
    const float ck = c[k - 1];
    const float4 p0 = W[k + N - 1], m0 = W[N - k], p1 = W[k + N], m1 = W[N - k + 1];
    a.x += ck * (p0.x - m0.x); a.y += ck * (p0.y - m0.y); a.z += ck * (p0.z - m0.z); a.w += ck * (p0.w - m0.w);
    b.x += ck * (p1.x - m1.x); b.y += ck * (p1.y - m1.y); b.z += ck * (p1.z - m1.z); b.w += ck * (p1.w - m1.w);
  }
  f4a(a, o0);
  f4a(b, o1);
}
template <int N, int W>
__device__ __forceinline__ void load_win(const float* base, int row0, int col, float4* Wv) {
#pragma unroll
  for (int t = 0; t <= 2 * N; t++) Wv[t] = ld4(base + (row0 + t) * W + col);
}

__device__ __forceinline__ bool pml_x(const Grid& g, int x0) {
  return g.npml > 0 && (x0 - 8 < g.npml || x0 + TILE_X + 8 > g.npml + g.nx - 1);
}
__device__ __forceinline__ bool pml_z(const Grid& g, int z0) {
  return g.npml > 0 && (z0 - 8 < g.npml || z0 + TILE_Z + 8 > g.npml + g.nz - 1);
}

// Node-local CPML update of 4 consecutive x nodes with x-dependent tables:
// psi <- b psi + a d (zero where a = 0), returns d + psi.
__device__ __forceinline__ void cpml_x4(bool on, const float* ta, const float* tb, int j, float* psi, long long id,
                                        float d[4]) {
  if (!on) return;
  const float4 a4 = ldg4(ta + j + TAB_OFF);
  if (!any4(a4)) return;
  const float4 b4 = ldg4(tb + j + TAB_OFF);
  const float4 P = ld4(psi + id);
  float4 Pn;
  Pn.x = b4.x * P.x + a4.x * d[0]; Pn.y = b4.y * P.y + a4.y * d[1];
  Pn.z = b4.z * P.z + a4.z * d[2]; Pn.w = b4.w * P.w + a4.w * d[3];
  st4(psi + id, Pn);
  d[0] += Pn.x; d[1] += Pn.y; d[2] += Pn.z; d[3] += Pn.w;
}
// The same with a row-uniform (z) table entry.
__device__ __forceinline__ void cpml_z4(bool on, const float* ta, const float* tb, int z, float* psi, long long id,
                                        float d[4]) {
  if (!on) return;
  const float a = __ldg(ta + z + TAB_OFF);
  if (a == 0.f) return;
  const float b = __ldg(tb + z + TAB_OFF);
  const float4 P = ld4(psi + id);
  float4 Pn;
  Pn.x = b * P.x + a * d[0]; Pn.y = b * P.y + a * d[1]; Pn.z = b * P.z + a * d[2]; Pn.w = b * P.w + a * d[3];
  st4(psi + id, Pn);
  d[0] += Pn.x; d[1] += Pn.y; d[2] += Pn.z; d[3] += Pn.w;
}

// Adjoint of a CPML term for 4 nodes given the incoming adjoint t of (d + psi):
// returns dbar = t + a (M + t) and, for owners, writes M' = b (M + t) (zero where a = 0).
__device__ __forceinline__ void cpml_adj_x4(bool on, const float* ta, const float* tb, int j, const float* Min,
                                            float* Mout, long long id, bool own, const float t[4], float d[4]) {
  d[0] = t[0]; d[1] = t[1]; d[2] = t[2]; d[3] = t[3];
  if (!on) return;
  const float4 a4 = ldg4(ta + j + TAB_OFF);
  if (!any4(a4)) return;
  const float4 b4 = ldg4(tb + j + TAB_OFF);
  float M[4], a[4], b[4];
  f4a(ldg4(Min + id), M);  // read-only in this kernel (the pair's other half is written)
  f4a(a4, a);
  f4a(b4, b);
  float Mn[4];
#pragma unroll
  for (int e = 0; e < 4; e++) {
    const float u = M[e] + t[e];
    d[e] = t[e] + a[e] * u;
    Mn[e] = a[e] != 0.f ? b[e] * u : 0.f;
  }
  if (own) st4(Mout + id, a4f(Mn));
}
__device__ __forceinline__ void cpml_adj_z4(bool on, const float* ta, const float* tb, int z, const float* Min,
                                            float* Mout, long long id, bool own, const float t[4], float d[4]) {
  d[0] = t[0]; d[1] = t[1]; d[2] = t[2]; d[3] = t[3];
  if (!on) return;
  const float a = __ldg(ta + z + TAB_OFF);
  if (a == 0.f) return;
  const float b = __ldg(tb + z + TAB_OFF);
  float M[4], Mn[4];
  f4a(ldg4(Min + id), M);  // read-only in this kernel (the pair's other half is written)
#pragma unroll
  for (int e = 0; e < 4; e++) {
    const float u = M[e] + t[e];
    d[e] = t[e] + a * u;
    Mn[e] = b * u;
  }
  if (own) st4(Mout + id, a4f(Mn));
}

// Deterministic CTA sum of three floats (fixed shuffle tree, fixed warp order).
__device__ __forceinline__ void cta_sum3(float v[3], float* red) {
  for (int k = 0; k < 3; k++)
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0)
    for (int k = 0; k < 3; k++) red[warp * 3 + k] = v[k];
  __syncthreads();
  if (threadIdx.x == 0)
    for (int k = 0; k < 3; k++) {
      float s = 0.f;
      for (int w = 0; w < NTHREADS / 32; w++) s += red[w * 3 + k];
      v[k] = s;
    }
  __syncthreads();
}

}  // namespace

// ---------------------------------------------------------------------------
// Persistent-walk skeleton shared by the four kernels: buffer b of iteration it
// holds tile t; the fetch of the next tile is issued before this one is used.
#define ELA_WALK_BEGIN(FETCH)                                                      \
  const int ntiles = p.S * g.ntx * g.ntz;                                        \
  if (tid == 0) {                                                                \
    mbar_init(&bar[0], 1);                                                       \
    mbar_init(&bar[1], 1);                                                       \
    fence_mbar_init();                                                           \
  }                                                                              \
  __syncthreads();                                                               \
  if (tid == 0 && (int)blockIdx.x < ntiles) FETCH(blockIdx.x, 0);                \
  int it = 0;                                                                    \
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x, it++) {                   \
    const int b = it & 1;                                                        \
    if (tid == 0 && t + (int)gridDim.x < ntiles) FETCH(t + (int)gridDim.x, b ^ 1); \
    const TileId id = tile_decode(g, t);                                         \
    const int s = id.s, x0 = id.x0, z0 = id.z0;                                  \
    const long long base = (long long)s * g.slice + g.off0;

#define ELA_WAIT()                                          \
  {                                                         \
    const bool ok_ = mbar_wait(&bar[b], (it >> 1) & 1);     \
    if (__syncthreads_or(!ok_)) {                           \
      if (tid == 0) {                                       \
        atomicOr(p.status, ST_TIMEOUT);                     \
        tma_drain(bar, it, t + (int)gridDim.x < ntiles);    \
      }                                                     \
      return;                                               \
    }                                                       \
  }

#define ELA_WALK_END() \
  __syncthreads();     \
  }

// Single-buffer walk (the adjoint kernels): one operand buffer and one barrier;
// the fetch of the next tile is issued by ELA_PREFETCH1 once every thread has
// read what it needs of the buffer, so the copy overlaps the rest of the tile
// and the other CTAs on the SM cover its latency. On a timeout the CTA lets a
// late copy land (bounded wait) before it returns.
#define ELA_WALK1_BEGIN(FETCH)                                      \
  const int ntiles = p.S * g.ntx * g.ntz;                           \
  if (tid == 0) {                                                   \
    mbar_init(&bar[0], 1);                                          \
    fence_mbar_init();                                              \
  }                                                                 \
  __syncthreads();                                                  \
  if (tid == 0 && (int)blockIdx.x < ntiles) FETCH(blockIdx.x);      \
  int it = 0;                                                       \
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x, it++) {      \
    const TileId id = tile_decode(g, t);                            \
    const int s = id.s, x0 = id.x0, z0 = id.z0;                     \
    const long long base = (long long)s * g.slice + g.off0;

#define ELA_WAIT1()                                      \
  {                                                      \
    const bool ok_ = mbar_wait(&bar[0], it & 1);         \
    if (__syncthreads_or(!ok_)) {                        \
      if (tid == 0) {                                    \
        atomicOr(p.status, ST_TIMEOUT);                  \
        mbar_wait(&bar[0], it & 1);                      \
      }                                                  \
      return;                                            \
    }                                                    \
  }

#define ELA_PREFETCH1(FETCH) \
  if (tid == 0 && t + (int)gridDim.x < ntiles) FETCH(t + (int)gridDim.x);

// Velocity half step: v^{n+1/2} = v^{n-1/2} + dt b (div sigma^n + CPML).
// Tile buffer: sxx rows [z0, z0+32) cols [x0-4, x0+68); szz rows [z0-4, z0+36)
// cols [x0, x0+64); sxz rows [z0-4, z0+36) cols [x0-4, x0+68).
constexpr int VEL_BUF = TILE_Z * W72 + H40 * TILE_X + H40 * W72;
template <int N, bool RECORD, bool STORE>
__global__ void __launch_bounds__(NTHREADS, N == 2 ? 3 : 2)  // 3 CTAs per SM at 4th order (80 registers)
    ela_vel_step(const __grid_constant__ CUtensorMap m_xx, const __grid_constant__ CUtensorMap m_zz,
                 const __grid_constant__ CUtensorMap m_xz, const EleStep p) {
  extern __shared__ __align__(128) float smem_e[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_e + 2 * VEL_BUF);
  const Grid& g = p.g;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int pitch = g.pitch;
  auto fetch = [&](int tt, int bb) {
    const TileId f = tile_decode(g, tt);
    float* d = smem_e + bb * VEL_BUF;
    fence_proxy_async();
    mbar_expect_tx(&bar[bb], VEL_BUF * 4);
    tma_3d(d, &m_xx, f.x0 - 4 + APRON, f.z0 + APRON, f.s, &bar[bb]);
    tma_3d(d + TILE_Z * W72, &m_zz, f.x0 + APRON, f.z0 - 4 + APRON, f.s, &bar[bb]);
    tma_3d(d + TILE_Z * W72 + H40 * TILE_X, &m_xz, f.x0 - 4 + APRON, f.z0 - 4 + APRON, f.s, &bar[bb]);
  };
  ELA_WALK_BEGIN(fetch)
  const int xb = x0 + 4 * tx, zr0 = z0 + 2 * ty;
  // per-node operands of this thread's 2 x 4 nodes
  float4 vo[2], wo[2], bxv[2], bzv[2];
#pragma unroll
  for (int rr = 0; rr < 2; rr++) {
    const long long id = base + (long long)(zr0 + rr) * pitch + xb;
    const long long im = g.off0 + (long long)(zr0 + rr) * pitch + xb;
    vo[rr] = ld4(p.vx + id);
    wo[rr] = ld4(p.vz + id);
    bxv[rr] = ldg4(p.bx + im);
    bzv[rr] = ldg4(p.bz + im);
  }
  int rb = 0, re = 0;
  if (RECORD) {
    const int key = (id.tz * g.ntx + id.tx) * NTHREADS + tid;
    rb = __ldg(p.thr_rec_start + key);
    re = __ldg(p.thr_rec_start + key + 1);
  }
  ELA_WAIT()
  const float* s_xx = smem_e + b * VEL_BUF;
  const float* s_zz = s_xx + TILE_Z * W72;
  const float* s_xz = s_zz + H40 * TILE_X;
  const bool px = pml_x(g, x0), pz = pml_z(g, z0);
  float d2[2][4], d4[2][4];
  {
    float4 W[2 * N + 1];
    load_win<N, W72>(s_xz, 2 * ty + 4 - N, 4 * tx + 4, W);  // sxz half rows around vx rows
    zwin<N>(p.cz, W, d2[0], d2[1]);
    load_win<N, TILE_X>(s_zz, 2 * ty + 5 - N, 4 * tx, W);  // szz rows around vz half rows
    zwin<N>(p.cz, W, d4[0], d4[1]);
  }
  float vxn[2][4], vzn[2][4];
#pragma unroll
  for (int rr = 0; rr < 2; rr++) {
    const int r = 2 * ty + rr, z = z0 + r;
    const long long id = base + (long long)z * pitch + xb;
    float v[12], d1[4], d3[4];
    seg12(s_xx + r * W72 + 4 * tx, v);
#pragma unroll
    for (int e = 0; e < 4; e++) d1[e] = plus12<N>(p.cx, v, e);
    seg12(s_xz + (r + 4) * W72 + 4 * tx, v);
#pragma unroll
    for (int e = 0; e < 4; e++) d3[e] = minus12<N>(p.cx, v, e);
    cpml_x4(px, p.axh, p.bxh, xb, p.psi[0], id, d1);
    cpml_z4(pz, p.az, p.bzt, z, p.psi[1], id, d2[rr]);
    cpml_x4(px, p.ax, p.bxt, xb, p.psi[2], id, d3);
    cpml_z4(pz, p.azh, p.bzh, z, p.psi[3], id, d4[rr]);
    float fx[4], fz[4], bxa[4], bza[4], voa[4], woa[4];
    f4a(bxv[rr], bxa);
    f4a(bzv[rr], bza);
    f4a(vo[rr], voa);
    f4a(wo[rr], woa);
#pragma unroll
    for (int e = 0; e < 4; e++) {
      fx[e] = d1[e] + d2[rr][e];
      fz[e] = d3[e] + d4[rr][e];
      vxn[rr][e] = voa[e] + p.dt * bxa[e] * fx[e];  // buoyancy is zero outside the vx nodes
      vzn[rr][e] = woa[e] + p.dt * bza[e] * fz[e];
    }
    st4(p.vx + id, a4f(vxn[rr]));
    st4(p.vz + id, a4f(vzn[rr]));
    if (STORE) {
      st4_stream(p.slot[0] + id, a4f(fx), l2_evict_first());
      st4_stream(p.slot[1] + id, a4f(fz), l2_evict_first());
    }
  }
  if (RECORD) {
    for (int q = rb; q < re; q++) {
      const int code = p.thr_rec[q];
      const int rc = code >> 3, rr = (code >> 2) & 1, e = code & 3;
      float va = 0.f, vb = 0.f;
#pragma unroll
      for (int r2 = 0; r2 < 2; r2++)
#pragma unroll
        for (int e2 = 0; e2 < 4; e2++)
          if (r2 == rr && e2 == e) {
            va = vxn[r2][e2];
            vb = vzn[r2][e2];
          }
      const long long o = ((long long)s * 2 * p.nrec + rc) * p.nt + p.n;
      p.seis[o] = va;
      p.seis[o + (long long)p.nrec * p.nt] = vb;
    }
  }
  ELA_WALK_END()
}

// ---------------------------------------------------------------------------
// Stress half step: sigma^{n+1} = sigma^n + dt C (grad v^{n+1/2} + CPML) - dt M g_n w.
// Tile buffer: vx and vz, rows [z0-4, z0+36), cols [x0-4, x0+68).
constexpr int STR_BUF = 2 * H40 * W72;
template <int N, bool STORE>
__global__ void __launch_bounds__(NTHREADS, N == 2 ? 3 : 2)  // 3 CTAs per SM at 4th order (80 registers)
    ela_str_step(const __grid_constant__ CUtensorMap m_vx, const __grid_constant__ CUtensorMap m_vz, const EleStep p) {
  extern __shared__ __align__(128) float smem_e[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_e + 2 * STR_BUF);
  const Grid& g = p.g;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int pitch = g.pitch;
  auto fetch = [&](int tt, int bb) {
    const TileId f = tile_decode(g, tt);
    float* d = smem_e + bb * STR_BUF;
    fence_proxy_async();
    mbar_expect_tx(&bar[bb], STR_BUF * 4);
    tma_3d(d, &m_vx, f.x0 - 4 + APRON, f.z0 - 4 + APRON, f.s, &bar[bb]);
    tma_3d(d + H40 * W72, &m_vz, f.x0 - 4 + APRON, f.z0 - 4 + APRON, f.s, &bar[bb]);
  };
  ELA_WALK_BEGIN(fetch)
  const int xb = x0 + 4 * tx, zr0 = z0 + 2 * ty;
  float4 so[2][3];
#pragma unroll
  for (int rr = 0; rr < 2; rr++) {
    const long long id = base + (long long)(zr0 + rr) * pitch + xb;
    so[rr][0] = ld4(p.sxx + id);
    so[rr][1] = ld4(p.szz + id);
    so[rr][2] = ld4(p.sxz + id);
  }
  const int2 bn = __ldg(reinterpret_cast<const int2*>(p.box_n) + s);
  const int2 bs = __ldg(reinterpret_cast<const int2*>(p.box_s) + s);
  const float g_n = __ldg(p.stf + (long long)s * p.nt + p.n);
  ELA_WAIT()
  const float* s_vx = smem_e + b * STR_BUF;
  const float* s_vz = s_vx + H40 * W72;
  const bool px = pml_x(g, x0), pz = pml_z(g, z0);
  float d6[2][4], d7[2][4];
  {
    float4 W[2 * N + 1];
    load_win<N, W72>(s_vz, 2 * ty + 4 - N, 4 * tx + 4, W);  // vz half rows around normal rows
    zwin<N>(p.cz, W, d6[0], d6[1]);
    load_win<N, W72>(s_vx, 2 * ty + 5 - N, 4 * tx + 4, W);  // vx rows around shear half rows
    zwin<N>(p.cz, W, d7[0], d7[1]);
  }
  const int nb = p.src_n;
  const float Mxx = p.mt[3 * s], Mzz = p.mt[3 * s + 1], Mxz = p.mt[3 * s + 2];
#pragma unroll
  for (int rr = 0; rr < 2; rr++) {
    const int r = 2 * ty + rr, z = z0 + r;
    const long long id = base + (long long)z * pitch + xb;
    const long long im = g.off0 + (long long)z * pitch + xb;
    float v[12], d5[4], d8[4];
    seg12(s_vx + (r + 4) * W72 + 4 * tx, v);
#pragma unroll
    for (int e = 0; e < 4; e++) d5[e] = minus12<N>(p.cx, v, e);
    seg12(s_vz + (r + 4) * W72 + 4 * tx, v);
#pragma unroll
    for (int e = 0; e < 4; e++) d8[e] = plus12<N>(p.cx, v, e);
    cpml_x4(px, p.ax, p.bxt, xb, p.psi[4], id, d5);
    cpml_z4(pz, p.az, p.bzt, z, p.psi[5], id, d6[rr]);
    cpml_z4(pz, p.azh, p.bzh, z, p.psi[6], id, d7[rr]);
    cpml_x4(px, p.axh, p.bxh, xb, p.psi[7], id, d8);
    float la[4], lp[4], mx[4], sx[4], sz[4], sh[4], exz[4];
    f4a(ldg4(p.lam + im), la);
    f4a(ldg4(p.lp2m + im), lp);
    f4a(ldg4(p.mxz + im), mx);
    f4a(so[rr][0], sx);
    f4a(so[rr][1], sz);
    f4a(so[rr][2], sh);
#pragma unroll
    for (int e = 0; e < 4; e++) {
      exz[e] = d7[rr][e] + d8[e];
      sx[e] += p.dt * (lp[e] * d5[e] + la[e] * d6[rr][e]);
      sz[e] += p.dt * (la[e] * d5[e] + lp[e] * d6[rr][e]);
      sh[e] += p.dt * mx[e] * exz[e];
    }
    // moment-tensor source on the normal and the shear grid
    if (bn.x >= 0) {
      const int di = z - bn.x;
      if (di >= 0 && di < nb)
#pragma unroll
        for (int e = 0; e < 4; e++) {
          const int dj = xb + e - bn.y;
          if (dj >= 0 && dj < nb) {
            const float w = p.dt * g_n * p.w_n[s * SRC_W * SRC_W + di * SRC_W + dj];
            sx[e] -= w * Mxx;
            sz[e] -= w * Mzz;
          }
        }
      const int ds = z - bs.x;
      if (ds >= 0 && ds < nb)
#pragma unroll
        for (int e = 0; e < 4; e++) {
          const int dj = xb + e - bs.y;
          if (dj >= 0 && dj < nb) sh[e] -= p.dt * g_n * p.w_s[s * SRC_W * SRC_W + ds * SRC_W + dj] * Mxz;
        }
    }
    st4(p.sxx + id, a4f(sx));
    st4(p.szz + id, a4f(sz));
    st4(p.sxz + id, a4f(sh));
    if (STORE) {
      st4_stream(p.slot[2] + id, a4f(d5), l2_evict_first());
      st4_stream(p.slot[3] + id, a4f(d6[rr]), l2_evict_first());
      st4_stream(p.slot[4] + id, a4f(exz), l2_evict_first());
    }
  }
  ELA_WALK_END()
}

// ---------------------------------------------------------------------------
// Adjoint of the stress half step of step n. Sbar (= adjoint of sigma^{n+1})
// flows through unchanged; this kernel adds its image to Vbar (the adjoint of
// v^{n+1/2}), adds the residual of sample n, updates the memory adjoints
// M5..M8 and accumulates the lambda, mu and mu_xz correlations and the
// source-parameter partials of step n.
constexpr int ADJA_BUF = 3 * H40 * W72;  // Sbar xx, zz, xz: rows [z0-4, z0+36), cols [x0-4, x0+68)
constexpr int ADJA_SCR = 2 * TILE_Z * W72 + 2 * H40 * TILE_X + 32;
template <int N>
__global__ void __launch_bounds__(NTHREADS, N == 2 ? 3 : 2)  // 3 CTAs per SM at 4th order (80 registers)
    ela_str_adj(const __grid_constant__ CUtensorMap m_Sxx, const __grid_constant__ CUtensorMap m_Szz,
                const __grid_constant__ CUtensorMap m_Sxz, const EleStep p) {
  extern __shared__ __align__(128) float smem_e[];
  float* d_vx = smem_e + ADJA_BUF;            // [TILE_Z][W72] normal nodes, own rows
  float* d_vz = d_vx + TILE_Z * W72;          // [H40][TILE_X] normal nodes, own cols
  float* d_vxz = d_vz + H40 * TILE_X;         // [H40][TILE_X] shear nodes, own cols
  float* d_vzx = d_vxz + H40 * TILE_X;        // [TILE_Z][W72] shear nodes, own rows
  float* red = d_vzx + TILE_Z * W72;          // [32]
  uint64_t* bar = reinterpret_cast<uint64_t*>(red + 32);
  const Grid& g = p.g;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int pitch = g.pitch;
  auto fetch = [&](int tt) {
    const TileId f = tile_decode(g, tt);
    fence_proxy_async();
    mbar_expect_tx(&bar[0], ADJA_BUF * 4);
    tma_3d(smem_e, &m_Sxx, f.x0 - 4 + APRON, f.z0 - 4 + APRON, f.s, &bar[0]);
    tma_3d(smem_e + H40 * W72, &m_Szz, f.x0 - 4 + APRON, f.z0 - 4 + APRON, f.s, &bar[0]);
    tma_3d(smem_e + 2 * H40 * W72, &m_Sxz, f.x0 - 4 + APRON, f.z0 - 4 + APRON, f.s, &bar[0]);
  };
  ELA_WALK1_BEGIN(fetch)
  const int xb = x0 + 4 * tx, zr0 = z0 + 2 * ty;
  float4 vpre[2][2];
#pragma unroll
  for (int rr = 0; rr < 2; rr++) {
    const long long id = base + (long long)(zr0 + rr) * pitch + xb;
    vpre[rr][0] = ld4(p.Vx + id);
    vpre[rr][1] = ld4(p.Vz + id);
  }
  const int key = (id.tz * g.ntx + id.tx) * NTHREADS + tid;
  const int rb = __ldg(p.thr_rec_start + key), re = __ldg(p.thr_rec_start + key + 1);
  ELA_WAIT1()
  const float* s_Sxx = smem_e;
  const float* s_Szz = s_Sxx + H40 * W72;
  const float* s_Sxz = s_Szz + H40 * W72;
  const bool px = pml_x(g, x0), pz = pml_z(g, z0);
  const float dt = p.dt;
  // the halo items of each kind (the own nodes' are merged below)
  auto item_a = [&](int k) {  // (a) strain-x adjoint at normal nodes, own rows, columns [x0-4, x0+68)
    const int r = k / (W72 / 4), gq = k - r * (W72 / 4);
    const int z = z0 + r, j = x0 - 4 + 4 * gq;
    const long long id = base + (long long)z * pitch + j, im = g.off0 + (long long)z * pitch + j;
    float sx[4], sz[4], la[4], lp[4], t[4], d[4];
    f4a(ld4(s_Sxx + (r + 4) * W72 + 4 * gq), sx);
    f4a(ld4(s_Szz + (r + 4) * W72 + 4 * gq), sz);
    f4a(ldg4(p.lam + im), la);
    f4a(ldg4(p.lp2m + im), lp);
#pragma unroll
    for (int e = 0; e < 4; e++) t[e] = dt * (lp[e] * sx[e] + la[e] * sz[e]);
    cpml_adj_x4(px, p.ax, p.bxt, j, p.Min[4], p.Mout[4], id, gq >= 1 && gq <= 16, t, d);
    st4(d_vx + r * W72 + 4 * gq, a4f(d));
  };
  auto item_b = [&](int k) {  // (b) strain-z adjoint at normal nodes, rows [z0-4, z0+36), own cols
    const int hr = k / (TILE_X / 4), c = k - hr * (TILE_X / 4);
    const int z = z0 - 4 + hr, j = x0 + 4 * c;
    const long long id = base + (long long)z * pitch + j, im = g.off0 + (long long)z * pitch + j;
    float sx[4], sz[4], la[4], lp[4], t[4], d[4];
    f4a(ld4(s_Sxx + hr * W72 + 4 * c + 4), sx);
    f4a(ld4(s_Szz + hr * W72 + 4 * c + 4), sz);
    f4a(ldg4(p.lam + im), la);
    f4a(ldg4(p.lp2m + im), lp);
#pragma unroll
    for (int e = 0; e < 4; e++) t[e] = dt * (la[e] * sx[e] + lp[e] * sz[e]);
    cpml_adj_z4(pz, p.az, p.bzt, z, p.Min[5], p.Mout[5], id, hr >= 4 && hr < 4 + TILE_Z, t, d);
    st4(d_vz + hr * TILE_X + 4 * c, a4f(d));
  };
  auto item_c = [&](int k) {  // (c) shear strain adjoint (z part) at shear nodes, all rows, own cols
    const int hr = k / (TILE_X / 4), c = k - hr * (TILE_X / 4);
    const int z = z0 - 4 + hr, j = x0 + 4 * c;
    const long long id = base + (long long)z * pitch + j, im = g.off0 + (long long)z * pitch + j;
    float sh[4], mx[4], t[4], d[4];
    f4a(ld4(s_Sxz + hr * W72 + 4 * c + 4), sh);
    f4a(ldg4(p.mxz + im), mx);
#pragma unroll
    for (int e = 0; e < 4; e++) t[e] = dt * mx[e] * sh[e];
    cpml_adj_z4(pz, p.azh, p.bzh, z, p.Min[6], p.Mout[6], id, hr >= 4 && hr < 4 + TILE_Z, t, d);
    st4(d_vxz + hr * TILE_X + 4 * c, a4f(d));
  };
  auto item_d = [&](int k) {  // (d) shear strain adjoint (x part) at shear nodes, own rows, columns [x0-4, x0+68)
    const int r = k / (W72 / 4), gq = k - r * (W72 / 4);
    const int z = z0 + r, j = x0 - 4 + 4 * gq;
    const long long id = base + (long long)z * pitch + j, im = g.off0 + (long long)z * pitch + j;
    float sh[4], mx[4], t[4], d[4];
    f4a(ld4(s_Sxz + (r + 4) * W72 + 4 * gq), sh);
    f4a(ldg4(p.mxz + im), mx);
#pragma unroll
    for (int e = 0; e < 4; e++) t[e] = dt * mx[e] * sh[e];
    cpml_adj_x4(px, p.axh, p.bxh, j, p.Min[7], p.Mout[7], id, gq >= 1 && gq <= 16, t, d);
    st4(d_vzx + r * W72 + 4 * gq, a4f(d));
  };
  // own nodes: items (a) and (b) of a normal-node group, and (c) and (d) of a
  // shear-node group, in one pass each, so that its medium is loaded once
  auto item_ab = [&](int k) {
    const int r = k >> 4, c = k & 15;
    const int z = z0 + r, j = x0 + 4 * c;
    const long long id = base + (long long)z * pitch + j, im = g.off0 + (long long)z * pitch + j;
    float sx[4], sz[4], la[4], lp[4], ta[4], tb[4], d[4];
    f4a(ld4(s_Sxx + (r + 4) * W72 + 4 * c + 4), sx);
    f4a(ld4(s_Szz + (r + 4) * W72 + 4 * c + 4), sz);
    f4a(ldg4(p.lam + im), la);
    f4a(ldg4(p.lp2m + im), lp);
#pragma unroll
    for (int e = 0; e < 4; e++) {
      ta[e] = dt * (lp[e] * sx[e] + la[e] * sz[e]);
      tb[e] = dt * (la[e] * sx[e] + lp[e] * sz[e]);
    }
    cpml_adj_x4(px, p.ax, p.bxt, j, p.Min[4], p.Mout[4], id, true, ta, d);
    st4(d_vx + r * W72 + 4 * (c + 1), a4f(d));
    cpml_adj_z4(pz, p.az, p.bzt, z, p.Min[5], p.Mout[5], id, true, tb, d);
    st4(d_vz + (r + 4) * TILE_X + 4 * c, a4f(d));
  };
  auto item_cd = [&](int k) {
    const int r = k >> 4, c = k & 15;
    const int z = z0 + r, j = x0 + 4 * c;
    const long long id = base + (long long)z * pitch + j, im = g.off0 + (long long)z * pitch + j;
    float sh[4], mx[4], t[4], d[4];
    f4a(ld4(s_Sxz + (r + 4) * W72 + 4 * c + 4), sh);
    f4a(ldg4(p.mxz + im), mx);
#pragma unroll
    for (int e = 0; e < 4; e++) t[e] = dt * mx[e] * sh[e];
    cpml_adj_z4(pz, p.azh, p.bzh, z, p.Min[6], p.Mout[6], id, true, t, d);
    st4(d_vxz + (r + 4) * TILE_X + 4 * c, a4f(d));
    cpml_adj_x4(px, p.axh, p.bxh, j, p.Min[7], p.Mout[7], id, true, t, d);
    st4(d_vzx + r * W72 + 4 * (c + 1), a4f(d));
  };
  constexpr int NOWN = TILE_Z * (TILE_X / 4);  // own 4-node groups: 512
#pragma unroll 2
  for (int k = tid; k < NOWN; k += NTHREADS) item_ab(k);
#pragma unroll 2
  for (int k = tid; k < NOWN; k += NTHREADS) item_cd(k);
  // halo nodes: the two halo column groups of every own row (items a, d) and
  // the 8 halo rows of the own columns (items b, c)
  if (tid < 2 * TILE_Z) {
    const int k = (tid >> 1) * (W72 / 4) + ((tid & 1) ? W72 / 4 - 1 : 0);
    item_a(k);
    item_d(k);
  } else if (tid < 2 * TILE_Z + 8 * (TILE_X / 4)) {
    const int h = (tid - 2 * TILE_Z) >> 4, c = tid & 15, hr = h < 4 ? h : h + TILE_Z;
    item_b(hr * (TILE_X / 4) + c);
    item_c(hr * (TILE_X / 4) + c);
  }
  // the own nodes' adjoint stresses, read before the buffer is refilled
  float Sx_own[2][4], Sz_own[2][4], Sh_own[2][4];
#pragma unroll
  for (int rr = 0; rr < 2; rr++) {
    const int o = (2 * ty + rr + 4) * W72 + 4 * tx + 4;
    f4a(ld4(s_Sxx + o), Sx_own[rr]);
    f4a(ld4(s_Szz + o), Sz_own[rr]);
    f4a(ld4(s_Sxz + o), Sh_own[rr]);
  }
  __syncthreads();
  ELA_PREFETCH1(fetch)
  float zx[2][4], zz[2][4];
  {
    float4 W[2 * N + 1];
    load_win<N, TILE_X>(d_vxz, 2 * ty + 4 - N, 4 * tx, W);  // D+z^T at vx rows
    zwin<N>(p.cz, W, zx[0], zx[1]);
    load_win<N, TILE_X>(d_vz, 2 * ty + 5 - N, 4 * tx, W);   // D-z^T at vz half rows
    zwin<N>(p.cz, W, zz[0], zz[1]);
  }
#pragma unroll
  for (int rr = 0; rr < 2; rr++) {
    const int r = 2 * ty + rr, z = z0 + r;
    const long long id = base + (long long)z * pitch + xb;
    float v[12], vxb[4], vzb[4];
    f4a(vpre[rr][0], vxb);
    f4a(vpre[rr][1], vzb);
    seg12(d_vx + r * W72 + 4 * tx, v);
#pragma unroll
    for (int e = 0; e < 4; e++) vxb[e] -= plus12<N>(p.cx, v, e) + zx[rr][e];
    seg12(d_vzx + r * W72 + 4 * tx, v);
#pragma unroll
    for (int e = 0; e < 4; e++) vzb[e] -= zz[rr][e] + minus12<N>(p.cx, v, e);
#pragma unroll
    for (int e = 0; e < 4; e++) {
      if (!(z < g.Nz && xb + e < g.Nx - 1)) vxb[e] = 0.f;
      if (!(z < g.Nz - 1 && xb + e < g.Nx)) vzb[e] = 0.f;
    }
    // residual of sample n at this thread's receivers
    for (int q = rb; q < re; q++) {
      const int code = p.thr_rec[q];
      if (((code >> 2) & 1) != rr) continue;
      const int rc = code >> 3, e = code & 3;
      const long long o = ((long long)s * 2 * p.nrec + rc) * p.nt + p.n;
      const float ax_ = p.res[o], az_ = p.res[o + (long long)p.nrec * p.nt];
#pragma unroll
      for (int e2 = 0; e2 < 4; e2++)
        if (e2 == e) {
          if (z < g.Nz && xb + e2 < g.Nx - 1) vxb[e2] += ax_;
          if (z < g.Nz - 1 && xb + e2 < g.Nx) vzb[e2] += az_;
        }
    }
    st4(p.Vx + id, a4f(vxb));
    st4(p.Vz + id, a4f(vzb));
    // gradient correlations of step n
    float ex[4], ez[4], exz[4], gl[4], gm[4], gx[4];
    f4a(ld4_stream(p.slot[2] + id, l2_evict_first()), ex);
    f4a(ld4_stream(p.slot[3] + id, l2_evict_first()), ez);
    f4a(ld4_stream(p.slot[4] + id, l2_evict_first()), exz);
    f4a(ld4(p.g_lam + id), gl);
    f4a(ld4(p.g_mu + id), gm);
    f4a(ld4(p.g_mxz + id), gx);
#pragma unroll
    for (int e = 0; e < 4; e++) {
      const bool nv = z < g.Nz && xb + e < g.Nx, sv = z < g.Nz - 1 && xb + e < g.Nx - 1;
      if (nv) {
        gl[e] += dt * (ex[e] + ez[e]) * (Sx_own[rr][e] + Sz_own[rr][e]);
        gm[e] += 2.f * dt * (ex[e] * Sx_own[rr][e] + ez[e] * Sz_own[rr][e]);
      }
      if (sv) gx[e] += dt * exz[e] * Sh_own[rr][e];
    }
    st4(p.g_lam + id, a4f(gl));
    st4(p.g_mu + id, a4f(gm));
    st4(p.g_mxz + id, a4f(gx));
  }
  // source-parameter partials of step n from sigma-bar^{n+1}:
  // sum w (M : sigma-bar), times (x_i - x0), (z_i - z0); normal box slots 0..3, shear box 4..7
  if (p.src_part != nullptr) {
    const int nb = p.src_n;
    const float xs = p.x0[2 * s], zs = p.x0[2 * s + 1];
    const float Mxx = p.mt[3 * s], Mzz = p.mt[3 * s + 1], Mxz = p.mt[3 * s + 2];
    for (int which = 0; which < 2; which++) {
      const int2 bx2 = __ldg(reinterpret_cast<const int2*>(which ? p.box_s : p.box_n) + s);
      if (!(bx2.x >= 0 && bx2.x < z0 + TILE_Z && bx2.x + nb > z0 && bx2.y < x0 + TILE_X && bx2.y + nb > x0)) continue;
      const float off = which ? 0.5f : 0.f;
      const float* w = (which ? p.w_s : p.w_n) + s * SRC_W * SRC_W;
      float acc[3] = {0.f, 0.f, 0.f};
#pragma unroll
      for (int rr = 0; rr < 2; rr++) {
        const int z = z0 + 2 * ty + rr, di = z - bx2.x;
        if (di < 0 || di >= nb) continue;
#pragma unroll
        for (int e = 0; e < 4; e++) {
          const int dj = xb + e - bx2.y;
          if (dj < 0 || dj >= nb) continue;
          const float ms = which ? Mxz * Sh_own[rr][e] : Mxx * Sx_own[rr][e] + Mzz * Sz_own[rr][e];
          const float wv = w[di * SRC_W + dj] * ms;
          acc[0] += wv;
          acc[1] += wv * (((float)(xb + e - g.npml) + off) * p.dx - xs);
          acc[2] += wv * (((float)(z - g.npml) + off) * p.dz - zs);
        }
      }
      cta_sum3(acc, red);
      if (tid == 0) {
        const int slot = 4 * which + 2 * (id.tz - bx2.x / TILE_Z) + (id.tx - bx2.y / TILE_X);
        float* dst = p.src_part + (((long long)s * p.nt + p.n) * ELA_SLOTS + slot) * 3;
        dst[0] = acc[0];
        dst[1] = acc[1];
        dst[2] = acc[2];
      }
    }
  }
  ELA_WALK_END()
}

// ---------------------------------------------------------------------------
// Adjoint of the velocity half step of step n: Vbar (complete adjoint of
// v^{n+1/2}) flows through to v^{n-1/2}; its image is added to Sbar (which
// becomes the adjoint of sigma^n), the memory adjoints M1..M4 are updated and
// the buoyancy correlations accumulated.
constexpr int ADJB_BUF = 2 * H40 * W72;  // Vbar x, z: rows [z0-4, z0+36), cols [x0-4, x0+68)
constexpr int ADJB_SCR = 2 * TILE_Z * W72 + 2 * H40 * TILE_X;
template <int N>
__global__ void __launch_bounds__(NTHREADS, N == 2 ? 3 : 2)  // 3 CTAs per SM at 4th order (80 registers)
    ela_vel_adj(const __grid_constant__ CUtensorMap m_Vx, const __grid_constant__ CUtensorMap m_Vz, const EleStep p) {
  extern __shared__ __align__(128) float smem_e[];
  float* d_sxx = smem_e + ADJB_BUF;           // [TILE_Z][W72] vx nodes, own rows
  float* d_sxz = d_sxx + TILE_Z * W72;        // [H40][TILE_X] vx nodes, own cols
  float* d_szz = d_sxz + H40 * TILE_X;        // [H40][TILE_X] vz nodes, own cols
  float* d_sxzx = d_szz + H40 * TILE_X;       // [TILE_Z][W72] vz nodes, own rows
  uint64_t* bar = reinterpret_cast<uint64_t*>(d_sxzx + TILE_Z * W72);
  const Grid& g = p.g;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int pitch = g.pitch;
  auto fetch = [&](int tt) {
    const TileId f = tile_decode(g, tt);
    fence_proxy_async();
    mbar_expect_tx(&bar[0], ADJB_BUF * 4);
    tma_3d(smem_e, &m_Vx, f.x0 - 4 + APRON, f.z0 - 4 + APRON, f.s, &bar[0]);
    tma_3d(smem_e + H40 * W72, &m_Vz, f.x0 - 4 + APRON, f.z0 - 4 + APRON, f.s, &bar[0]);
  };
  ELA_WALK1_BEGIN(fetch)
  const int xb = x0 + 4 * tx, zr0 = z0 + 2 * ty;
  float4 spre[2][3];
#pragma unroll
  for (int rr = 0; rr < 2; rr++) {
    const long long id = base + (long long)(zr0 + rr) * pitch + xb;
    spre[rr][0] = ld4(p.Sxx + id);
    spre[rr][1] = ld4(p.Szz + id);
    spre[rr][2] = ld4(p.Sxz + id);
  }
  ELA_WAIT1()
  const float* s_Vx = smem_e;
  const float* s_Vz = s_Vx + H40 * W72;
  const bool px = pml_x(g, x0), pz = pml_z(g, z0);
  const float dt = p.dt;
  // the halo items of each kind (the own nodes' are merged below)
  auto item_a = [&](int k) {  // (a) at vx nodes, own rows, columns [x0-4, x0+68): psi1 adjoint (x)
    const int r = k / (W72 / 4), gq = k - r * (W72 / 4);
    const int z = z0 + r, j = x0 - 4 + 4 * gq;
    const long long id = base + (long long)z * pitch + j, im = g.off0 + (long long)z * pitch + j;
    float v[4], b[4], t[4], d[4];
    f4a(ld4(s_Vx + (r + 4) * W72 + 4 * gq), v);
    f4a(ldg4(p.bx + im), b);
#pragma unroll
    for (int e = 0; e < 4; e++) t[e] = dt * b[e] * v[e];
    cpml_adj_x4(px, p.axh, p.bxh, j, p.Min[0], p.Mout[0], id, gq >= 1 && gq <= 16, t, d);
    st4(d_sxx + r * W72 + 4 * gq, a4f(d));
  };
  auto item_b = [&](int k) {  // (b) at vx nodes, rows [z0-4, z0+36), own cols: psi2 adjoint (z)
    const int hr = k / (TILE_X / 4), c = k - hr * (TILE_X / 4);
    const int z = z0 - 4 + hr, j = x0 + 4 * c;
    const long long id = base + (long long)z * pitch + j, im = g.off0 + (long long)z * pitch + j;
    float v[4], b[4], t[4], d[4];
    f4a(ld4(s_Vx + hr * W72 + 4 * c + 4), v);
    f4a(ldg4(p.bx + im), b);
#pragma unroll
    for (int e = 0; e < 4; e++) t[e] = dt * b[e] * v[e];
    cpml_adj_z4(pz, p.az, p.bzt, z, p.Min[1], p.Mout[1], id, hr >= 4 && hr < 4 + TILE_Z, t, d);
    st4(d_sxz + hr * TILE_X + 4 * c, a4f(d));
  };
  auto item_c = [&](int k) {  // (c) at vz nodes, rows [z0-4, z0+36), own cols: psi4 adjoint (z)
    const int hr = k / (TILE_X / 4), c = k - hr * (TILE_X / 4);
    const int z = z0 - 4 + hr, j = x0 + 4 * c;
    const long long id = base + (long long)z * pitch + j, im = g.off0 + (long long)z * pitch + j;
    float v[4], b[4], t[4], d[4];
    f4a(ld4(s_Vz + hr * W72 + 4 * c + 4), v);
    f4a(ldg4(p.bz + im), b);
#pragma unroll
    for (int e = 0; e < 4; e++) t[e] = dt * b[e] * v[e];
    cpml_adj_z4(pz, p.azh, p.bzh, z, p.Min[3], p.Mout[3], id, hr >= 4 && hr < 4 + TILE_Z, t, d);
    st4(d_szz + hr * TILE_X + 4 * c, a4f(d));
  };
  auto item_d = [&](int k) {  // (d) at vz nodes, own rows, columns [x0-4, x0+68): psi3 adjoint (x)
    const int r = k / (W72 / 4), gq = k - r * (W72 / 4);
    const int z = z0 + r, j = x0 - 4 + 4 * gq;
    const long long id = base + (long long)z * pitch + j, im = g.off0 + (long long)z * pitch + j;
    float v[4], b[4], t[4], d[4];
    f4a(ld4(s_Vz + (r + 4) * W72 + 4 * gq), v);
    f4a(ldg4(p.bz + im), b);
#pragma unroll
    for (int e = 0; e < 4; e++) t[e] = dt * b[e] * v[e];
    cpml_adj_x4(px, p.ax, p.bxt, j, p.Min[2], p.Mout[2], id, gq >= 1 && gq <= 16, t, d);
    st4(d_sxzx + r * W72 + 4 * gq, a4f(d));
  };
  // own nodes: items (a) and (b) of a vx-node group, and (c) and (d) of a
  // vz-node group, in one pass each, so that its buoyancy is loaded once
  auto item_ab = [&](int k) {
    const int r = k >> 4, c = k & 15;
    const int z = z0 + r, j = x0 + 4 * c;
    const long long id = base + (long long)z * pitch + j, im = g.off0 + (long long)z * pitch + j;
    float v[4], b[4], t[4], d[4];
    f4a(ld4(s_Vx + (r + 4) * W72 + 4 * c + 4), v);
    f4a(ldg4(p.bx + im), b);
#pragma unroll
    for (int e = 0; e < 4; e++) t[e] = dt * b[e] * v[e];
    cpml_adj_x4(px, p.axh, p.bxh, j, p.Min[0], p.Mout[0], id, true, t, d);
    st4(d_sxx + r * W72 + 4 * (c + 1), a4f(d));
    cpml_adj_z4(pz, p.az, p.bzt, z, p.Min[1], p.Mout[1], id, true, t, d);
    st4(d_sxz + (r + 4) * TILE_X + 4 * c, a4f(d));
  };
  auto item_cd = [&](int k) {
    const int r = k >> 4, c = k & 15;
    const int z = z0 + r, j = x0 + 4 * c;
    const long long id = base + (long long)z * pitch + j, im = g.off0 + (long long)z * pitch + j;
    float v[4], b[4], t[4], d[4];
    f4a(ld4(s_Vz + (r + 4) * W72 + 4 * c + 4), v);
    f4a(ldg4(p.bz + im), b);
#pragma unroll
    for (int e = 0; e < 4; e++) t[e] = dt * b[e] * v[e];
    cpml_adj_z4(pz, p.azh, p.bzh, z, p.Min[3], p.Mout[3], id, true, t, d);
    st4(d_szz + (r + 4) * TILE_X + 4 * c, a4f(d));
    cpml_adj_x4(px, p.ax, p.bxt, j, p.Min[2], p.Mout[2], id, true, t, d);
    st4(d_sxzx + r * W72 + 4 * (c + 1), a4f(d));
  };
  constexpr int NOWN = TILE_Z * (TILE_X / 4);  // own 4-node groups: 512
#pragma unroll 2
  for (int k = tid; k < NOWN; k += NTHREADS) item_ab(k);
#pragma unroll 2
  for (int k = tid; k < NOWN; k += NTHREADS) item_cd(k);
  // halo nodes: the two halo column groups of every own row (items a, d) and
  // the 8 halo rows of the own columns (items b, c)
  if (tid < 2 * TILE_Z) {
    const int k = (tid >> 1) * (W72 / 4) + ((tid & 1) ? W72 / 4 - 1 : 0);
    item_a(k);
    item_d(k);
  } else if (tid < 2 * TILE_Z + 8 * (TILE_X / 4)) {
    const int h = (tid - 2 * TILE_Z) >> 4, c = tid & 15, hr = h < 4 ? h : h + TILE_Z;
    item_b(hr * (TILE_X / 4) + c);
    item_c(hr * (TILE_X / 4) + c);
  }
  // the own nodes' adjoint velocities, read before the buffer is refilled
  float vx_own[2][4], vz_own[2][4];
#pragma unroll
  for (int rr = 0; rr < 2; rr++) {
    const int o = (2 * ty + rr + 4) * W72 + 4 * tx + 4;
    f4a(ld4(s_Vx + o), vx_own[rr]);
    f4a(ld4(s_Vz + o), vz_own[rr]);
  }
  __syncthreads();
  ELA_PREFETCH1(fetch)
  float zs[2][4], zh[2][4];
  {
    float4 W[2 * N + 1];
    load_win<N, TILE_X>(d_szz, 2 * ty + 4 - N, 4 * tx, W);  // D+z^T at normal rows
    zwin<N>(p.cz, W, zs[0], zs[1]);
    load_win<N, TILE_X>(d_sxz, 2 * ty + 5 - N, 4 * tx, W);  // D-z^T at shear half rows
    zwin<N>(p.cz, W, zh[0], zh[1]);
  }
#pragma unroll
  for (int rr = 0; rr < 2; rr++) {
    const int r = 2 * ty + rr, z = z0 + r;
    const long long id = base + (long long)z * pitch + xb;
    float v[12], sx[4], sz[4], sh[4];
    f4a(spre[rr][0], sx);
    f4a(spre[rr][1], sz);
    f4a(spre[rr][2], sh);
    seg12(d_sxx + r * W72 + 4 * tx, v);
#pragma unroll
    for (int e = 0; e < 4; e++) sx[e] -= minus12<N>(p.cx, v, e);
    seg12(d_sxzx + r * W72 + 4 * tx, v);
#pragma unroll
    for (int e = 0; e < 4; e++) {
      sz[e] -= zs[rr][e];
      sh[e] -= zh[rr][e] + plus12<N>(p.cx, v, e);
      if (!(z < g.Nz && xb + e < g.Nx)) {
        sx[e] = 0.f;
        sz[e] = 0.f;
      }
      if (!(z < g.Nz - 1 && xb + e < g.Nx - 1)) sh[e] = 0.f;
    }
    st4(p.Sxx + id, a4f(sx));
    st4(p.Szz + id, a4f(sz));
    st4(p.Sxz + id, a4f(sh));
    // buoyancy correlations
    float fx[4], fz[4], gbx[4], gbz[4];
    const float* vx_ = vx_own[rr];
    const float* vz_ = vz_own[rr];
    f4a(ld4_stream(p.slot[0] + id, l2_evict_first()), fx);
    f4a(ld4_stream(p.slot[1] + id, l2_evict_first()), fz);
    f4a(ld4(p.g_bx + id), gbx);
    f4a(ld4(p.g_bz + id), gbz);
#pragma unroll
    for (int e = 0; e < 4; e++) {
      if (z < g.Nz && xb + e < g.Nx - 1) gbx[e] += dt * vx_[e] * fx[e];
      if (z < g.Nz - 1 && xb + e < g.Nx) gbz[e] += dt * vz_[e] * fz[e];
    }
    st4(p.g_bx + id, a4f(gbx));
    st4(p.g_bz + id, a4f(gbz));
  }
  ELA_WALK_END()
}

// ---------------------------------------------------------------------------
// Medium on the padded grid from the physical vp, vs, rho (edge-replicated):
// lambda and lambda + 2 mu at the normal nodes, buoyancy 2/(rho_a + rho_b)
// at the velocity nodes, harmonic mean of the four mu at the shear nodes (zero
// if any is zero); every allocated cell is written (zero off the nodes).
__global__ void k_ela_medium(const float* __restrict__ vp, const float* __restrict__ vs,
                             const float* __restrict__ rho, Grid g, float* lam, float* lp2m, float* bx, float* bz,
                             float* mxz, float* mu_pad) {
  const long long total = (long long)g.rows * g.pitch;
  auto cell = [&](int i, int j, float* r, float* m, float* l) {
    const int ci = min(max(i - g.npml, 0), g.nz - 1), cj = min(max(j - g.npml, 0), g.nx - 1);
    const long long c = (long long)ci * g.nx + cj;
    const float rr = rho[c], a = vp[c], b = vs[c];
    *r = rr;
    *m = rr * b * b;
    *l = rr * (a * a - 2.f * b * b);
  };
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int row = (int)(idx / g.pitch), col = (int)(idx - (long long)row * g.pitch);
    const int i = row - APRON, j = col - APRON;
    float L = 0.f, LP = 0.f, BX = 0.f, BZ = 0.f, MX = 0.f, MU = 0.f;
    if (i >= 0 && i < g.Nz && j >= 0 && j < g.Nx) {
      float r0, m0, l0;
      cell(i, j, &r0, &m0, &l0);
      L = l0;
      LP = l0 + 2.f * m0;
      MU = m0;
      float r1, m1, l1;
      if (j + 1 < g.Nx) {
        cell(i, j + 1, &r1, &m1, &l1);
        BX = 2.f / (r0 + r1);
      }
      if (i + 1 < g.Nz) {
        cell(i + 1, j, &r1, &m1, &l1);
        BZ = 2.f / (r0 + r1);
      }
      if (i + 1 < g.Nz && j + 1 < g.Nx) {
        float ra, mb, mc, md, la;
        cell(i, j + 1, &ra, &mb, &la);
        cell(i + 1, j, &ra, &mc, &la);
        cell(i + 1, j + 1, &ra, &md, &la);
        if (m0 != 0.f && mb != 0.f && mc != 0.f && md != 0.f)
          MX = (float)(4.0 / (1.0 / m0 + 1.0 / mb + 1.0 / mc + 1.0 / md));
      }
    }
    lam[idx] = L;
    lp2m[idx] = LP;
    bx[idx] = BX;
    bz[idx] = BZ;
    mxz[idx] = MX;
    mu_pad[idx] = MU;
  }
}

// Source boxes and weights on the normal grid (offset 0) and the shear grid
// (offset 1/2): 1/(dx dz) on the nearest node, or the Gaussian
// g/(2 pi s^2) exp(-r^2/(2 s^2)), s = dx/2, on its 7 x 7 neighbourhood.
__global__ void k_ela_src_prep(int S, int kind, const float* __restrict__ x0, Grid g, float dx, float dz, int* box_n,
                               int* box_s, float* w_n, float* w_s, int* status) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  const double xr = x0[2 * s], zr = x0[2 * s + 1];
  bool ok = isfinite(xr) && isfinite(zr);
  for (int which = 0; which < 2; which++) {
    const double off = which ? 0.5 : 0.0;
    const int ni = which ? g.Nz - 1 : g.Nz, nj = which ? g.Nx - 1 : g.Nx;
    int* box = which ? box_s : box_n;
    float* ws = (which ? w_s : w_n) + s * SRC_W * SRC_W;
    for (int q = 0; q < SRC_W * SRC_W; q++) ws[q] = 0.f;
    const int jc = (int)llround(xr / (double)dx - off) + g.npml;
    const int ic = (int)llround(zr / (double)dz - off) + g.npml;
    if (kind == 0) {
      ok = ok && ic >= 0 && ic < ni && jc >= 0 && jc < nj;
      box[2 * s] = ic;
      box[2 * s + 1] = jc;
      ws[0] = (float)(1.0 / ((double)dx * (double)dz));
    } else {
      ok = ok && ic - 3 >= 0 && ic + 3 < ni && jc - 3 >= 0 && jc + 3 < nj;
      box[2 * s] = ic - 3;
      box[2 * s + 1] = jc - 3;
      const double sg = 0.5 * (double)dx;
      for (int di = 0; di < SRC_W; di++)
        for (int dj = 0; dj < SRC_W; dj++) {
          const double xi = ((double)(jc - 3 + dj - g.npml) + off) * dx - xr;
          const double zi = ((double)(ic - 3 + di - g.npml) + off) * dz - zr;
          ws[di * SRC_W + dj] = (float)(exp(-(xi * xi + zi * zi) / (2.0 * sg * sg)) / (2.0 * M_PI * sg * sg));
        }
    }
  }
  if (!ok) {
    box_n[2 * s] = box_n[2 * s + 1] = -1;
    box_s[2 * s] = box_s[2 * s + 1] = -1;
    atomicOr(status, ST_BADSRC);
  }
}

// vp, vs, rho finite with vp > 0, rho > 0, vs >= 0, lambda >= 0; CFL on vp.
__global__ void k_ela_model_check(const float* __restrict__ vp, const float* __restrict__ vs,
                                  const float* __restrict__ rho, long long n, float coef, int* status) {
  __shared__ float smax[32];
  __shared__ int sbad;
  if (threadIdx.x == 0) sbad = 0;
  __syncthreads();
  float mx = 0.f;
  int bad = 0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) {
    const float a = vp[i], b = vs[i], r = rho[i];
    if (!(a > 0.f) || !isfinite(a) || !(b >= 0.f) || !isfinite(b) || !(r > 0.f) || !isfinite(r) ||
        a * a < 2.f * b * b)
      bad = 1;
    else
      mx = fmaxf(mx, a);
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = mx;
  if (bad) atomicOr(&sbad, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) m = fmaxf(m, smax[w]);
    if (sbad) atomicOr(status, ST_BADMODEL);
    else if (m * coef > 1.f) atomicOr(status, ST_CFL);
  }
}

// Segment fold of the five FP32 correlation partials into FP64 (sum over shots).
struct Parts5 {
  float* f[5];
};
__global__ void k_ela_fold(Parts5 parts, int S, long long slice, double* G) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < slice;
       i += (long long)gridDim.x * blockDim.x) {
    for (int f = 0; f < 5; f++) {
      float* pp = parts.f[f];
      double acc = 0.0;
      for (int s = 0; s < S; s++) {
        acc += (double)pp[(long long)s * slice + i];
        pp[(long long)s * slice + i] = 0.f;
      }
      G[(long long)f * slice + i] += acc;
    }
  }
}

// Chain rule to the physical lambda, mu, rho: mu also collects the shear-node
// correlation through the harmonic mean (d mu_xz / d mu_k = mu_xz^2 / (4 mu_k^2)),
// rho collects the buoyancy correlations (d b / d rho = -b^2 / 2 for each of
// the two cells averaged), and a physical cell collects the CPML cells that
// replicate it. G = [lam, mu, mxz, bx, bz] FP64 partials on the padded nodes.
__global__ void k_ela_grad(const double* __restrict__ G, Grid g, const float* __restrict__ mxz,
                           const float* __restrict__ mu_pad, const float* __restrict__ bx,
                           const float* __restrict__ bz, float* out) {
  const long long n = (long long)g.nz * g.nx;
  const long long sl = g.slice;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const int iz = (int)(idx / g.nx), ix = (int)(idx - (long long)iz * g.nx);
    const int i_lo = iz == 0 ? 0 : iz + g.npml, i_hi = iz == g.nz - 1 ? g.Nz - 1 : iz + g.npml;
    const int j_lo = ix == 0 ? 0 : ix + g.npml, j_hi = ix == g.nx - 1 ? g.Nx - 1 : ix + g.npml;
    double gl = 0.0, gm = 0.0, gr = 0.0;
    for (int i = i_lo; i <= i_hi; i++)
      for (int j = j_lo; j <= j_hi; j++) {
        const long long c = g.off0 + (long long)i * g.pitch + j;
        gl += G[c];
        gm += G[sl + c];
        const double mu = mu_pad[c];
        for (int di = -1; di <= 0; di++)
          for (int dj = -1; dj <= 0; dj++) {
            const int si = i + di, sj = j + dj;
            if (si < 0 || sj < 0 || si >= g.Nz - 1 || sj >= g.Nx - 1) continue;
            const long long sc = g.off0 + (long long)si * g.pitch + sj;
            const double m = mxz[sc];
            if (m != 0.0) gm += G[2 * sl + sc] * m * m / (4.0 * mu * mu);
          }
        for (int dj = -1; dj <= 0; dj++) {
          const int sj = j + dj;
          if (sj < 0 || sj >= g.Nx - 1) continue;
          const long long sc = g.off0 + (long long)i * g.pitch + sj;
          const double b = bx[sc];
          gr += -0.5 * b * b * G[3 * sl + sc];
        }
        for (int di = -1; di <= 0; di++) {
          const int si = i + di;
          if (si < 0 || si >= g.Nz - 1) continue;
          const long long sc = g.off0 + (long long)si * g.pitch + j;
          const double b = bz[sc];
          gr += -0.5 * b * b * G[4 * sl + sc];
        }
      }
    out[idx] = (float)gl;
    out[n + idx] = (float)gm;
    out[2 * n + idx] = (float)gr;
  }
}

// Chain rule from (lambda, mu, rho) to (vp, vs, rho) per cell; in place allowed.
__global__ void k_ela_velocity_grad(const float* __restrict__ vp, const float* __restrict__ vs,
                                    const float* __restrict__ rho, const float* gin, float* gout, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float a = vp[i], b = vs[i], r = rho[i];
    const float gl = gin[i], gm = gin[n + i], gr = gin[2 * n + i];
    gout[i] = 2.f * r * a * gl;
    gout[n + i] = 2.f * r * b * (gm - 2.f * gl);
    gout[2 * n + i] = (a * a - 2.f * b * b) * gl + b * b * gm + gr;
  }
}

// ---------------------------------------------------------------------------
// launchers: one-time kernel attributes and occupancy-sized persistent grids
// per device, tensor maps per call.
namespace {
constexpr size_t VEL_SMEM = sizeof(float) * 2 * VEL_BUF + 2 * sizeof(uint64_t);
constexpr size_t STR_SMEM = sizeof(float) * 2 * STR_BUF + 2 * sizeof(uint64_t);
constexpr size_t ADJ_A_SMEM = sizeof(float) * (ADJA_BUF + ADJA_SCR) + sizeof(uint64_t);  // one operand buffer
constexpr size_t ADJ_B_SMEM = sizeof(float) * (ADJB_BUF + ADJB_SCR) + sizeof(uint64_t);

std::mutex g_ela_mu;
unsigned long long g_ela_inited = 0;  // bit per device
// [device][order 4/8][variant]: vel (plain, record, store), str (plain, store), adjA, adjB,
// vel (record and store: the forward sweep over the last checkpoint segment)
int g_ela_grid[64][2][8];

template <typename K>
cudaError_t ela_setup(K k, size_t smem, int* grid) {
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0, nb = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, NTHREADS, smem)) != cudaSuccess) return e;
  *grid = (nb < 1 ? 1 : nb) * nsm;
  return cudaSuccess;
}

template <int N>
cudaError_t ela_setup_order(int* gr) {
  cudaError_t e;
  if ((e = ela_setup(ela_vel_step<N, false, false>, VEL_SMEM, &gr[0])) != cudaSuccess) return e;
  if ((e = ela_setup(ela_vel_step<N, true, false>, VEL_SMEM, &gr[1])) != cudaSuccess) return e;
  if ((e = ela_setup(ela_vel_step<N, false, true>, VEL_SMEM, &gr[2])) != cudaSuccess) return e;
  if ((e = ela_setup(ela_str_step<N, false>, STR_SMEM, &gr[3])) != cudaSuccess) return e;
  if ((e = ela_setup(ela_str_step<N, true>, STR_SMEM, &gr[4])) != cudaSuccess) return e;
  if ((e = ela_setup(ela_str_adj<N>, ADJ_A_SMEM, &gr[5])) != cudaSuccess) return e;
  if ((e = ela_setup(ela_vel_step<N, true, true>, VEL_SMEM, &gr[7])) != cudaSuccess) return e;
  return ela_setup(ela_vel_adj<N>, ADJ_B_SMEM, &gr[6]);
}

cudaError_t ela_ensure_init(int* dev_out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  *dev_out = dev;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_ela_mu);
  if (g_ela_inited & (1ull << dev)) return cudaSuccess;
  if ((e = ela_setup_order<2>(g_ela_grid[dev][0])) != cudaSuccess) return e;
  if ((e = ela_setup_order<4>(g_ela_grid[dev][1])) != cudaSuccess) return e;
  g_ela_inited |= 1ull << dev;
  return cudaSuccess;
}

int ela_grid(const EleStep& p, int dev, int variant) {
  return std::min(p.S * p.g.ntx * p.g.ntz, g_ela_grid[dev][p.N == 2 ? 0 : 1][variant]);
}
}  // namespace

cudaError_t ela_kernels_init() {
  int dev;
  return ela_ensure_init(&dev);
}

// TMA descriptors for a call over the five forward fields f = (vx, vz, sxx,
// szz, sxz) and, if a is not null, the five adjoint fields in the same order;
// each field is [S][rows][pitch].
cudaError_t ela_make_maps(EleMaps* maps, const Grid& g, int S, float* const* f, float* const* a) {
  const cuuint64_t d3[3] = {(cuuint64_t)g.pitch, (cuuint64_t)g.rows, (cuuint64_t)S};
  const cuuint64_t s3[2] = {(cuuint64_t)g.pitch * 4, (cuuint64_t)g.slice * 4};
  const cuuint32_t bxx[3] = {(cuuint32_t)W72, (cuuint32_t)TILE_Z, 1};
  const cuuint32_t bzz[3] = {(cuuint32_t)TILE_X, (cuuint32_t)H40, 1};
  const cuuint32_t bfull[3] = {(cuuint32_t)W72, (cuuint32_t)H40, 1};
  bool ok = tma_host::encode(&maps->vx, f[0], 3, d3, s3, bfull) && tma_host::encode(&maps->vz, f[1], 3, d3, s3, bfull) &&
            tma_host::encode(&maps->sxx, f[2], 3, d3, s3, bxx) && tma_host::encode(&maps->szz, f[3], 3, d3, s3, bzz) &&
            tma_host::encode(&maps->sxz, f[4], 3, d3, s3, bfull);
  if (ok && a)
    ok = tma_host::encode(&maps->Vx, a[0], 3, d3, s3, bfull) && tma_host::encode(&maps->Vz, a[1], 3, d3, s3, bfull) &&
         tma_host::encode(&maps->Sxx, a[2], 3, d3, s3, bfull) && tma_host::encode(&maps->Szz, a[3], 3, d3, s3, bfull) &&
         tma_host::encode(&maps->Sxz, a[4], 3, d3, s3, bfull);
  return ok ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_ela_vel(const EleStep& p, const EleMaps& m, bool record, bool store, cudaStream_t st) {
  int dev;
  cudaError_t e = ela_ensure_init(&dev);
  if (e != cudaSuccess) return e;
  const int grid = ela_grid(p, dev, record ? (store ? 7 : 1) : (store ? 2 : 0));
  if (p.N == 2) {
    if (record && store) ela_vel_step<2, true, true><<<grid, NTHREADS, VEL_SMEM, st>>>(m.sxx, m.szz, m.sxz, p);
    else if (record) ela_vel_step<2, true, false><<<grid, NTHREADS, VEL_SMEM, st>>>(m.sxx, m.szz, m.sxz, p);
    else if (store) ela_vel_step<2, false, true><<<grid, NTHREADS, VEL_SMEM, st>>>(m.sxx, m.szz, m.sxz, p);
    else ela_vel_step<2, false, false><<<grid, NTHREADS, VEL_SMEM, st>>>(m.sxx, m.szz, m.sxz, p);
  } else {
    if (record && store) ela_vel_step<4, true, true><<<grid, NTHREADS, VEL_SMEM, st>>>(m.sxx, m.szz, m.sxz, p);
    else if (record) ela_vel_step<4, true, false><<<grid, NTHREADS, VEL_SMEM, st>>>(m.sxx, m.szz, m.sxz, p);
    else if (store) ela_vel_step<4, false, true><<<grid, NTHREADS, VEL_SMEM, st>>>(m.sxx, m.szz, m.sxz, p);
    else ela_vel_step<4, false, false><<<grid, NTHREADS, VEL_SMEM, st>>>(m.sxx, m.szz, m.sxz, p);
  }
  return cudaGetLastError();
}

cudaError_t launch_ela_str(const EleStep& p, const EleMaps& m, bool store, cudaStream_t st) {
  int dev;
  cudaError_t e = ela_ensure_init(&dev);
  if (e != cudaSuccess) return e;
  const int grid = ela_grid(p, dev, store ? 4 : 3);
  if (p.N == 2) {
    if (store) ela_str_step<2, true><<<grid, NTHREADS, STR_SMEM, st>>>(m.vx, m.vz, p);
    else ela_str_step<2, false><<<grid, NTHREADS, STR_SMEM, st>>>(m.vx, m.vz, p);
  } else {
    if (store) ela_str_step<4, true><<<grid, NTHREADS, STR_SMEM, st>>>(m.vx, m.vz, p);
    else ela_str_step<4, false><<<grid, NTHREADS, STR_SMEM, st>>>(m.vx, m.vz, p);
  }
  return cudaGetLastError();
}

cudaError_t launch_ela_adj(const EleStep& p, const EleMaps& m, cudaStream_t st) {
  int dev;
  cudaError_t e = ela_ensure_init(&dev);
  if (e != cudaSuccess) return e;
  const int ga = ela_grid(p, dev, 5), gb = ela_grid(p, dev, 6);
  if (p.N == 2) {
    ela_str_adj<2><<<ga, NTHREADS, ADJ_A_SMEM, st>>>(m.Sxx, m.Szz, m.Sxz, p);
    ela_vel_adj<2><<<gb, NTHREADS, ADJ_B_SMEM, st>>>(m.Vx, m.Vz, p);
  } else {
    ela_str_adj<4><<<ga, NTHREADS, ADJ_A_SMEM, st>>>(m.Sxx, m.Szz, m.Sxz, p);
    ela_vel_adj<4><<<gb, NTHREADS, ADJ_B_SMEM, st>>>(m.Vx, m.Vz, p);
  }
  return cudaGetLastError();
}

cudaError_t launch_ela_medium(const float* vp, const float* vs, const float* rho, const Grid& g, float* lam,
                              float* lp2m, float* bx, float* bz, float* mxz, float* mu_pad, cudaStream_t st) {
  k_ela_medium<<<304, 256, 0, st>>>(vp, vs, rho, g, lam, lp2m, bx, bz, mxz, mu_pad);
  return cudaGetLastError();
}
cudaError_t launch_ela_src_prep(int S, int kind, const float* x0, const Grid& g, float dx, float dz, int* box_n,
                                int* box_s, float* w_n, float* w_s, int* status, cudaStream_t st) {
  k_ela_src_prep<<<(S + 127) / 128, 128, 0, st>>>(S, kind, x0, g, dx, dz, box_n, box_s, w_n, w_s, status);
  return cudaGetLastError();
}
cudaError_t launch_ela_model_check(const float* vp, const float* vs, const float* rho, long long n, float coef,
                                   int* status, cudaStream_t st) {
  k_ela_model_check<<<1, 1024, 0, st>>>(vp, vs, rho, n, coef, status);
  return cudaGetLastError();
}
cudaError_t launch_ela_fold(float* const* parts, int S, long long slice, double* G, cudaStream_t st) {
  Parts5 p5;
  for (int f = 0; f < 5; f++) p5.f[f] = parts[f];
  k_ela_fold<<<608, 256, 0, st>>>(p5, S, slice, G);
  return cudaGetLastError();
}
cudaError_t launch_ela_velocity_grad(const float* vp, const float* vs, const float* rho, const float* gin,
                                     float* gout, long long n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const long long blocks = std::min<long long>((n + 255) / 256, 1216);
  k_ela_velocity_grad<<<(int)blocks, 256, 0, st>>>(vp, vs, rho, gin, gout, n);
  return cudaGetLastError();
}
cudaError_t launch_ela_grad(const double* G, const Grid& g, const float* mxz, const float* mu_pad, const float* bx,
                            const float* bz, float* out, cudaStream_t st) {
  k_ela_grad<<<304, 256, 0, st>>>(G, g, mxz, mu_pad, bx, bz, out);
  return cudaGetLastError();
}

}  // namespace fwi
