// acoustic_kernels.cu - sm_103a step kernels of the acoustic hot path.
//
// One time step of the recursion U_{k+1} = A(theta) U_k + F_k (Method,
// Eq. forward) for u_tt = div(c^2 grad u) + f (Implementation, Eq. acoustic)
// on the staggered grid with CPML, and one step of its exact transpose
// lambda_k = A^T lambda_{k+1} + residual (Eq. adjoint-backward) fused with the
// gradient correlation lambda^T (dA/dm) U (Eq. adjoint-gradient).
//
// Design (memory bound, no dense contraction, so no tensor cores):
//   * persistent CTAs (grid = resident CTAs of the GPU) walk the tiles of all
//     shots; a tile is 64 x 32 cells of one shot;
//   * the stencil operand tiles with their 8-cell halo and the coefficient tile are
//     fetched by TMA (cp.async.bulk.tensor) into the CTA's one operand buffer
//     as soon as stage 1 (their last reader) has passed its barrier, so the
//     next tile's fetch overlaps the current tile's stage 2 and the other
//     resident CTAs cover the rest; the completion wait on the mbarrier is
//     bounded and reports a timeout;
//   * stage 1 evaluates each half-point flux once (x: q at the half columns
//     of the tile and its halo; z: a register window over two rows per thread),
//     stage 2 the divergence, update, sources and receivers;
//   * per-cell operands that do not need a halo: u^{n-1} is copied into shared
//     memory by cp.async issued before the wait (its latency overlaps the tile
//     fetch and stage 1 without holding registers); the adjoint's stored fluxes
//     are float4 loads issued there too, its lambda_{n+2} and gradient partial
//     are loaded at the start of stage 2.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <type_traits>

#include "fwi_internal.cuh"
#include "tma.cuh"

namespace fwi {

namespace {

constexpr int H = 8;                     // wavefield halo (>= 2N-1)
constexpr int UW = TILE_X + 2 * H;       // 80: wavefield tile width
constexpr int UH = TILE_Z + 2 * H;       // 48: wavefield tile height
constexpr int MW = TILE_X + 12;          // 76: m tile cols [x0-4, x0+TX+8)
constexpr int MH = TILE_Z + 9;           // 41: m tile rows [z0-4, z0+TZ+5)
constexpr int QXW = TILE_X + 8;          // 72: half cols [x0-4, x0+TX+4)
constexpr int QZH = TILE_Z + 8;          // 40: half rows [z0-4, z0+TZ+4)
constexpr int M_BYTES = MW * MH * 4;     // 12464
constexpr int M_SLOT = (M_BYTES + 127) / 128 * 128;
#ifndef FWI_FWD_CTAS
#define FWI_FWD_CTAS 4
#endif
constexpr int FWD_CTAS = FWI_FWD_CTAS;     // resident forward CTAs per SM the registers are sized for
constexpr int XS_BYTES = TILE_Z * UW * 4;  // 10240: adjoint x operand tile
// Geometry of a forward tile of TZ rows (TZ = 32 or 64) and TILE_X columns: 16
// columns of threads, each thread owning 2 rows x 4 columns (so 8 * TZ threads).
template <int TZ>
struct FwdGeo {
  static constexpr int NT = 8 * TZ;           // threads per CTA
  static constexpr int UHT = TZ + 2 * H;      // wavefield tile height
  static constexpr int MHT = TZ + 9;          // m tile rows [z0-4, z0+TZ+5)
  static constexpr int QZHT = TZ + 8;         // half rows [z0-4, z0+TZ+4)
  static constexpr int UB = UW * UHT * 4;
  static constexpr int MB = MW * MHT * 4;
  static constexpr int MSLOT = (MB + 127) / 128 * 128;
};
constexpr int ZS_BYTES = UH * TILE_X * 4;  // 12288: adjoint z operand tile

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float4 ldg4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ void unpack12(const float* s, float v[12]) {
  const float4 a = ld4(s), b = ld4(s + 4), c = ld4(s + 8);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  v[8] = c.x; v[9] = c.y; v[10] = c.z; v[11] = c.w;
}
__device__ __forceinline__ void f4a(const float4 v, float o[4]) {
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
// float4 stencil accumulation: acc += c (p - m)
__device__ __forceinline__ void acc4(float4& acc, float c, const float4 p, const float4 m) {
  acc.x += c * (p.x - m.x); acc.y += c * (p.y - m.y); acc.z += c * (p.z - m.z); acc.w += c * (p.w - m.w);
}

// 16-byte asynchronous global -> shared copies (L2 only): per-cell operands of
// stage 2 land in shared memory while stage 1 runs, holding no registers.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ bool tile_pml_x(const Grid& g, int x0) {
  return g.npml > 0 && (x0 - H < g.npml || x0 + TILE_X + H > g.npml + g.nx - 1);
}
template <int TZ = TILE_Z>
__device__ __forceinline__ bool tile_pml_z(const Grid& g, int z0) {
  return g.npml > 0 && (z0 - H < g.npml || z0 + TZ + H > g.npml + g.nz - 1);
}
// Tile t of a walk over TZ-row tiles (the 32-row walk is tile_decode).
template <int TZ>
__device__ __forceinline__ TileId tile_decode_t(const Grid& g, int t) {
  if (TZ == TILE_Z) return tile_decode(g, t);
  const int ntz = (g.Nz + TZ - 1) / TZ;
  TileId r;
  r.tx = t % g.ntx;
  const int q = t / g.ntx;
  r.tz = q % ntz;
  r.s = q / ntz;
  r.x0 = r.tx * TILE_X;
  r.z0 = r.tz * TZ;
  return r;
}

// Points of one axis where the CPML coefficients can be nonzero (the tables are
// built with a layer distance l > 0 only there): half points h < npml or
// h >= npml + n - 1, integer points x < npml or x >= npml + n (n physical
// cells). A tile that touches a layer runs its CPML updates only on the items
// [h0, h1] that meet one; elsewhere a = 0 and the memory variables stay zero.
__device__ __forceinline__ bool layer_h(int h0, int h1, int npml, int n) { return h0 < npml || h1 >= npml + n - 1; }
__device__ __forceinline__ bool layer_c(int x0, int x1, int npml, int n) { return x0 < npml || x1 >= npml + n; }

// Tiles that leave hhat behind for the next adjoint step: those whose own
// columns (rows) lie in the stencil reach of a CPML tile (itself or a neighbour).
__device__ __forceinline__ bool tile_writes_hx(const Grid& g, int tx) {
  bool w = false;
#pragma unroll
  for (int d = -1; d <= 1; d++) {
    const int t2 = tx + d;
    w = w || (t2 >= 0 && t2 < g.ntx && tile_pml_x(g, t2 * TILE_X));
  }
  return w;
}
__device__ __forceinline__ bool tile_writes_hz(const Grid& g, int tz) {
  bool w = false;
#pragma unroll
  for (int d = -1; d <= 1; d++) {
    const int t2 = tz + d;
    w = w || (t2 >= 0 && t2 < g.ntz && tile_pml_z(g, t2 * TILE_Z));
  }
  return w;
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

// Issue the TMA fetches of tile t (TZ rows) into one buffer (one elected thread).
// plane0: the pair plane of this launch's first shot.
template <int TZ = TILE_Z>
__device__ __forceinline__ void fetch_tile(const CUtensorMap* fmap, const CUtensorMap* mmap, const Grid& g, int plane0,
                                           int t, float* dst_u, float* dst_m, uint64_t* bar) {
  const TileId id = tile_decode_t<TZ>(g, t);
  fence_proxy_async();
  mbar_expect_tx(bar, FwdGeo<TZ>::UB + FwdGeo<TZ>::MB);
  // allocation coordinates: padded (i, j) -> (i + APRON, j + APRON)
  tma_3d(dst_u, fmap, id.x0 - H + APRON, id.z0 - H + APRON, plane0 + id.s, bar);
  tma_2d(dst_m, mmap, id.x0 - 4 + APRON, id.z0 - 4 + APRON, bar);
}

// Shared memory of the step kernels (every array a multiple of 128 bytes).
template <int TZ>
struct FwdSmemT {
  float u[FwdGeo<TZ>::UHT * UW];
  float m[FwdGeo<TZ>::MSLOT / 4];
  float qx[TZ * QXW];
  float qz[FwdGeo<TZ>::QZHT * TILE_X];
  float4 up4[2 * FwdGeo<TZ>::NT];  // u^{n-1} of the own cells, [row][thread] (cp.async)
  float red[32];
  uint64_t bar;
};
using FwdSmem = FwdSmemT<TILE_Z>;
struct AdjSmem {
  float xs[TILE_Z * UW];     // x stencil operand (lambda or Hx): own rows, cols [x0-H, x0+TX+H)
  float zs[UH * TILE_X];     // z stencil operand (lambda or Hz): rows [z0-H, z0+TZ+H), own cols
  float m[M_SLOT / 4];
  float gx[TILE_Z * QXW];
  float gz[QZH * TILE_X];
  float imz[(NTHREADS / 16 + 1) * TILE_X];  // image at half row z0-1 and at each thread row's lower half row
  float imx[TILE_Z];                        // image at half column x0-1 of every row
  float red[32];
  uint64_t bar;
};
// Multi-instance launches keep the current tile's step parameters after the
// kernel's own shared memory.
constexpr size_t FWD_SMEM_MAIN = (sizeof(FwdSmem) + 15) / 16 * 16;
constexpr size_t ADJ_SMEM_MAIN = (sizeof(AdjSmem) + 15) / 16 * 16;

// Multi-instance launches: the instance of tile t (the last i with tile_start[i] <= t).
__device__ __forceinline__ int batch_instance(const BatchArgs& b, int t) {
  int lo = 0, hi = b.n_active - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(b.tile_start + mid) <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}
// Orders the host's writes of a tensor map in global memory before the TMA
// unit reads it.
__device__ __forceinline__ void tensormap_acquire(const CUtensorMap* m) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(m))
               : "memory");
}
// Step parameters of instance i at step b.n, copied into shared memory by warp 0
// (then one barrier). KIND: 0 forward sweep (stores the fluxes from the
// instance's last segment on), 1 recompute (stores), 2 adjoint.
template <int KIND>
__device__ __forceinline__ void batch_load_step(const BatchArgs& b, int i, AcuStep& dst) {
  if (threadIdx.x < 32) {
    const AcuInst* in = b.inst + i;
    const int* src = reinterpret_cast<const int*>(&in->p);
    int* d = reinterpret_cast<int*>(&dst);
    for (int w = threadIdx.x; w < (int)(sizeof(AcuStep) / 4); w += 32) d[w] = __ldg(src + w);
    __syncwarp();
    if (threadIdx.x == 0) {
      const int n = b.n;
      const long long f = in->field;
      float* slot = in->slot + (long long)(n - (n / b.K) * b.K) * 2 * f;
      dst.n = n;
      if (KIND == 2) {
        dst.cur = (n + 1) & 1;  // lambda_{n+1}; lambda_{n+2} -> lambda_n in the other half
        dst.slot_px = slot;
        dst.slot_pz = slot + f;
        dst.zx_in = in->zx[(n + 1) & 1];
        dst.zx_out = in->zx[n & 1];
        dst.zz_in = in->zz[(n + 1) & 1];
        dst.zz_out = in->zz[n & 1];
        dst.px_in = in->px[(n + 1) & 1];
        dst.px_out = in->px[n & 1];
        dst.pz_in = in->pz[(n + 1) & 1];
        dst.pz_out = in->pz[n & 1];
        dst.hx_out = in->hxp + (n & 1) * f;
        dst.hz_out = in->hzp + (n & 1) * f;
      } else {
        dst.cur = n & 1;
        dst.psix_in = in->psix[n & 1];
        dst.psix_out = in->psix[(n + 1) & 1];
        dst.psiz_in = in->psiz[n & 1];
        dst.psiz_out = in->psiz[(n + 1) & 1];
        const bool keep = KIND == 1 || n >= in->nlast;
        dst.slot_px = keep ? slot : nullptr;
        dst.slot_pz = keep ? slot + f : nullptr;
      }
    }
  }
  __syncthreads();
}

}  // namespace

// ---------------------------------------------------------------------------
// Forward step n: u^{n+1} = 2 u^n - u^{n-1} + dt^2 (D-(m_half (D+ u^n + psi)) + zeta + f^n)
// per axis, with psi <- b_h psi + a_h D+u and zeta <- b zeta + a D-(q) (zeta is
// kept multiplied by dt^2). RECORD writes the receiver samples; STORE keeps
// p = D+u + psi of every half point (the operand of the gradient correlation).
//
// MULTI: one launch over the tiles of several instances (BatchArgs); each tile
// takes its instance's parameters and tensor maps from the device table, and a
// forward-sweep launch (RECORD and STORE) stores the fluxes only for the
// instances in their last segment (a null slot otherwise).
//
// TZ: the tile height, 32 (256 threads) or 64 (512 threads, a compile-time
// variant for the autotuner: half the z-halo recompute per cell, the same
// per-thread work); multi-instance launches use 32.
// LAP: the c^2 Laplacian operator instead of the divergence form: the fluxes
// carry no coefficient (q = D+u + psi), the update is
// u^{n+1} = 2u^n - u^{n-1} + m dt^2 (D-q + zeta) + dt^2 w g(t_n) with m = c^2 at
// the cell, and STORE keeps r = dt^2 (D-q + zeta) at the cells (the operand of
// its gradient correlation dJ/dm = sum_n lambda_{n+1} r^n) instead of the fluxes.
template <int N, bool RECORD, bool STORE, bool MULTI, int TZ, bool LAP = false>
__global__ void __launch_bounds__(FwdGeo<TZ>::NT, TZ == TILE_Z ? FWD_CTAS : 2)
    acu_fwd_step(const __grid_constant__ CUtensorMap tmap_u, const __grid_constant__ CUtensorMap tmap_m,
                 const __grid_constant__ AcuStep p0, const AcuCoef cf, const BatchArgs b) {
  static_assert(TZ == TILE_Z || (TZ == 2 * TILE_Z && !MULTI), "tile heights: 32, or 64 for single-instance launches");
  static_assert(!LAP || (TZ == TILE_Z && !MULTI), "the Laplacian operator runs on 32-row single-instance launches");
  constexpr int NT = FwdGeo<TZ>::NT;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  FwdSmemT<TZ>& sh = *reinterpret_cast<FwdSmemT<TZ>*>(smem_raw);
  AcuStep& shp = *reinterpret_cast<AcuStep*>(smem_raw + FWD_SMEM_MAIN);  // MULTI only
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const uint64_t pol = STORE ? l2_evict_first() : 0ull;  // segment slots stream through L2
  const int ntiles = MULTI ? b.ntiles : p0.ntiles;
  // TMA fetch of tile tt (one thread)
  auto fetch_next = [&](int tt) {
    if (MULTI) {
      const int i = batch_instance(b, tt);
      const AcuInst* in = b.inst + i;
      const Grid gi = in->p.g;
      tensormap_acquire(&in->mu);
      tensormap_acquire(&in->mm);
      fetch_tile(&in->mu, &in->mm, gi, (b.n & 1) * in->p.S, tt - __ldg(b.tile_start + i), sh.u, sh.m, &sh.bar);
    } else {
      fetch_tile<TZ>(&tmap_u, &tmap_m, p0.g, p0.cur * p0.S_pair + p0.s0, tt, sh.u, sh.m, &sh.bar);
    }
  };

  // one operand buffer: the next tile's fetch is issued once stage 1 of this
  // tile (its last reader) is done, and overlaps stage 2
  if (tid == 0) {
    mbar_init(&sh.bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0 && (int)blockIdx.x < ntiles) fetch_next(blockIdx.x);

  int it = 0, inst_loaded = -1;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x, it++) {
    const int tn = t + gridDim.x;
    int tl = t;  // tile index within its instance
    if (MULTI) {
      const int i = batch_instance(b, t);
      tl = t - __ldg(b.tile_start + i);
      if (i != inst_loaded) {  // the parameters stay in shared memory while the instance does not change
        batch_load_step<RECORD ? 0 : 1>(b, i, shp);  // after the previous tile's closing barrier
        inst_loaded = i;
      }
    }
    const AcuStep& p = MULTI ? shp : p0;
    const Grid& g = p.g;
    const int pitch = g.pitch;
    const TileId id = tile_decode_t<TZ>(g, tl);
    const int x0 = id.x0, z0 = id.z0, s = id.s;
    const long long base = (long long)s * g.slice + g.off0;
    float* __restrict__ uprev = p.u + (long long)((p.cur ^ 1) * p.S_pair + p.s0) * g.slice + base;
    // u^{n-1} of this thread's 2 x 4 cells: copied into shared memory while the
    // tile is fetched and stage 1 runs
    const int xb = x0 + 4 * tx, zr0 = z0 + 2 * ty;
#pragma unroll
    for (int rr = 0; rr < 2; rr++) cp_async16(&sh.up4[rr * NT + tid], uprev + (long long)(zr0 + rr) * pitch + xb);
    cp_async_commit();
    // small per-tile operands, fetched before the wait as well
    const int2 box = __ldg(reinterpret_cast<const int2*>(p.src_box) + s);
    const float stf_n = __ldg(p.stf + (long long)s * p.nt + p.n);
    // receivers: the lists are kept per thread of a 32-row tile; a thread of a
    // 64-row tile owns the same 2 x 4 cells as thread (ty % 16, tx) of 32-row
    // tile 2 tz + ty / 16 (beyond the grid's last 32-row tile: no receivers)
    const int tz32 = id.tz * (TZ / TILE_Z) + ty / 16;
    int rb = 0, re = 0;
    if (RECORD && tz32 < g.ntz) {
      const int key = (tz32 * g.ntx + id.tx) * NTHREADS + (ty % 16) * 16 + tx;
      rb = __ldg(p.thr_rec_start + key);
      re = __ldg(p.thr_rec_start + key + 1);
    }

    const bool ok = mbar_wait(&sh.bar, it & 1);
    if (__syncthreads_or(!ok)) {
      cp_async_wait_all();  // no copy may land after the CTA has exited
      if (tid == 0) {
        atomicOr(p.status, ST_TIMEOUT);
        mbar_wait(&sh.bar, it & 1);  // let a late copy land before the CTA exits
      }
      return;
    }
    const float* su = sh.u;
    const float* sm = sh.m;
    const bool pmlx = tile_pml_x(g, x0), pmlz = tile_pml_z<TZ>(g, z0);

    // ---- stage 1a: x fluxes q = m_half (D+u + psi) at 4 half columns of row r
    auto qx_item = [&](int r, int gq, bool own) {
      const int z = z0 + r, hb = x0 - 4 + 4 * gq;
      float v[12];
      unpack12(su + (r + H) * UW + 4 * gq, v);
      const float4 m4 = ld4(sm + (r + 4) * MW + 4 * gq);
      const float mv[5] = {m4.x, m4.y, m4.z, m4.w, sm[(r + 4) * MW + 4 * gq + 4]};
      float q[4], pp[4];
#pragma unroll
      for (int e = 0; e < 4; e++) {
        float gx = 0.f;
#pragma unroll
        for (int k = 1; k <= N; k++) gx += cf.c1x[k - 1] * (v[e + 4 + k] - v[e + 5 - k]);
        pp[e] = gx;
      }
      const long long id0 = base + (long long)z * pitch + hb;
      if (pmlx && layer_h(hb, hb + 3, g.npml, g.nx)) {
        const float4 a4 = ldg4(p.axh + hb + TAB_OFF);
        if (a4.x != 0.f || a4.y != 0.f || a4.z != 0.f || a4.w != 0.f) {
          // psi <- b psi + a g; zero where a = 0 (psi stays zero outside the layer)
          const float4 b4 = ldg4(p.bxh + hb + TAB_OFF);
          const float4 po = ld4(p.psix_in + id0);
          float4 pn;
          pn.x = b4.x * po.x + a4.x * pp[0]; pn.y = b4.y * po.y + a4.y * pp[1];
          pn.z = b4.z * po.z + a4.z * pp[2]; pn.w = b4.w * po.w + a4.w * pp[3];
          if (own && z < g.Nz) st4(p.psix_out + id0, pn);
          pp[0] += pn.x; pp[1] += pn.y; pp[2] += pn.z; pp[3] += pn.w;
        }
      }
      const bool rowok = z < g.Nz;
#pragma unroll
      for (int e = 0; e < 4; e++)
        q[e] = (rowok && hb + e >= 0 && hb + e < g.Nx - 1) ? (LAP ? pp[e] : (mv[e] + mv[e + 1]) * pp[e]) : 0.f;
      st4(sh.qx + r * QXW + 4 * gq, make_float4(q[0], q[1], q[2], q[3]));
      // every own row is written (zero beyond the grid): the adjoint multiplies these by zero there
      if (STORE && !LAP && own && (!MULTI || p.slot_px))
        st4_stream(p.slot_px + id0, rowok ? make_float4(pp[0], pp[1], pp[2], pp[3]) : make_float4(0.f, 0.f, 0.f, 0.f), pol);
    };
    // ---- stage 1b: z fluxes at one half row (the tile's halo rows)
    auto qz_item = [&](int hr, int c) {
      const int hz = z0 - 4 + hr, xc = x0 + 4 * c;
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int k = 1; k <= N; k++)
        acc4(acc, cf.c1z[k - 1], ld4(su + (hr + 4 + k) * UW + 8 + 4 * c), ld4(su + (hr + 5 - k) * UW + 8 + 4 * c));
      float pp[4];
      f4a(acc, pp);
      if (pmlz && layer_h(hz, hz, g.npml, g.nz)) {
        const float aa = __ldg(p.azh + hz + TAB_OFF);
        if (aa != 0.f) {
          // psi' = b psi + a g, then p = g + psi': the same operations, in the same
          // order, as the owner's update, so a half row computed here as halo and by
          // its owner tile agrees bit for bit (whatever the tile height)
          const float bb = __ldg(p.bzh + hz + TAB_OFF);
          const float4 po = *reinterpret_cast<const float4*>(p.psiz_in + base + (long long)hz * pitch + xc);
          pp[0] += fmaf(aa, pp[0], bb * po.x); pp[1] += fmaf(aa, pp[1], bb * po.y);
          pp[2] += fmaf(aa, pp[2], bb * po.z); pp[3] += fmaf(aa, pp[3], bb * po.w);
        }
      }
      const float4 ma = ld4(sm + hr * MW + 4 * c + 4), mb = ld4(sm + (hr + 1) * MW + 4 * c + 4);
      const bool hv = hz >= 0 && hz < g.Nz - 1;
      const float q0 = (hv && xc + 0 < g.Nx) ? (LAP ? pp[0] : (ma.x + mb.x) * pp[0]) : 0.f;
      const float q1 = (hv && xc + 1 < g.Nx) ? (LAP ? pp[1] : (ma.y + mb.y) * pp[1]) : 0.f;
      const float q2 = (hv && xc + 2 < g.Nx) ? (LAP ? pp[2] : (ma.z + mb.z) * pp[2]) : 0.f;
      const float q3 = (hv && xc + 3 < g.Nx) ? (LAP ? pp[3] : (ma.w + mb.w) * pp[3]) : 0.f;
      st4(sh.qz + hr * TILE_X + 4 * c, make_float4(q0, q1, q2, q3));
    };

    qx_item(2 * ty, tx + 1, true);
    qx_item(2 * ty + 1, tx + 1, true);
    {
      // own z fluxes at half rows 2ty, 2ty+1 (tile-local) from a (2N+1)-row window
      float4 w[2 * N + 1];
#pragma unroll
      for (int t2 = 0; t2 <= 2 * N; t2++) w[t2] = ld4(su + (2 * ty + H - N + 1 + t2) * UW + 8 + 4 * tx);
      float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0;
#pragma unroll
      for (int k = 1; k <= N; k++) {
        acc4(a0, cf.c1z[k - 1], w[k + N - 1], w[N - k]);
        acc4(a1, cf.c1z[k - 1], w[k + N], w[N - k + 1]);
      }
      float pp[2][4];
      f4a(a0, pp[0]);
      f4a(a1, pp[1]);
#pragma unroll
      for (int rr = 0; rr < 2; rr++) {
        const int hz = zr0 + rr;
        const long long idz = base + (long long)hz * pitch + xb;
        if (pmlz && layer_h(hz, hz, g.npml, g.nz)) {
          const float aa = __ldg(p.azh + hz + TAB_OFF);
          if (aa != 0.f) {
            const float bb = __ldg(p.bzh + hz + TAB_OFF);
            const float4 po = *reinterpret_cast<const float4*>(p.psiz_in + idz);
            float4 pn;  // the operations of the halo items' update, in the same order
            pn.x = fmaf(aa, pp[rr][0], bb * po.x); pn.y = fmaf(aa, pp[rr][1], bb * po.y);
            pn.z = fmaf(aa, pp[rr][2], bb * po.z); pn.w = fmaf(aa, pp[rr][3], bb * po.w);
            if (xb + 0 >= g.Nx) pn.x = 0.f;
            if (xb + 1 >= g.Nx) pn.y = 0.f;
            if (xb + 2 >= g.Nx) pn.z = 0.f;
            if (xb + 3 >= g.Nx) pn.w = 0.f;
            st4(p.psiz_out + idz, pn);
            pp[rr][0] += pn.x; pp[rr][1] += pn.y; pp[rr][2] += pn.z; pp[rr][3] += pn.w;
          }
        }
        const float4 ma = ld4(sm + (2 * ty + 4 + rr) * MW + 4 * tx + 4);
        const float4 mb = ld4(sm + (2 * ty + 5 + rr) * MW + 4 * tx + 4);
        const bool hv = hz < g.Nz - 1;
        float q[4];
        q[0] = (hv && xb + 0 < g.Nx) ? (LAP ? pp[rr][0] : (ma.x + mb.x) * pp[rr][0]) : 0.f;
        q[1] = (hv && xb + 1 < g.Nx) ? (LAP ? pp[rr][1] : (ma.y + mb.y) * pp[rr][1]) : 0.f;
        q[2] = (hv && xb + 2 < g.Nx) ? (LAP ? pp[rr][2] : (ma.z + mb.z) * pp[rr][2]) : 0.f;
        q[3] = (hv && xb + 3 < g.Nx) ? (LAP ? pp[rr][3] : (ma.w + mb.w) * pp[rr][3]) : 0.f;
        st4(sh.qz + (2 * ty + 4 + rr) * TILE_X + 4 * tx, make_float4(q[0], q[1], q[2], q[3]));
        if (STORE && !LAP && (!MULTI || p.slot_pz))
          st4_stream(p.slot_pz + idz, hz < g.Nz ? make_float4(pp[rr][0], pp[rr][1], pp[rr][2], pp[rr][3])
                                                : make_float4(0.f, 0.f, 0.f, 0.f), pol);
      }
    }
    if (tid < 128) {  // the 8 halo half rows, 16 items each
      const int hr0 = tid >> 4;
      qz_item(hr0 < 4 ? hr0 : hr0 + TZ, tid & 15);
    } else if (tid < 128 + 2 * TZ) {  // the two halo column groups of every row
      const int k = tid - 128;
      qx_item(k >> 1, (k & 1) ? QXW / 4 - 1 : 0, false);
    }
    // u^n at the own cells (and, for the Laplacian operator, m/2 there), read
    // before the operand buffer is refilled
    float4 ucur[2], mown[2];
    ucur[0] = ld4(su + (2 * ty + H) * UW + 4 * tx + H);
    ucur[1] = ld4(su + (2 * ty + 1 + H) * UW + 4 * tx + H);
    if (LAP) {
      mown[0] = ld4(sm + (2 * ty + 4) * MW + 4 * tx + 4);
      mown[1] = ld4(sm + (2 * ty + 5) * MW + 4 * tx + 4);
    }
    __syncthreads();
    if (tid == 0 && tn < ntiles) fetch_next(tn);

    // ---- stage 2: divergence + CPML zeta + leapfrog + source + receivers
    cp_async_wait_all();  // this thread's own u^{n-1} copies
    float hzv[2][4];
    {
      float4 w[2 * N + 1];
#pragma unroll
      for (int t2 = 0; t2 <= 2 * N; t2++) w[t2] = ld4(sh.qz + (2 * ty + 4 - N + t2) * TILE_X + 4 * tx);
      float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0;
#pragma unroll
      for (int k = 1; k <= N; k++) {
        acc4(a0, cf.c2z[k - 1], w[k + N - 1], w[N - k]);
        acc4(a1, cf.c2z[k - 1], w[k + N], w[N - k + 1]);
      }
      f4a(a0, hzv[0]);
      f4a(a1, hzv[1]);
    }
    const int i0 = box.x, j0 = box.y, nb = p.src_n;
    const bool srcbox = i0 >= 0 && i0 < z0 + TZ && i0 + nb > z0 && j0 < x0 + TILE_X && j0 + nb > x0;
    float4 ax4 = make_float4(0.f, 0.f, 0.f, 0.f), bx4 = ax4;
    if (pmlx && layer_c(xb, xb + 3, g.npml, g.nx)) ax4 = ldg4(p.ax + xb + TAB_OFF);
    const bool zx_on = ax4.x != 0.f || ax4.y != 0.f || ax4.z != 0.f || ax4.w != 0.f;
    if (zx_on) bx4 = ldg4(p.bx + xb + TAB_OFF);
    float un[2][4];
#pragma unroll
    for (int rr = 0; rr < 2; rr++) {
      const int r = 2 * ty + rr, z = z0 + r;
      const long long idc0 = base + (long long)z * pitch + xb;
      float v[12];
      unpack12(sh.qx + r * QXW + 4 * tx, v);
      float hxv[4], rv[4];
#pragma unroll
      for (int e = 0; e < 4; e++) {
        float hx = 0.f;
#pragma unroll
        for (int k = 1; k <= N; k++) hx += cf.c2x[k - 1] * (v[e + k + 3] - v[e - k + 4]);
        hxv[e] = hx;
        rv[e] = hx + hzv[rr][e];
      }
      // CPML zeta (dt^2-scaled) <- b zeta + a h; it stays zero where a = 0 and
      // outside the grid (h = 0 there), so whole float4 groups are written
      if (zx_on) {
        const float4 zo = ld4(p.zetx + idc0);
        float4 zn;
        zn.x = bx4.x * zo.x + ax4.x * hxv[0]; zn.y = bx4.y * zo.y + ax4.y * hxv[1];
        zn.z = bx4.z * zo.z + ax4.z * hxv[2]; zn.w = bx4.w * zo.w + ax4.w * hxv[3];
        st4(p.zetx + idc0, zn);
        rv[0] += zn.x; rv[1] += zn.y; rv[2] += zn.z; rv[3] += zn.w;
      }
      if (pmlz && layer_c(z, z, g.npml, g.nz)) {
        const float aa = __ldg(p.az + z + TAB_OFF);
        if (aa != 0.f) {
          const float bb = __ldg(p.bz + z + TAB_OFF);
          const float4 zo = ld4(p.zetz + idc0);
          float4 zn;
          zn.x = bb * zo.x + aa * hzv[rr][0]; zn.y = bb * zo.y + aa * hzv[rr][1];
          zn.z = bb * zo.z + aa * hzv[rr][2]; zn.w = bb * zo.w + aa * hzv[rr][3];
          st4(p.zetz + idc0, zn);
          rv[0] += zn.x; rv[1] += zn.y; rv[2] += zn.z; rv[3] += zn.w;
        }
      }
      const float4 uc = ucur[rr];
      const float4 upv = sh.up4[rr * NT + tid];
      if (LAP) {
        // r^n (dt^2-scaled) is the gradient operand; the update takes m r, m = 2 (m/2)
        if (STORE) {
          float r4[4];
#pragma unroll
          for (int e = 0; e < 4; e++) r4[e] = (z < g.Nz && xb + e < g.Nx) ? rv[e] : 0.f;  // zero off the grid
          st4_stream(p.slot_px + idc0, make_float4(r4[0], r4[1], r4[2], r4[3]), pol);
        }
        rv[0] *= 2.f * mown[rr].x;
        rv[1] *= 2.f * mown[rr].y;
        rv[2] *= 2.f * mown[rr].z;
        rv[3] *= 2.f * mown[rr].w;
      }
      un[rr][0] = 2.f * uc.x - upv.x + rv[0];
      un[rr][1] = 2.f * uc.y - upv.y + rv[1];
      un[rr][2] = 2.f * uc.z - upv.z + rv[2];
      un[rr][3] = 2.f * uc.w - upv.w + rv[3];
      if (srcbox) {
        const int di = z - i0;
        if (di >= 0 && di < nb) {
          const float amp = cf.dt2 * stf_n;
#pragma unroll
          for (int e = 0; e < 4; e++) {
            const int dj = xb + e - j0;
            if (dj >= 0 && dj < nb) un[rr][e] += amp * p.src_w[s * SRC_W * SRC_W + di * SRC_W + dj];
          }
        }
      }
#pragma unroll
      for (int e = 0; e < 4; e++)
        if (!(z < g.Nz && xb + e < g.Nx)) un[rr][e] = 0.f;
      st4(uprev + (long long)z * pitch + xb, make_float4(un[rr][0], un[rr][1], un[rr][2], un[rr][3]));
    }
    if (RECORD) {
      // receivers of this thread's 2 x 4 cells: (index << 3) | (row << 2) | column
      for (int q = rb; q < re; q++) {
        const int code = p.thr_rec[q];
        const int rc = code >> 3, rr = (code >> 2) & 1, e = code & 3;
        const float* ur = un[rr];
        p.seis[((long long)s * p.nrec + rc) * p.nt + p.n] = e == 0 ? ur[0] : (e == 1 ? ur[1] : (e == 2 ? ur[2] : ur[3]));
      }
    }
    __syncthreads();  // the flux arrays are free again
  }
}

// ---------------------------------------------------------------------------
// Adjoint step n (reverse of forward step n, statement by statement; Z is kept
// divided by dt^2):
//   hhat = lambda_{n+1} + a (Z + lambda_{n+1}),  Z <- b (Z + lambda_{n+1})
//   qbar = -dt^2 D+ hhat                         (= D-^T applied to dt^2 hhat)
//   2 dJ/dm += qbar * p^n at both neighbours of each half point (gradient correlation)
//   pbar = m_half qbar;  gbar = pbar + a_h (P + pbar),  P <- b_h (P + pbar)
//   lambda_n = 2 lambda_{n+1} - lambda_{n+2} - D- gbar + residual(sample n-1)
// hhat is needed with an N-cell halo, so the step that produces lambda_{n+1}
// also leaves hhat behind: every tile within one tile of a CPML tile writes
// Hx = (1 + a_x) lambda + a_x Zx and Hz likewise at its own cells, and a CPML
// tile fetches its x (z) stencil operand from Hx (Hz) instead of lambda. Z is
// then read and written only by the thread that owns the cell.
// MULTI: one launch over the tiles of several instances, as for the forward step.
// LAP: the adjoint of the c^2 Laplacian step: rbar = dt^2 m lambda_{n+1}, so
// m lambda takes lambda's place in Z and hhat (written by every tile, and every
// tile fetches its operands from Hx and Hz), pbar = qbar (no half-point
// coefficient), and the gradient correlation is 2 dJ/dm += 2 lambda_{n+1} r^n at
// the cells, with r^n (dt^2-scaled) stored by the forward step.
template <int N, bool MULTI, bool LAP = false>
__global__ void __launch_bounds__(NTHREADS, 3)
    acu_adj_step(const __grid_constant__ CUtensorMap tmap_lx, const __grid_constant__ CUtensorMap tmap_lz,
                 const __grid_constant__ CUtensorMap tmap_hx, const __grid_constant__ CUtensorMap tmap_hz,
                 const __grid_constant__ CUtensorMap tmap_m, const __grid_constant__ AcuStep p0, const AcuCoef cf,
                 const BatchArgs b) {
  static_assert(!LAP || !MULTI, "the Laplacian operator runs on single-instance launches");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  AdjSmem& sh = *reinterpret_cast<AdjSmem*>(smem_raw);
  AcuStep& shp = *reinterpret_cast<AcuStep*>(smem_raw + ADJ_SMEM_MAIN);  // MULTI only
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const uint64_t pol = l2_evict_first();  // the stored fluxes are read once: evict them first
  const int ntiles = MULTI ? b.ntiles : p0.ntiles;

  // one operand buffer: the next tile's fetch is issued once stage 1 of this
  // tile (its last reader) is done, and overlaps stage 2
  auto fetch = [&](int tt) {
    const CUtensorMap *mlx = &tmap_lx, *mlz = &tmap_lz, *mhx = &tmap_hx, *mhz = &tmap_hz, *mm = &tmap_m;
    Grid gf = p0.g;
    int plane0 = p0.cur * p0.S_pair + p0.s0, tl = tt;
    if (MULTI) {
      const int i = batch_instance(b, tt);
      const AcuInst* in = b.inst + i;
      gf = in->p.g;
      plane0 = ((b.n + 1) & 1) * in->p.S;
      tl = tt - __ldg(b.tile_start + i);
      mlx = &in->lx;
      mlz = &in->lz;
      mhx = &in->hx;
      mhz = &in->hz;
      mm = &in->mm;
    }
    const TileId f = tile_decode(gf, tl);
    const int plane = plane0 + f.s;
    const CUtensorMap* xm = (LAP || tile_pml_x(gf, f.x0)) ? mhx : mlx;
    const CUtensorMap* zm = (LAP || tile_pml_z(gf, f.z0)) ? mhz : mlz;
    if (MULTI) {
      tensormap_acquire(xm);
      tensormap_acquire(zm);
      tensormap_acquire(mm);
    }
    fence_proxy_async();
    mbar_expect_tx(&sh.bar, XS_BYTES + ZS_BYTES + M_BYTES);
    tma_3d(sh.xs, xm, f.x0 - H + APRON, f.z0 + APRON, plane, &sh.bar);
    tma_3d(sh.zs, zm, f.x0 + APRON, f.z0 - H + APRON, plane, &sh.bar);
    tma_2d(sh.m, mm, f.x0 - 4 + APRON, f.z0 - 4 + APRON, &sh.bar);
  };

  if (tid == 0) {
    mbar_init(&sh.bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0 && (int)blockIdx.x < ntiles) fetch(blockIdx.x);

  int it = 0, inst_loaded = -1;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x, it++) {
    const int tn = t + gridDim.x;
    int tl = t;  // tile index within its instance
    if (MULTI) {
      const int i = batch_instance(b, t);
      tl = t - __ldg(b.tile_start + i);
      if (i != inst_loaded) {  // the parameters stay in shared memory while the instance does not change
        batch_load_step<2>(b, i, shp);  // after the previous tile's closing barrier
        inst_loaded = i;
      }
    }
    const AcuStep& p = MULTI ? shp : p0;
    const Grid& g = p.g;
    const int pitch = g.pitch;
    const TileId id = tile_decode(g, tl);
    const int x0 = id.x0, z0 = id.z0, s = id.s;
    const long long base = (long long)s * g.slice + g.off0;
    const int xb = x0 + 4 * tx, zr0 = z0 + 2 * ty;
    // stored fluxes p^n of this thread's own half points (x and z), fetched before the wait
    float4 pfx[2], pfz[2];
    // (LAP: pfx holds r^n of the own cells and pfz is not used)
    pfx[0] = ld4_stream(p.slot_px + base + (long long)zr0 * pitch + xb, pol);
    pfx[1] = ld4_stream(p.slot_px + base + (long long)(zr0 + 1) * pitch + xb, pol);
    if (!LAP) {
      pfz[0] = ld4_stream(p.slot_pz + base + (long long)zr0 * pitch + xb, pol);
      pfz[1] = ld4_stream(p.slot_pz + base + (long long)(zr0 + 1) * pitch + xb, pol);
    } else {
      pfz[0] = pfz[1] = make_float4(0.f, 0.f, 0.f, 0.f);
    }

    const bool ok = mbar_wait(&sh.bar, it & 1);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicOr(p.status, ST_TIMEOUT);
        mbar_wait(&sh.bar, it & 1);  // let a late copy land before the CTA exits
      }
      return;
    }
    // the tile body, compiled twice: with the grid-edge masks, and without them for
    // tiles whose stencils and halo stay strictly inside the padded grid
    auto tile_body = [&](auto edge_c) {
      constexpr bool EDGE = decltype(edge_c)::value;
      const float* sx = sh.xs;  // [TILE_Z][UW]: x operand, cols [x0-H, x0+TX+H)
      const float* sz = sh.zs;  // [UH][TILE_X]: z operand, rows [z0-H, z0+TZ+H)
      const float* sm = sh.m;
      const bool pmlx = tile_pml_x(g, x0), pmlz = tile_pml_z(g, z0);

      // ---- stage 1a: x half points of row r: qbar, correlation, gbar
      auto x_item = [&](int r, int gq, bool own, bool image, const float4* pre, float im[4]) {
        const int z = z0 + r, hb = x0 - 4 + 4 * gq;
        float v[12];
        unpack12(sx + r * UW + 4 * gq, v);
        const long long id0 = base + (long long)z * pitch + hb;
        const float4 m4 = ld4(sm + (r + 4) * MW + 4 * gq);
        const float mv[5] = {m4.x, m4.y, m4.z, m4.w, sm[(r + 4) * MW + 4 * gq + 4]};
        float pf[4] = {0.f, 0.f, 0.f, 0.f};
        if (!LAP && pre) f4a(*pre, pf);
        else if (!LAP && image && (!EDGE || hb >= 0)) f4a(ld4_stream(p.slot_px + id0, pol), pf);  // the apron holds no flux
        const bool rowok = !EDGE || z < g.Nz;
        float4 a4 = make_float4(0.f, 0.f, 0.f, 0.f), b4 = a4, P4 = a4;
        if (pmlx && layer_h(hb, hb + 3, g.npml, g.nx)) {  // one round trip: tables and P together
          a4 = ldg4(p.axh + hb + TAB_OFF);
          b4 = ldg4(p.bxh + hb + TAB_OFF);
          P4 = ld4(p.px_in + id0);
        }
        float av[4], bv[4], Pv[4];
        f4a(a4, av);
        f4a(b4, bv);
        f4a(P4, Pv);
        float gb[4], Pn[4];
  #pragma unroll
        for (int e = 0; e < 4; e++) {
          float dq = 0.f;
  #pragma unroll
          for (int k = 1; k <= N; k++) dq += cf.c1x[k - 1] * (v[e + 4 + k] - v[e + 5 - k]);
          const bool inh = !EDGE || (rowok && hb + e >= 0 && hb + e < g.Nx - 1);
          const float qb = inh ? dq : 0.f;
          const float pb = LAP ? qb : (mv[e] + mv[e + 1]) * qb;
          const float tt = Pv[e] + pb;
          gb[e] = inh ? pb + av[e] * tt : 0.f;
          Pn[e] = av[e] != 0.f ? bv[e] * tt : 0.f;  // P stays zero outside the layer
          im[e] = LAP ? 0.f : qb * pf[e];
        }
        if (pmlx && own && rowok && (av[0] != 0.f || av[1] != 0.f || av[2] != 0.f || av[3] != 0.f))
          st4(p.px_out + id0, make_float4(Pn[0], Pn[1], Pn[2], Pn[3]));
        st4(sh.gx + r * QXW + 4 * gq, make_float4(gb[0], gb[1], gb[2], gb[3]));
      };
      // ---- stage 1b: one z half row (the tile's halo rows)
      auto z_item = [&](int hr, int c, bool image) {
        const int hz = z0 - 4 + hr, xc = x0 + 4 * c;
        const long long idz = base + (long long)hz * pitch + xc;
        float pf[4] = {0.f, 0.f, 0.f, 0.f};
        if (!LAP && image && (!EDGE || hz >= 0)) f4a(ld4_stream(p.slot_pz + idz, pol), pf);
        float aa = 0.f;
        float Pv[4] = {0.f, 0.f, 0.f, 0.f};
        if (pmlz && layer_h(hz, hz, g.npml, g.nz)) {
          aa = __ldg(p.azh + hz + TAB_OFF);
          f4a(*reinterpret_cast<const float4*>(p.pz_in + idz), Pv);
        }
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  #pragma unroll
        for (int k = 1; k <= N; k++)
          acc4(acc, cf.c1z[k - 1], ld4(sz + (hr + 4 + k) * TILE_X + 4 * c), ld4(sz + (hr + 5 - k) * TILE_X + 4 * c));
        float dq[4];
        f4a(acc, dq);
        const bool hv = !EDGE || (hz >= 0 && hz < g.Nz - 1);
        const float4 ma = ld4(sm + hr * MW + 4 * c + 4), mb = ld4(sm + (hr + 1) * MW + 4 * c + 4);
        const float mhv[4] = {ma.x + mb.x, ma.y + mb.y, ma.z + mb.z, ma.w + mb.w};
        float gb[4], im[4];
  #pragma unroll
        for (int e = 0; e < 4; e++) {
          const bool inh = !EDGE || (hv && xc + e < g.Nx);
          const float qb = inh ? dq[e] : 0.f;
          const float pb = LAP ? qb : mhv[e] * qb;
          gb[e] = inh ? pb + aa * (Pv[e] + pb) : 0.f;
          im[e] = LAP ? 0.f : qb * pf[e];
        }
        st4(sh.gz + hr * TILE_X + 4 * c, make_float4(gb[0], gb[1], gb[2], gb[3]));
        if (image) st4(sh.imz + 4 * c, make_float4(im[0], im[1], im[2], im[3]));
      };

      // own x half points xb+e+1/2 of rows 2ty, 2ty+1: their images stay in registers
      float imx[2][4], imz[2][4];
      x_item(2 * ty, tx + 1, true, true, &pfx[0], imx[0]);
      x_item(2 * ty + 1, tx + 1, true, true, &pfx[1], imx[1]);
      {
        // own z half rows 2ty, 2ty+1 from a (2N+1)-row window of hhat
        float aa[2] = {0.f, 0.f}, bb[2] = {1.f, 1.f};
        float4 Pz[2] = {make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f)};
        if (pmlz && layer_h(zr0, zr0 + 1, g.npml, g.nz)) {
  #pragma unroll
          for (int rr = 0; rr < 2; rr++) {
            aa[rr] = __ldg(p.azh + zr0 + rr + TAB_OFF);
            bb[rr] = __ldg(p.bzh + zr0 + rr + TAB_OFF);
            Pz[rr] = *reinterpret_cast<const float4*>(p.pz_in + base + (long long)(zr0 + rr) * pitch + xb);
          }
        }
        float4 w[2 * N + 1];
  #pragma unroll
        for (int t2 = 0; t2 <= 2 * N; t2++) w[t2] = ld4(sz + (2 * ty + H - N + 1 + t2) * TILE_X + 4 * tx);
        float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0;
  #pragma unroll
        for (int k = 1; k <= N; k++) {
          acc4(a0, cf.c1z[k - 1], w[k + N - 1], w[N - k]);
          acc4(a1, cf.c1z[k - 1], w[k + N], w[N - k + 1]);
        }
        float dq[2][4];
        f4a(a0, dq[0]);
        f4a(a1, dq[1]);
  #pragma unroll
        for (int rr = 0; rr < 2; rr++) {
          const int hz = zr0 + rr;
          const long long idz = base + (long long)hz * pitch + xb;
          const bool hv = !EDGE || hz < g.Nz - 1;
          const float4 ma = ld4(sm + (2 * ty + 4 + rr) * MW + 4 * tx + 4);
          const float4 mb = ld4(sm + (2 * ty + 5 + rr) * MW + 4 * tx + 4);
          const float mhv[4] = {ma.x + mb.x, ma.y + mb.y, ma.z + mb.z, ma.w + mb.w};
          float pf[4], Pv[4];
          f4a(pfz[rr], pf);
          f4a(Pz[rr], Pv);
          float gb[4], Pn[4];
  #pragma unroll
          for (int e = 0; e < 4; e++) {
            const bool inh = !EDGE || (hv && xb + e < g.Nx);
            const float qb = inh ? dq[rr][e] : 0.f;
            const float pb = LAP ? qb : mhv[e] * qb;
            const float tt = Pv[e] + pb;
            gb[e] = inh ? pb + aa[rr] * tt : 0.f;
            Pn[e] = inh ? bb[rr] * tt : 0.f;
            imz[rr][e] = LAP ? 0.f : qb * pf[e];
          }
          if (aa[rr] != 0.f && (!EDGE || hz < g.Nz)) st4(p.pz_out + idz, make_float4(Pn[0], Pn[1], Pn[2], Pn[3]));
          st4(sh.gz + (2 * ty + 4 + rr) * TILE_X + 4 * tx, make_float4(gb[0], gb[1], gb[2], gb[3]));
        }
        // half row 2ty+1 is the upper neighbour of the next thread row's cells
        st4(sh.imz + (ty + 1) * TILE_X + 4 * tx, make_float4(imz[1][0], imz[1][1], imz[1][2], imz[1][3]));
      }
      if (tid < 128) {
        const int hr0 = tid >> 4;
        const int hr = hr0 < 4 ? hr0 : hr0 + 32;
        z_item(hr, tid & 15, hr == 3);  // of the halo rows only half row z0-1 feeds this tile's gradient
      } else if (tid < 192) {
        const int k = tid - 128;
        const bool left = (k & 1) == 0;
        float im[4];
        x_item(k >> 1, left ? 0 : QXW / 4 - 1, false, left, nullptr, im);  // only half column x0-1 feeds the gradient
        if (left) sh.imx[k >> 1] = im[3];
      }
      // lambda_{n+1} at the own cells, from a stencil tile that holds lambda itself
      // (the Laplacian operator's tiles hold m lambda: lambda from memory, m = 2 (m/2)
      // of the own cells from the coefficient tile)
      float4 lc[2], m2[2];
  #pragma unroll
      for (int rr = 0; rr < 2; rr++) {
        const int r = 2 * ty + rr;
        if (!LAP && !pmlx) lc[rr] = ld4(sx + r * UW + H + 4 * tx);
        else if (!LAP && !pmlz) lc[rr] = ld4(sz + (r + H) * TILE_X + 4 * tx);
        else lc[rr] = ldg4(p.lam + (long long)(p.cur * p.S_pair + p.s0) * g.slice + base + (long long)(z0 + r) * pitch + xb);
        if (LAP) {
          const float4 mh = ld4(sm + (r + 4) * MW + 4 * tx + 4);
          m2[rr] = make_float4(2.f * mh.x, 2.f * mh.y, 2.f * mh.z, 2.f * mh.w);
        }
      }
      // lambda_{n+2} and the gradient partial of the own cells: issued before the
      // barrier, so that their latency overlaps the other warps' halo items
      float* __restrict__ lprev = p.lam + (long long)((p.cur ^ 1) * p.S_pair + p.s0) * g.slice + base;
      float* __restrict__ gp = p.gpart + base;
      float4 lo[2], go[2];
      lo[0] = ldg4(lprev + (long long)zr0 * pitch + xb);
      lo[1] = ldg4(lprev + (long long)(zr0 + 1) * pitch + xb);
      go[0] = ldg4(gp + (long long)zr0 * pitch + xb);
      go[1] = ldg4(gp + (long long)(zr0 + 1) * pitch + xb);
      __syncthreads();
      if (tid == 0 && tn < ntiles) fetch(tn);  // the operand buffer is free

      // ---- stage 2: lambda_n, gradient, residual, Z update, hhat for step n-1, source partials
      const int2 box = __ldg(reinterpret_cast<const int2*>(p.src_box) + s);
      const int key = (id.tz * g.ntx + id.tx) * NTHREADS + tid;
      const int rb = __ldg(p.thr_rec_start + key), re = __ldg(p.thr_rec_start + key + 1);
      float dzv[2][4];
      {
        float4 w[2 * N + 1];
  #pragma unroll
        for (int t2 = 0; t2 <= 2 * N; t2++) w[t2] = ld4(sh.gz + (2 * ty + 4 - N + t2) * TILE_X + 4 * tx);
        float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0;
  #pragma unroll
        for (int k = 1; k <= N; k++) {
          acc4(a0, cf.c2z[k - 1], w[k + N - 1], w[N - k]);
          acc4(a1, cf.c2z[k - 1], w[k + N], w[N - k + 1]);
        }
        f4a(a0, dzv[0]);
        f4a(a1, dzv[1]);
      }
      // image of the half row above (2ty-1) and of the half column left of the thread (xb-1/2)
      float imzu[4] = {0.f, 0.f, 0.f, 0.f};
      float imxl[2] = {0.f, 0.f};
      if (!LAP) {
        f4a(ld4(sh.imz + ty * TILE_X + 4 * tx), imzu);
  #pragma unroll
        for (int rr = 0; rr < 2; rr++) {
          const float up = __shfl_up_sync(0xffffffffu, imx[rr][3], 1, 16);
          imxl[rr] = tx == 0 ? sh.imx[2 * ty + rr] : up;
        }
      }
      float lnew[2][4];
  #pragma unroll
      for (int rr = 0; rr < 2; rr++) {
        const int r = 2 * ty + rr, z = z0 + r;
        float v[12];
        unpack12(sh.gx + r * QXW + 4 * tx, v);
        float lcv[4], lov[4], gov[4];
        f4a(lc[rr], lcv);
        f4a(lo[rr], lov);
        f4a(go[rr], gov);
        float gn[4];
  #pragma unroll
        for (int e = 0; e < 4; e++) {
          float dxv = 0.f;
  #pragma unroll
          for (int k = 1; k <= N; k++) dxv += cf.c2x[k - 1] * (v[e + k + 3] - v[e - k + 4]);
          const bool valid = !EDGE || (z < g.Nz && xb + e < g.Nx);
          lnew[rr][e] = valid ? 2.f * lcv[e] - lov[e] - (dxv + dzv[rr][e]) : 0.f;
          const float ixl = e == 0 ? imxl[rr] : imx[rr][e - 1];
          const float izu = rr == 0 ? imzu[e] : imz[0][e];
          float rst[4];
          f4a(pfx[rr], rst);
          // divergence form: the four half-point images; Laplacian: 2 lambda_{n+1} r^n at the cell
          const float inc = LAP ? 2.f * lcv[e] * rst[e] : (ixl + imx[rr][e] + izu + imz[rr][e]);
          gn[e] = valid ? gov[e] + inc : 0.f;
        }
        st4(gp + (long long)z * pitch + xb, make_float4(gn[0], gn[1], gn[2], gn[3]));
      }
      if (p.n >= 1) {
        // residual of the sample recorded from u^n (sample n-1) at this thread's receivers
        for (int q = rb; q < re; q++) {
          const int code = p.thr_rec[q];
          const int rc = code >> 3, rr = (code >> 2) & 1, e = code & 3;
          const float rv = p.res[((long long)s * p.nrec + rc) * p.nt + p.n - 1];
  #pragma unroll
          for (int r2 = 0; r2 < 2; r2++)
  #pragma unroll
            for (int e2 = 0; e2 < 4; e2++)
              if (r2 == rr && e2 == e) lnew[r2][e2] += rv;
        }
      }
      const bool wx = LAP || tile_writes_hx(g, id.tx), wz = LAP || tile_writes_hz(g, id.tz);
      float4 ax4 = make_float4(0.f, 0.f, 0.f, 0.f), bx4 = ax4;
      if (pmlx && layer_c(xb, xb + 3, g.npml, g.nx)) {
        ax4 = ldg4(p.ax + xb + TAB_OFF);
        bx4 = ldg4(p.bx + xb + TAB_OFF);
      }
      const bool zx_on = ax4.x != 0.f || ax4.y != 0.f || ax4.z != 0.f || ax4.w != 0.f;
  #pragma unroll
      for (int rr = 0; rr < 2; rr++) {
        const int z = zr0 + rr;
        const long long idc0 = base + (long long)z * pitch + xb;
        const float4 l4 = make_float4(lnew[rr][0], lnew[rr][1], lnew[rr][2], lnew[rr][3]);
        st4(lprev + (long long)z * pitch + xb, l4);
        // what rbar / dt^2 is made of: lambda (divergence form) or m lambda (Laplacian)
        const float4 lcm = LAP ? make_float4(m2[rr].x * lc[rr].x, m2[rr].y * lc[rr].y, m2[rr].z * lc[rr].z,
                                             m2[rr].w * lc[rr].w)
                               : lc[rr];
        const float4 l4m = LAP ? make_float4(m2[rr].x * l4.x, m2[rr].y * l4.y, m2[rr].z * l4.z, m2[rr].w * l4.w) : l4;
        // CPML Z (divided by dt^2) <- b (Z + lambda_{n+1}); zero outside the layer and the grid
        float4 Zx = make_float4(0.f, 0.f, 0.f, 0.f), Zz = Zx;
        if (zx_on) {
          const float4 Zo = ld4(p.zx_in + idc0);
          Zx.x = ax4.x != 0.f && (!EDGE || z < g.Nz) ? bx4.x * (Zo.x + lcm.x) : 0.f;
          Zx.y = ax4.y != 0.f && (!EDGE || z < g.Nz) ? bx4.y * (Zo.y + lcm.y) : 0.f;
          Zx.z = ax4.z != 0.f && (!EDGE || z < g.Nz) ? bx4.z * (Zo.z + lcm.z) : 0.f;
          Zx.w = ax4.w != 0.f && (!EDGE || z < g.Nz) ? bx4.w * (Zo.w + lcm.w) : 0.f;
          st4(p.zx_out + idc0, Zx);
        }
        float az = 0.f;
        if (pmlz && layer_c(z, z, g.npml, g.nz)) {
          az = __ldg(p.az + z + TAB_OFF);
          if (az != 0.f) {
            const float bz = __ldg(p.bz + z + TAB_OFF);
            const float4 Zo = ld4(p.zz_in + idc0);
            Zz.x = (!EDGE || xb + 0 < g.Nx) ? bz * (Zo.x + lcm.x) : 0.f;
            Zz.y = (!EDGE || xb + 1 < g.Nx) ? bz * (Zo.y + lcm.y) : 0.f;
            Zz.z = (!EDGE || xb + 2 < g.Nx) ? bz * (Zo.z + lcm.z) : 0.f;
            Zz.w = (!EDGE || xb + 3 < g.Nx) ? bz * (Zo.w + lcm.w) : 0.f;
            st4(p.zz_out + idc0, Zz);
          }
        }
        // hhat of step n-1 (lambda_n, or m lambda_n, with the updated Z); equal to that outside the layer
        if (wx)
          st4(p.hx_out + idc0, make_float4(l4m.x + ax4.x * (Zx.x + l4m.x), l4m.y + ax4.y * (Zx.y + l4m.y),
                                           l4m.z + ax4.z * (Zx.z + l4m.z), l4m.w + ax4.w * (Zx.w + l4m.w)));
        if (wz)
          st4(p.hz_out + idc0, make_float4(l4m.x + az * (Zz.x + l4m.x), l4m.y + az * (Zz.y + l4m.y),
                                           l4m.z + az * (Zz.z + l4m.z), l4m.w + az * (Zz.w + l4m.w)));
      }
      // source-parameter partials from lambda_n (index n-1): sum w lambda,
      // sum w lambda (x_i - x0), sum w lambda (z_i - z0); at most 4 tiles touch a box
      if (p.src_part != nullptr && p.n >= 1) {
        const int i0 = box.x, j0 = box.y, nb = p.src_n;
        if (i0 >= 0 && i0 < z0 + TILE_Z && i0 + nb > z0 && j0 < x0 + TILE_X && j0 + nb > x0) {
          float acc[3] = {0.f, 0.f, 0.f};
          const float xs = p.x0[2 * s], zs = p.x0[2 * s + 1];
  #pragma unroll
          for (int rr = 0; rr < 2; rr++) {
            const int z = zr0 + rr, di = z - i0;
            if (di >= 0 && di < nb) {
  #pragma unroll
              for (int e = 0; e < 4; e++) {
                const int dj = xb + e - j0;
                if (dj >= 0 && dj < nb) {
                  const float wl = p.src_w[s * SRC_W * SRC_W + di * SRC_W + dj] * lnew[rr][e];
                  acc[0] += wl;
                  acc[1] += wl * ((float)(xb + e - g.npml) * p.dx - xs);
                  acc[2] += wl * ((float)(z - g.npml) * p.dz - zs);
                }
              }
            }
          }
          cta_sum3(acc, sh.red);
          if (tid == 0) {
            const int slot = 2 * (id.tz - i0 / TILE_Z) + (id.tx - j0 / TILE_X);
            float* dst = p.src_part + (((long long)s * p.nt + (p.n - 1)) * SRC_SLOTS + slot) * 3;
            dst[0] = acc[0];
            dst[1] = acc[1];
            dst[2] = acc[2];
          }
        }
      }
      __syncthreads();  // the stage arrays are free again
    };
    const bool edge = x0 < 4 || x0 + TILE_X + 5 > g.Nx || z0 < 4 || z0 + TILE_Z + 5 > g.Nz;
    if (edge) tile_body(std::true_type{});
    else tile_body(std::false_type{});
  }
}

// ---------------------------------------------------------------------------
// Self-test of the bounded wait: one thread waits, as a step kernel waits for
// its tile, on an mbarrier whose 16 expected bytes no copy will ever deliver.
__global__ void k_selftest_wait(int* status, unsigned long long* waited_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    mbar_expect_tx(&bar, 16);
    const unsigned long long t0 = global_ns();
    const bool ok = mbar_wait(&bar, 0);
    *waited_ns = global_ns() - t0;
    *status = ok ? 0 : ST_TIMEOUT;
  }
}

// ---------------------------------------------------------------------------
// Host side: tensor maps, one-time kernel attributes, launchers.
namespace {

std::mutex g_init_mu;
unsigned long long g_inited = 0;  // bit per device
// resident-CTA grids: single-instance forward variants (record, store), adjoint,
// and the multi-instance forward sweep / recompute and adjoint
int g_grid_fwd[64][2][4], g_grid_adj[64][2], g_grid_fwd_m[64][2][2], g_grid_adj_m[64][2];
int g_grid_fwd64[64][2][4];  // the 64-row forward variants
int g_grid_fwd_lap[64][2][4], g_grid_adj_lap[64][2];  // the c^2 Laplacian operator

template <typename K>
cudaError_t setup_kernel(K k, int smem, int* grid, int threads = NTHREADS) {
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0, nb = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, threads, smem)) != cudaSuccess) return e;
  *grid = (nb < 1 ? 1 : nb) * nsm;
  return cudaSuccess;
}

constexpr int FWD_SMEM_M = (int)(FWD_SMEM_MAIN + sizeof(AcuStep));
constexpr int ADJ_SMEM_M = (int)(ADJ_SMEM_MAIN + sizeof(AcuStep));

template <int N>
cudaError_t setup_order(int dev, int o) {
  const int fs = (int)sizeof(FwdSmem), as = (int)sizeof(AdjSmem), f64 = (int)sizeof(FwdSmemT<64>);
  constexpr int T64 = FwdGeo<64>::NT;
  cudaError_t e;
  if ((e = setup_kernel(acu_fwd_step<N, false, false, false, 32>, fs, &g_grid_fwd[dev][o][0])) != cudaSuccess) return e;
  if ((e = setup_kernel(acu_fwd_step<N, true, false, false, 32>, fs, &g_grid_fwd[dev][o][1])) != cudaSuccess) return e;
  if ((e = setup_kernel(acu_fwd_step<N, false, true, false, 32>, fs, &g_grid_fwd[dev][o][2])) != cudaSuccess) return e;
  if ((e = setup_kernel(acu_fwd_step<N, true, true, false, 32>, fs, &g_grid_fwd[dev][o][3])) != cudaSuccess) return e;
  if ((e = setup_kernel(acu_fwd_step<N, false, false, false, 64>, f64, &g_grid_fwd64[dev][o][0], T64)) != cudaSuccess)
    return e;
  if ((e = setup_kernel(acu_fwd_step<N, true, false, false, 64>, f64, &g_grid_fwd64[dev][o][1], T64)) != cudaSuccess)
    return e;
  if ((e = setup_kernel(acu_fwd_step<N, false, true, false, 64>, f64, &g_grid_fwd64[dev][o][2], T64)) != cudaSuccess)
    return e;
  if ((e = setup_kernel(acu_fwd_step<N, true, true, false, 64>, f64, &g_grid_fwd64[dev][o][3], T64)) != cudaSuccess)
    return e;
  if ((e = setup_kernel(acu_fwd_step<N, true, true, true, 32>, FWD_SMEM_M, &g_grid_fwd_m[dev][o][0])) != cudaSuccess)
    return e;
  if ((e = setup_kernel(acu_fwd_step<N, false, true, true, 32>, FWD_SMEM_M, &g_grid_fwd_m[dev][o][1])) != cudaSuccess)
    return e;
  if ((e = setup_kernel(acu_adj_step<N, false>, as, &g_grid_adj[dev][o])) != cudaSuccess) return e;
  if ((e = setup_kernel(acu_adj_step<N, false, true>, as, &g_grid_adj_lap[dev][o])) != cudaSuccess) return e;
  for (int v = 0; v < 4; v++) {
    auto k = v == 0 ? acu_fwd_step<N, false, false, false, 32, true> : v == 1 ? acu_fwd_step<N, true, false, false, 32, true>
           : v == 2 ? acu_fwd_step<N, false, true, false, 32, true> : acu_fwd_step<N, true, true, false, 32, true>;
    if ((e = setup_kernel(k, fs, &g_grid_fwd_lap[dev][o][v])) != cudaSuccess) return e;
  }
  return setup_kernel(acu_adj_step<N, true>, ADJ_SMEM_M, &g_grid_adj_m[dev][o]);
}

cudaError_t ensure_init(int* dev_out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  *dev_out = dev;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_init_mu);
  if (g_inited & (1ull << dev)) return cudaSuccess;
  if ((e = setup_order<2>(dev, 0)) != cudaSuccess) return e;
  if ((e = setup_order<4>(dev, 1)) != cudaSuccess) return e;
  g_inited |= 1ull << dev;
  return cudaSuccess;
}

AcuCoef coef_of(const AcuStep& p) {
  AcuCoef c;
  for (int k = 0; k < 4; k++) {
    c.c1x[k] = p.c1x[k];
    c.c1z[k] = p.c1z[k];
    c.c2x[k] = p.c2x[k];
    c.c2z[k] = p.c2z[k];
  }
  c.dt2 = p.dt2;
  return c;
}

}  // namespace

cudaError_t launch_selftest_wait(int* status, unsigned long long* waited_ns, cudaStream_t st) {
  k_selftest_wait<<<1, 32, 0, st>>>(status, waited_ns);
  return cudaGetLastError();
}

cudaError_t acu_kernels_init() {
  int dev;
  return ensure_init(&dev);
}

// TMA descriptors for a call: u is the [2][S][slice] wavefield pair, mh one
// [slice] field.
cudaError_t acu_make_maps(AcuMaps* maps, const Grid& g, int S, float* u_pair, const float* mh) {
  const cuuint64_t d3[3] = {(cuuint64_t)g.pitch, (cuuint64_t)g.rows, (cuuint64_t)(2 * S)};
  const cuuint64_t s3[2] = {(cuuint64_t)g.pitch * 4, (cuuint64_t)g.slice * 4};
  const cuuint32_t b3[3] = {(cuuint32_t)UW, (cuuint32_t)UH, 1};
  const cuuint64_t d2[2] = {(cuuint64_t)g.pitch, (cuuint64_t)g.rows};
  const cuuint64_t s2[1] = {(cuuint64_t)g.pitch * 4};
  const cuuint32_t b2[2] = {(cuuint32_t)MW, (cuuint32_t)MH};
  if (!tma_host::encode(&maps->u, u_pair, 3, d3, s3, b3)) return cudaErrorInvalidValue;
  if (!tma_host::encode(&maps->m, const_cast<float*>(mh), 2, d2, s2, b2)) return cudaErrorInvalidValue;
  // the 64-row forward tiles (the layout's rows are padded to 64, so these boxes fit)
  const cuuint32_t b3t[3] = {(cuuint32_t)UW, (cuuint32_t)FwdGeo<64>::UHT, 1};
  const cuuint32_t b2t[2] = {(cuuint32_t)MW, (cuuint32_t)FwdGeo<64>::MHT};
  if (!tma_host::encode(&maps->u64, u_pair, 3, d3, s3, b3t)) return cudaErrorInvalidValue;
  if (!tma_host::encode(&maps->m64, const_cast<float*>(mh), 2, d2, s2, b2t)) return cudaErrorInvalidValue;
  return cudaSuccess;
}

// Forward step on tiles of tz rows (32 or 64; 64 needs the 64-row boxes of
// acu_make_maps and is for single-instance launches).
cudaError_t launch_acu_fwd_tz(const AcuStep& p_in, const AcuMaps& maps, bool record, bool store, int tz,
                              cudaStream_t st, bool lap) {
  int dev;
  cudaError_t e = ensure_init(&dev);
  if (e != cudaSuccess) return e;
  const int v = (record ? 1 : 0) + (store ? 2 : 0);
  const int o = p_in.N == 2 ? 0 : 1;
  const AcuCoef cf = coef_of(p_in);
  BatchArgs nb;
  memset(&nb, 0, sizeof nb);
  if (lap) {  // the c^2 Laplacian operator: 32-row tiles
    const AcuStep& p = p_in;
    const int grid = std::min(p.ntiles, g_grid_fwd_lap[dev][o][v]);
    const size_t smem = sizeof(FwdSmem);
#define FWD_LAUNCH(NN, R, S) \
  acu_fwd_step<NN, R, S, false, 32, true><<<grid, NTHREADS, smem, st>>>(maps.u, maps.m, p, cf, nb)
    if (p.N == 2) {
      if (record && store) FWD_LAUNCH(2, true, true);
      else if (record) FWD_LAUNCH(2, true, false);
      else if (store) FWD_LAUNCH(2, false, true);
      else FWD_LAUNCH(2, false, false);
    } else {
      if (record && store) FWD_LAUNCH(4, true, true);
      else if (record) FWD_LAUNCH(4, true, false);
      else if (store) FWD_LAUNCH(4, false, true);
      else FWD_LAUNCH(4, false, false);
    }
#undef FWD_LAUNCH
    return cudaGetLastError();
  }
  if (tz == 64) {
    AcuStep p = p_in;
    p.ntiles = p.S * p.g.ntx * ((p.g.Nz + 63) / 64);
    const int grid = std::min(p.ntiles, g_grid_fwd64[dev][o][v]);
    const size_t smem = sizeof(FwdSmemT<64>);
    constexpr int T = FwdGeo<64>::NT;
#define FWD_LAUNCH(NN, R, S) acu_fwd_step<NN, R, S, false, 64><<<grid, T, smem, st>>>(maps.u64, maps.m64, p, cf, nb)
    if (p.N == 2) {
      if (record && store) FWD_LAUNCH(2, true, true);
      else if (record) FWD_LAUNCH(2, true, false);
      else if (store) FWD_LAUNCH(2, false, true);
      else FWD_LAUNCH(2, false, false);
    } else {
      if (record && store) FWD_LAUNCH(4, true, true);
      else if (record) FWD_LAUNCH(4, true, false);
      else if (store) FWD_LAUNCH(4, false, true);
      else FWD_LAUNCH(4, false, false);
    }
#undef FWD_LAUNCH
    return cudaGetLastError();
  }
  const AcuStep& p = p_in;
  const int grid = std::min(p.ntiles, g_grid_fwd[dev][o][v]);
  const size_t smem = sizeof(FwdSmem);
#define FWD_LAUNCH(NN, R, S) acu_fwd_step<NN, R, S, false, 32><<<grid, NTHREADS, smem, st>>>(maps.u, maps.m, p, cf, nb)
  if (p.N == 2) {
    if (record && store) FWD_LAUNCH(2, true, true);
    else if (record) FWD_LAUNCH(2, true, false);
    else if (store) FWD_LAUNCH(2, false, true);
    else FWD_LAUNCH(2, false, false);
  } else {
    if (record && store) FWD_LAUNCH(4, true, true);
    else if (record) FWD_LAUNCH(4, true, false);
    else if (store) FWD_LAUNCH(4, false, true);
    else FWD_LAUNCH(4, false, false);
  }
#undef FWD_LAUNCH
  return cudaGetLastError();
}

cudaError_t launch_acu_fwd(const AcuStep& p, const AcuMaps& maps, bool record, bool store, cudaStream_t st) {
  return launch_acu_fwd_tz(p, maps, record, store, TILE_Z, st, false);
}

// Multi-instance forward step b.n over the tiles of instances [0, b.n_active):
// the forward sweep (record: receivers recorded, fluxes stored by instances in
// their last segment) or the recompute of a segment (fluxes stored).
cudaError_t launch_acu_fwd_batch(const BatchArgs& b, const AcuCoef& cf, int N, bool record, cudaStream_t st) {
  int dev;
  cudaError_t e = ensure_init(&dev);
  if (e != cudaSuccess) return e;
  if (b.ntiles <= 0) return cudaSuccess;
  const int o = N == 2 ? 0 : 1;
  const int grid = std::min(b.ntiles, g_grid_fwd_m[dev][o][record ? 0 : 1]);
  CUtensorMap none;
  memset(&none, 0, sizeof none);
  AcuStep p0;
  memset(&p0, 0, sizeof p0);
#define FWD_LAUNCH(NN, R) acu_fwd_step<NN, R, true, true, 32><<<grid, NTHREADS, FWD_SMEM_M, st>>>(none, none, p0, cf, b)
  if (N == 2) {
    if (record) FWD_LAUNCH(2, true);
    else FWD_LAUNCH(2, false);
  } else {
    if (record) FWD_LAUNCH(4, true);
    else FWD_LAUNCH(4, false);
  }
#undef FWD_LAUNCH
  return cudaGetLastError();
}

// Adjoint operand maps: lambda and the hhat pairs Hx, Hz, each [2][S][slice],
// with the x-operand box (own rows, 80 columns) and the z-operand box (48 rows,
// own columns).
cudaError_t acu_make_adj_maps(AcuMaps* maps, const Grid& g, int S, float* lam_pair, float* hx_pair, float* hz_pair) {
  const cuuint64_t d3[3] = {(cuuint64_t)g.pitch, (cuuint64_t)g.rows, (cuuint64_t)(2 * S)};
  const cuuint64_t s3[2] = {(cuuint64_t)g.pitch * 4, (cuuint64_t)g.slice * 4};
  const cuuint32_t bx[3] = {(cuuint32_t)UW, (cuuint32_t)TILE_Z, 1};
  const cuuint32_t bz[3] = {(cuuint32_t)TILE_X, (cuuint32_t)UH, 1};
  const bool ok = tma_host::encode(&maps->lx, lam_pair, 3, d3, s3, bx) &&
                  tma_host::encode(&maps->lz, lam_pair, 3, d3, s3, bz) &&
                  tma_host::encode(&maps->hx, hx_pair, 3, d3, s3, bx) &&
                  tma_host::encode(&maps->hz, hz_pair, 3, d3, s3, bz);
  return ok ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_acu_adj(const AcuStep& p, const AcuMaps& maps, cudaStream_t st, bool lap) {
  int dev;
  cudaError_t e = ensure_init(&dev);
  if (e != cudaSuccess) return e;
  const int grid = std::min(p.ntiles, (lap ? g_grid_adj_lap : g_grid_adj)[dev][p.N == 2 ? 0 : 1]);
  const size_t smem = sizeof(AdjSmem);
  const AcuCoef cf = coef_of(p);
  BatchArgs nb;
  memset(&nb, 0, sizeof nb);
  if (lap) {
    if (p.N == 2)
      acu_adj_step<2, false, true><<<grid, NTHREADS, smem, st>>>(maps.lx, maps.lz, maps.hx, maps.hz, maps.m, p, cf, nb);
    else
      acu_adj_step<4, false, true><<<grid, NTHREADS, smem, st>>>(maps.lx, maps.lz, maps.hx, maps.hz, maps.m, p, cf, nb);
    return cudaGetLastError();
  }
  if (p.N == 2)
    acu_adj_step<2, false><<<grid, NTHREADS, smem, st>>>(maps.lx, maps.lz, maps.hx, maps.hz, maps.m, p, cf, nb);
  else
    acu_adj_step<4, false><<<grid, NTHREADS, smem, st>>>(maps.lx, maps.lz, maps.hx, maps.hz, maps.m, p, cf, nb);
  return cudaGetLastError();
}

// Multi-instance adjoint step b.n over the tiles of instances [0, b.n_active).
cudaError_t launch_acu_adj_batch(const BatchArgs& b, const AcuCoef& cf, int N, cudaStream_t st) {
  int dev;
  cudaError_t e = ensure_init(&dev);
  if (e != cudaSuccess) return e;
  if (b.ntiles <= 0) return cudaSuccess;
  const int grid = std::min(b.ntiles, g_grid_adj_m[dev][N == 2 ? 0 : 1]);
  CUtensorMap none;
  memset(&none, 0, sizeof none);
  AcuStep p0;
  memset(&p0, 0, sizeof p0);
  if (N == 2) acu_adj_step<2, true><<<grid, NTHREADS, ADJ_SMEM_M, st>>>(none, none, none, none, none, p0, cf, b);
  else acu_adj_step<4, true><<<grid, NTHREADS, ADJ_SMEM_M, st>>>(none, none, none, none, none, p0, cf, b);
  return cudaGetLastError();
}

}  // namespace fwi
