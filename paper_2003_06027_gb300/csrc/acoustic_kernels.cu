// acoustic_kernels.cu - sm_103a kernels of the acoustic hot path.
//
// One time step of the recursion U_{k+1} = A(theta) U_k + F_k (Method,
// Eq. forward) for u_tt = div(c^2 grad u) + f (Implementation, Eq. acoustic)
// on the staggered grid, and one step of its exact transpose
// lambda_k = A^T lambda_{k+1} + residual (Eq. adjoint-backward) fused with the
// gradient correlation lambda^T (dA/dm) U (Eq. adjoint-gradient).
//
// Both step kernels are memory bound (no dense contraction): one CTA owns a
// 64 x 16 tile of one shot, stages the tile plus its halo in shared memory with
// coalesced float4 loads, evaluates the first-stage half-point fluxes once per
// half point in shared memory, then the second-stage divergence, and streams
// each field through HBM once per step. CPML memory variables are read and
// written only where the damping coefficient is non-zero.
#include <cuda_runtime.h>

#include "fwi_internal.cuh"

namespace fwi {

namespace {

constexpr int H = 8;                        // halo of the wavefield tile
constexpr int SUW = TILE_X + 2 * H;         // 80
constexpr int SUH = TILE_Z + 2 * H;         // 32
constexpr int SMW = TILE_X + 12;            // m tile cols [x0-4, x0+TX+8)
constexpr int SMH = TILE_Z + 9;             // m tile rows [z0-4, z0+TZ+5)
constexpr int QXW = TILE_X + 8;             // half cols [x0-4, x0+TX+4)
constexpr int QZH = TILE_Z + 8;             // half rows [z0-4, z0+TZ+4)
constexpr int NQX = TILE_Z * (QXW / 4);
constexpr int NQZ = QZH * (TILE_X / 4);

__device__ __forceinline__ float4 ld4s(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4s(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }

// Stage a rows x (4*c4n) window of a field whose top-left global cell is
// (zt, xt) into shared memory (row stride w floats).
__device__ __forceinline__ void stage(float* dst, int w, const float* __restrict__ src, int pitch,
                                      int zt, int xt, int nrows, int c4n) {
  for (int idx = threadIdx.x; idx < nrows * c4n; idx += NTHREADS) {
    int r = idx / c4n, c4 = idx - r * c4n;
    float4 v = __ldg(reinterpret_cast<const float4*>(src + (long long)(zt + r) * pitch + (xt + 4 * c4)));
    st4s(dst + r * w + 4 * c4, v);
  }
}

__device__ __forceinline__ bool tile_pml_x(const Grid& g, int x0) {
  return g.npml > 0 && (x0 - H < g.npml || x0 + TILE_X + H > g.npml + g.nx - 1);
}
__device__ __forceinline__ bool tile_pml_z(const Grid& g, int z0) {
  return g.npml > 0 && (z0 - H < g.npml || z0 + TILE_Z + H > g.npml + g.nz - 1);
}

// Deterministic CTA sum of three floats (fixed shuffle tree, fixed warp order).
__device__ __forceinline__ void cta_sum3(float v[3], float (*red)[3]) {
  for (int k = 0; k < 3; k++)
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0)
    for (int k = 0; k < 3; k++) red[warp][k] = v[k];
  __syncthreads();
  if (threadIdx.x == 0)
    for (int k = 0; k < 3; k++) {
      float s = 0.f;
      for (int w = 0; w < NTHREADS / 32; w++) s += red[w][k];
      v[k] = s;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Forward step n: u^{n+1} = 2 u^n - u^{n-1} + dt^2 (div(m grad u^n) + f^n) with
// CPML. RECORD writes the receiver samples; STORE saves u^n and the updated
// psi (the operands of the gradient correlation) into the segment slot.
template <int N, bool RECORD, bool STORE>
__global__ void __launch_bounds__(NTHREADS) acu_fwd_step(const AcuStep p) {
  __shared__ __align__(16) float su[SUH][SUW];
  __shared__ __align__(16) float sm[SMH][SMW];
  __shared__ __align__(16) float sqx[TILE_Z][QXW];
  __shared__ __align__(16) float sqz[QZH][TILE_X];

  const Grid& g = p.g;
  const int tid = threadIdx.x, s = blockIdx.z;
  const int x0 = blockIdx.x * TILE_X, z0 = blockIdx.y * TILE_Z;
  const int pitch = g.pitch;
  const long long sh = (long long)s * g.slice + g.off0;

  stage(&su[0][0], SUW, p.u_cur + sh, pitch, z0 - H, x0 - H, SUH, SUW / 4);
  stage(&sm[0][0], SMW, p.m + g.off0, pitch, z0 - 4, x0 - 4, SMH, SMW / 4);
  __syncthreads();

  const bool pmlx = tile_pml_x(g, x0), pmlz = tile_pml_z(g, z0);
  const float inv_dx = p.inv_dx, inv_dz = p.inv_dz;

  // Stage 1: q = m_half * (D+ u + psi) at the half points of the tile + halo.
  for (int it = tid; it < NQX + NQZ; it += NTHREADS) {
    if (it < NQX) {
      const int r = it / (QXW / 4), gq = it - r * (QXW / 4);
      const int z = z0 + r, hb = x0 - 4 + 4 * gq;
      float v[12];
      {
        const float* row = &su[r + H][4 * gq];
        float4 a0 = ld4s(row), a1 = ld4s(row + 4), a2 = ld4s(row + 8);
        v[0] = a0.x; v[1] = a0.y; v[2] = a0.z; v[3] = a0.w;
        v[4] = a1.x; v[5] = a1.y; v[6] = a1.z; v[7] = a1.w;
        v[8] = a2.x; v[9] = a2.y; v[10] = a2.z; v[11] = a2.w;
      }
      float q[4];
#pragma unroll
      for (int e = 0; e < 4; e++) {
        float gx = 0.f;
#pragma unroll
        for (int k = 1; k <= N; k++) gx += p.a[k - 1] * (v[e + 4 + k] - v[e + 5 - k]);
        gx *= inv_dx;
        const int h = hb + e;
        float pp = gx;
        if (pmlx) {
          const float aa = __ldg(p.axh + h + TAB_OFF);
          if (aa != 0.f) {
            const float bb = __ldg(p.bxh + h + TAB_OFF);
            const long long id = sh + (long long)z * pitch + h;
            const float ps = bb * p.psix_in[id] + aa * gx;
            if (h >= x0 && h < x0 + TILE_X && z < g.Nz) {
              p.psix_out[id] = ps;
              if (STORE) p.slot_psix[id] = ps;
            }
            pp += ps;
          }
        }
        const float mh = 0.5f * (sm[r + 4][4 * gq + e] + sm[r + 4][4 * gq + e + 1]);
        q[e] = (h >= 0 && h < g.Nx - 1 && z < g.Nz) ? mh * pp : 0.f;
      }
      st4s(&sqx[r][4 * gq], make_float4(q[0], q[1], q[2], q[3]));
    } else {
      const int k2 = it - NQX;
      const int hr = k2 / (TILE_X / 4), c = k2 - hr * (TILE_X / 4);
      const int hz = z0 - 4 + hr, xb = x0 + 4 * c;
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int k = 1; k <= N; k++) {
        const float4 wp = ld4s(&su[hr + 4 + k][8 + 4 * c]);
        const float4 wm = ld4s(&su[hr + 5 - k][8 + 4 * c]);
        acc.x += p.a[k - 1] * (wp.x - wm.x);
        acc.y += p.a[k - 1] * (wp.y - wm.y);
        acc.z += p.a[k - 1] * (wp.z - wm.z);
        acc.w += p.a[k - 1] * (wp.w - wm.w);
      }
      float gz[4] = {acc.x * inv_dz, acc.y * inv_dz, acc.z * inv_dz, acc.w * inv_dz};
      float pp[4] = {gz[0], gz[1], gz[2], gz[3]};
      if (pmlz) {
        const float aa = __ldg(p.azh + hz + TAB_OFF);
        if (aa != 0.f) {
          const float bb = __ldg(p.bzh + hz + TAB_OFF);
          const bool own = hz >= z0 && hz < z0 + TILE_Z;
          const long long id = sh + (long long)hz * pitch + xb;
          const float4 po = *reinterpret_cast<const float4*>(p.psiz_in + id);
          float4 pn;
          pn.x = bb * po.x + aa * gz[0];
          pn.y = bb * po.y + aa * gz[1];
          pn.z = bb * po.z + aa * gz[2];
          pn.w = bb * po.w + aa * gz[3];
          if (own) {
            // columns beyond Nx are outside the grid: keep them zero
            if (xb + 0 >= g.Nx) pn.x = 0.f;
            if (xb + 1 >= g.Nx) pn.y = 0.f;
            if (xb + 2 >= g.Nx) pn.z = 0.f;
            if (xb + 3 >= g.Nx) pn.w = 0.f;
            *reinterpret_cast<float4*>(p.psiz_out + id) = pn;
            if (STORE) *reinterpret_cast<float4*>(p.slot_psiz + id) = pn;
          }
          pp[0] += pn.x; pp[1] += pn.y; pp[2] += pn.z; pp[3] += pn.w;
        }
      }
      const bool hv = hz >= 0 && hz < g.Nz - 1;
      float q[4];
#pragma unroll
      for (int e = 0; e < 4; e++) {
        const float mh = 0.5f * (sm[hr][4 * c + 4 + e] + sm[hr + 1][4 * c + 4 + e]);
        q[e] = (hv && xb + e < g.Nx) ? mh * pp[e] : 0.f;
      }
      st4s(&sqz[hr][4 * c], make_float4(q[0], q[1], q[2], q[3]));
    }
  }
  __syncthreads();

  // Stage 2: divergence D- q + CPML zeta, leapfrog, source, receivers.
  const int tx = tid & 15, ty = tid >> 4;
  const int z = z0 + ty, xb = x0 + 4 * tx;
  float v[12];
  {
    const float* row = &sqx[ty][4 * tx];
    float4 a0 = ld4s(row), a1 = ld4s(row + 4), a2 = ld4s(row + 8);
    v[0] = a0.x; v[1] = a0.y; v[2] = a0.z; v[3] = a0.w;
    v[4] = a1.x; v[5] = a1.y; v[6] = a1.z; v[7] = a1.w;
    v[8] = a2.x; v[9] = a2.y; v[10] = a2.z; v[11] = a2.w;
  }
  float4 hz4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int k = 1; k <= N; k++) {
    const float4 wp = ld4s(&sqz[ty + k + 3][4 * tx]);
    const float4 wm = ld4s(&sqz[ty - k + 4][4 * tx]);
    hz4.x += p.a[k - 1] * (wp.x - wm.x);
    hz4.y += p.a[k - 1] * (wp.y - wm.y);
    hz4.z += p.a[k - 1] * (wp.z - wm.z);
    hz4.w += p.a[k - 1] * (wp.w - wm.w);
  }
  const float hzv[4] = {hz4.x * inv_dz, hz4.y * inv_dz, hz4.z * inv_dz, hz4.w * inv_dz};
  const bool zin = z < g.Nz;
  const float az_ = pmlz ? __ldg(p.az + z + TAB_OFF) : 0.f;
  const float bz_ = pmlz ? __ldg(p.bz + z + TAB_OFF) : 1.f;
  float rr[4];
#pragma unroll
  for (int e = 0; e < 4; e++) {
    float hx = 0.f;
#pragma unroll
    for (int k = 1; k <= N; k++) hx += p.a[k - 1] * (v[e + k + 3] - v[e - k + 4]);
    hx *= inv_dx;
    const int j = xb + e;
    const bool valid = zin && j < g.Nx;
    float r = hx + hzv[e];
    const long long id = sh + (long long)z * pitch + j;
    if (pmlx) {
      const float aa = __ldg(p.ax + j + TAB_OFF);
      if (aa != 0.f) {
        const float zn = __ldg(p.bx + j + TAB_OFF) * p.zetx[id] + aa * hx;
        if (valid) p.zetx[id] = zn;
        r += zn;
      }
    }
    if (az_ != 0.f) {
      const float zn = bz_ * p.zetz[id] + az_ * hzv[e];
      if (valid) p.zetz[id] = zn;
      r += zn;
    }
    rr[e] = r;
  }
  const float4 uc = ld4s(&su[ty + H][4 * tx + H]);
  float* upp = p.u_prev + sh + (long long)z * pitch + xb;
  const float4 uo = *reinterpret_cast<const float4*>(upp);
  float un[4];
  un[0] = 2.f * uc.x - uo.x + p.dt2 * rr[0];
  un[1] = 2.f * uc.y - uo.y + p.dt2 * rr[1];
  un[2] = 2.f * uc.z - uo.z + p.dt2 * rr[2];
  un[3] = 2.f * uc.w - uo.w + p.dt2 * rr[3];
  {
    // source term dt^2 w g(t_n) on the cells of this tile inside the box
    const int i0 = p.src_box[2 * s], j0 = p.src_box[2 * s + 1], nb = p.src_n;
    if (i0 >= 0 && i0 < z0 + TILE_Z && i0 + nb > z0 && j0 < x0 + TILE_X && j0 + nb > x0) {
      const float amp = p.dt2 * p.stf[(long long)s * p.nt + p.n];
      const int di = z - i0;
      if (di >= 0 && di < nb) {
#pragma unroll
        for (int e = 0; e < 4; e++) {
          const int dj = xb + e - j0;
          if (dj >= 0 && dj < nb) un[e] += amp * p.src_w[s * SRC_W * SRC_W + di * SRC_W + dj];
        }
      }
    }
  }
#pragma unroll
  for (int e = 0; e < 4; e++)
    if (!(zin && xb + e < g.Nx)) un[e] = 0.f;
  *reinterpret_cast<float4*>(upp) = make_float4(un[0], un[1], un[2], un[3]);
  if (STORE) *reinterpret_cast<float4*>(p.slot_u + sh + (long long)z * pitch + xb) = uc;
  if (RECORD) {
    const int t = blockIdx.y * g.ntx + blockIdx.x;
    const int rb = p.tile_rec_start[t], re = p.tile_rec_start[t + 1];
    for (int q = rb; q < re; q++) {
      const int r = p.tile_rec[q];
      const int ri = p.rec_cell[2 * r], rj = p.rec_cell[2 * r + 1];
      const int d = rj - xb;
      if (ri == z && d >= 0 && d < 4) {
        const float val = d == 0 ? un[0] : (d == 1 ? un[1] : (d == 2 ? un[2] : un[3]));
        p.seis[((long long)s * p.nrec + r) * p.nt + p.n] = val;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Adjoint step n (reverse of forward step n, statement by statement):
//   rbar = dt^2 lambda_{n+1};   hbar = rbar + a (Z + rbar),  Z <- b (Z + rbar)
//   qbar = D-^T hbar = -D+ hbar (half points)
//   g_m  += qbar * p^n           (gradient correlation, Eq. adjoint-gradient)
//   pbar = m_half qbar;  gbar = pbar + a_h (P + pbar),  P <- b_h (P + pbar)
//   lambda_n = 2 lambda_{n+1} - lambda_{n+2} + D+^T gbar + residual(n-1)
// The cell gradient receives half of each adjacent half-point correlation.
struct AdjSmem {
  float sl[SUH][SUW];      // lambda_{n+1}, halo 8
  float su[SUH][SUW];      // u^n, halo 8
  float sm[SMH][SMW];
  float shx[TILE_Z][SUW];  // hbar_x (CPML tiles)
  float shz[SUH][SUW];     // hbar_z (CPML tiles)
  float sgx[TILE_Z][QXW];
  float sgz[QZH][TILE_X];
  float simx[TILE_Z][QXW];
  float simz[QZH][TILE_X];
  float red[NTHREADS / 32][3];
};

template <int N>
__global__ void __launch_bounds__(NTHREADS) acu_adj_step(const AcuStep p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  AdjSmem& S = *reinterpret_cast<AdjSmem*>(smem_raw);
  auto& sl = S.sl;
  auto& su = S.su;
  auto& sm = S.sm;
  auto& shx = S.shx;
  auto& shz = S.shz;
  auto& sgx = S.sgx;
  auto& sgz = S.sgz;
  auto& simx = S.simx;
  auto& simz = S.simz;
  auto& red = S.red;

  const Grid& g = p.g;
  const int tid = threadIdx.x, s = blockIdx.z;
  const int x0 = blockIdx.x * TILE_X, z0 = blockIdx.y * TILE_Z;
  const int pitch = g.pitch;
  const long long sh = (long long)s * g.slice + g.off0;
  const float dt2 = p.dt2, inv_dx = p.inv_dx, inv_dz = p.inv_dz;

  stage(&sl[0][0], SUW, p.l_cur + sh, pitch, z0 - H, x0 - H, SUH, SUW / 4);
  stage(&su[0][0], SUW, p.slot_u + sh, pitch, z0 - H, x0 - H, SUH, SUW / 4);
  stage(&sm[0][0], SMW, p.m + g.off0, pitch, z0 - 4, x0 - 4, SMH, SMW / 4);
  __syncthreads();

  const bool pmlx = tile_pml_x(g, x0), pmlz = tile_pml_z(g, z0);

  // Stage 0 (CPML tiles): hbar including the memory variable Z.
  if (pmlx) {
    for (int idx = tid; idx < TILE_Z * SUW; idx += NTHREADS) {
      const int r = idx / SUW, c = idx - r * SUW;
      const int z = z0 + r, j = x0 - H + c;
      const float rb = dt2 * sl[r + H][c];
      float hb = rb;
      const float aa = __ldg(p.ax + j + TAB_OFF);
      if (aa != 0.f) {
        const long long id = sh + (long long)z * pitch + j;
        const float t = p.zx_in[id] + rb;
        hb = rb + aa * t;
        if (c >= H && c < H + TILE_X && z < g.Nz && j < g.Nx) p.zx_out[id] = __ldg(p.bx + j + TAB_OFF) * t;
      }
      shx[r][c] = hb;
    }
  }
  if (pmlz) {
    for (int idx = tid; idx < SUH * TILE_X; idx += NTHREADS) {
      const int r = idx / TILE_X, c = idx - r * TILE_X;
      const int z = z0 - H + r, j = x0 + c;
      const float rb = dt2 * sl[r][c + H];
      float hb = rb;
      const float aa = __ldg(p.az + z + TAB_OFF);
      if (aa != 0.f) {
        const long long id = sh + (long long)z * pitch + j;
        const float t = p.zz_in[id] + rb;
        hb = rb + aa * t;
        if (r >= H && r < H + TILE_Z && z < g.Nz && j < g.Nx) p.zz_out[id] = __ldg(p.bz + z + TAB_OFF) * t;
      }
      shz[r][c + H] = hb;
    }
  }
  __syncthreads();
  // hbar sources: CPML tiles read the staged hbar, others dt^2 lambda
  const float* hxb = pmlx ? &shx[0][0] : &sl[H][0];
  const float hxs = pmlx ? 1.f : dt2;
  const float* hzb = pmlz ? &shz[0][0] : &sl[0][0];
  const float hzs = pmlz ? 1.f : dt2;

  // Stage 1: qbar, gradient correlation, gbar at the half points.
  for (int it = tid; it < NQX + NQZ; it += NTHREADS) {
    if (it < NQX) {
      const int r = it / (QXW / 4), gq = it - r * (QXW / 4);
      const int z = z0 + r, hb = x0 - 4 + 4 * gq;
      float v[12], w[12];
      {
        const float* row = hxb + r * SUW + 4 * gq;
        float4 a0 = ld4s(row), a1 = ld4s(row + 4), a2 = ld4s(row + 8);
        v[0] = a0.x; v[1] = a0.y; v[2] = a0.z; v[3] = a0.w;
        v[4] = a1.x; v[5] = a1.y; v[6] = a1.z; v[7] = a1.w;
        v[8] = a2.x; v[9] = a2.y; v[10] = a2.z; v[11] = a2.w;
        const float* urow = &su[r + H][4 * gq];
        a0 = ld4s(urow); a1 = ld4s(urow + 4); a2 = ld4s(urow + 8);
        w[0] = a0.x; w[1] = a0.y; w[2] = a0.z; w[3] = a0.w;
        w[4] = a1.x; w[5] = a1.y; w[6] = a1.z; w[7] = a1.w;
        w[8] = a2.x; w[9] = a2.y; w[10] = a2.z; w[11] = a2.w;
      }
      float gb[4], im[4];
#pragma unroll
      for (int e = 0; e < 4; e++) {
        float dq = 0.f, du = 0.f;
#pragma unroll
        for (int k = 1; k <= N; k++) {
          dq += p.a[k - 1] * (v[e + 4 + k] - v[e + 5 - k]);
          du += p.a[k - 1] * (w[e + 4 + k] - w[e + 5 - k]);
        }
        const int h = hb + e;
        const bool inh = h >= 0 && h < g.Nx - 1 && z < g.Nz;
        const float qb = inh ? -dq * inv_dx * hxs : 0.f;
        float px = du * inv_dx;
        const float mh = 0.5f * (sm[r + 4][4 * gq + e] + sm[r + 4][4 * gq + e + 1]);
        const float pb = mh * qb;
        float gbar = pb;
        if (pmlx) {
          const float aa = __ldg(p.axh + h + TAB_OFF);
          if (aa != 0.f) {
            const long long id = sh + (long long)z * pitch + h;
            px += p.slot_psix[id];
            const float t = p.px_in[id] + pb;
            gbar = pb + aa * t;
            if (h >= x0 && h < x0 + TILE_X && z < g.Nz) p.px_out[id] = __ldg(p.bxh + h + TAB_OFF) * t;
          }
        }
        gb[e] = inh ? gbar : 0.f;
        im[e] = qb * px;
      }
      st4s(&sgx[r][4 * gq], make_float4(gb[0], gb[1], gb[2], gb[3]));
      st4s(&simx[r][4 * gq], make_float4(im[0], im[1], im[2], im[3]));
    } else {
      const int k2 = it - NQX;
      const int hr = k2 / (TILE_X / 4), c = k2 - hr * (TILE_X / 4);
      const int hz = z0 - 4 + hr, xb = x0 + 4 * c;
      float4 dq = make_float4(0.f, 0.f, 0.f, 0.f), du = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int k = 1; k <= N; k++) {
        const float4 hp = ld4s(hzb + (hr + 4 + k) * SUW + 8 + 4 * c);
        const float4 hm = ld4s(hzb + (hr + 5 - k) * SUW + 8 + 4 * c);
        const float4 up = ld4s(&su[hr + 4 + k][8 + 4 * c]);
        const float4 um = ld4s(&su[hr + 5 - k][8 + 4 * c]);
        const float ak = p.a[k - 1];
        dq.x += ak * (hp.x - hm.x); dq.y += ak * (hp.y - hm.y);
        dq.z += ak * (hp.z - hm.z); dq.w += ak * (hp.w - hm.w);
        du.x += ak * (up.x - um.x); du.y += ak * (up.y - um.y);
        du.z += ak * (up.z - um.z); du.w += ak * (up.w - um.w);
      }
      const float dqv[4] = {dq.x, dq.y, dq.z, dq.w};
      const float duv[4] = {du.x, du.y, du.z, du.w};
      const bool hv = hz >= 0 && hz < g.Nz - 1;
      const float aa = pmlz ? __ldg(p.azh + hz + TAB_OFF) : 0.f;
      const float bb = pmlz ? __ldg(p.bzh + hz + TAB_OFF) : 1.f;
      const bool own = hz >= z0 && hz < z0 + TILE_Z;
      float gb[4], im[4];
#pragma unroll
      for (int e = 0; e < 4; e++) {
        const bool inh = hv && xb + e < g.Nx;
        const float qb = inh ? -dqv[e] * inv_dz * hzs : 0.f;
        float pz = duv[e] * inv_dz;
        const float mh = 0.5f * (sm[hr][4 * c + 4 + e] + sm[hr + 1][4 * c + 4 + e]);
        const float pb = mh * qb;
        float gbar = pb;
        if (aa != 0.f) {
          const long long id = sh + (long long)hz * pitch + xb + e;
          pz += p.slot_psiz[id];
          const float t = p.pz_in[id] + pb;
          gbar = pb + aa * t;
          if (own && xb + e < g.Nx) p.pz_out[id] = bb * t;
        }
        gb[e] = inh ? gbar : 0.f;
        im[e] = qb * pz;
      }
      st4s(&sgz[hr][4 * c], make_float4(gb[0], gb[1], gb[2], gb[3]));
      st4s(&simz[hr][4 * c], make_float4(im[0], im[1], im[2], im[3]));
    }
  }
  __syncthreads();

  // Stage 2: lambda_n and the cell gradient.
  const int tx = tid & 15, ty = tid >> 4;
  const int z = z0 + ty, xb = x0 + 4 * tx;
  float v[12];
  {
    const float* row = &sgx[ty][4 * tx];
    float4 a0 = ld4s(row), a1 = ld4s(row + 4), a2 = ld4s(row + 8);
    v[0] = a0.x; v[1] = a0.y; v[2] = a0.z; v[3] = a0.w;
    v[4] = a1.x; v[5] = a1.y; v[6] = a1.z; v[7] = a1.w;
    v[8] = a2.x; v[9] = a2.y; v[10] = a2.z; v[11] = a2.w;
  }
  float4 dz4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int k = 1; k <= N; k++) {
    const float4 wp = ld4s(&sgz[ty + k + 3][4 * tx]);
    const float4 wm = ld4s(&sgz[ty - k + 4][4 * tx]);
    dz4.x += p.a[k - 1] * (wp.x - wm.x);
    dz4.y += p.a[k - 1] * (wp.y - wm.y);
    dz4.z += p.a[k - 1] * (wp.z - wm.z);
    dz4.w += p.a[k - 1] * (wp.w - wm.w);
  }
  const float dzv[4] = {dz4.x * inv_dz, dz4.y * inv_dz, dz4.z * inv_dz, dz4.w * inv_dz};
  const float4 lc = ld4s(&sl[ty + H][4 * tx + H]);
  const float lcv[4] = {lc.x, lc.y, lc.z, lc.w};
  const long long id0 = sh + (long long)z * pitch + xb;
  const float4 lo = *reinterpret_cast<const float4*>(p.l_prev + id0);
  const float lov[4] = {lo.x, lo.y, lo.z, lo.w};
  const float4 gold = *reinterpret_cast<const float4*>(p.gpart + id0);
  const float goldv[4] = {gold.x, gold.y, gold.z, gold.w};
  const float4 imzu = ld4s(&simz[ty + 3][4 * tx]);
  const float4 imzd = ld4s(&simz[ty + 4][4 * tx]);
  const float imzuv[4] = {imzu.x, imzu.y, imzu.z, imzu.w};
  const float imzdv[4] = {imzd.x, imzd.y, imzd.z, imzd.w};
  float ln[4], gn[4];
  const bool zin = z < g.Nz;
#pragma unroll
  for (int e = 0; e < 4; e++) {
    float dxv = 0.f;
#pragma unroll
    for (int k = 1; k <= N; k++) dxv += p.a[k - 1] * (v[e + k + 3] - v[e - k + 4]);
    dxv *= inv_dx;
    const bool valid = zin && xb + e < g.Nx;
    ln[e] = valid ? 2.f * lcv[e] - lov[e] - (dxv + dzv[e]) : 0.f;
    const float gi = 0.5f * (simx[ty][4 * tx + e + 3] + simx[ty][4 * tx + e + 4] + imzuv[e] + imzdv[e]);
    gn[e] = valid ? goldv[e] + gi : 0.f;
  }
  // residual of the sample recorded from u^n (sample n-1)
  if (p.n >= 1) {
    const int t = blockIdx.y * g.ntx + blockIdx.x;
    const int rb = p.tile_rec_start[t], re = p.tile_rec_start[t + 1];
    for (int q = rb; q < re; q++) {
      const int r = p.tile_rec[q];
      const int ri = p.rec_cell[2 * r], rj = p.rec_cell[2 * r + 1];
      const int d = rj - xb;
      if (ri == z && d >= 0 && d < 4) {
        const float rv = p.res[((long long)s * p.nrec + r) * p.nt + p.n - 1];
#pragma unroll
        for (int e = 0; e < 4; e++)
          if (e == d) ln[e] += rv;
      }
    }
  }
  *reinterpret_cast<float4*>(p.l_prev + id0) = make_float4(ln[0], ln[1], ln[2], ln[3]);
  *reinterpret_cast<float4*>(p.gpart + id0) = make_float4(gn[0], gn[1], gn[2], gn[3]);

  // source-parameter partials from lambda_n (index n-1): sum w lambda,
  // sum w lambda (x_i - x0), sum w lambda (z_i - z0); at most 4 tiles touch a box
  if (p.src_part != nullptr && p.n >= 1) {
    const int i0 = p.src_box[2 * s], j0 = p.src_box[2 * s + 1], nb = p.src_n;
    if (i0 >= 0 && i0 < z0 + TILE_Z && i0 + nb > z0 && j0 < x0 + TILE_X && j0 + nb > x0) {
      float acc[3] = {0.f, 0.f, 0.f};
      const int di = z - i0;
      if (di >= 0 && di < nb) {
        const float xs = p.x0[2 * s], zs = p.x0[2 * s + 1];
#pragma unroll
        for (int e = 0; e < 4; e++) {
          const int dj = xb + e - j0;
          if (dj >= 0 && dj < nb) {
            const float wl = p.src_w[s * SRC_W * SRC_W + di * SRC_W + dj] * ln[e];
            acc[0] += wl;
            acc[1] += wl * ((float)(xb + e - g.npml) * p.dx - xs);
            acc[2] += wl * ((float)(z - g.npml) * p.dz - zs);
          }
        }
      }
      cta_sum3(acc, red);
      if (tid == 0) {
        const int slot = 2 * (blockIdx.y - i0 / TILE_Z) + (blockIdx.x - j0 / TILE_X);
        float* dst = p.src_part + (((long long)s * p.nt + (p.n - 1)) * SRC_SLOTS + slot) * 3;
        dst[0] = acc[0];
        dst[1] = acc[1];
        dst[2] = acc[2];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Host-side launchers (called from fwi_capi.cu).
cudaError_t launch_acu_fwd(const AcuStep& p, bool record, bool store, cudaStream_t st) {
  dim3 grid(p.g.ntx, p.g.ntz, p.S);
  if (p.N == 2) {
    if (record) acu_fwd_step<2, true, false><<<grid, NTHREADS, 0, st>>>(p);
    else if (store) acu_fwd_step<2, false, true><<<grid, NTHREADS, 0, st>>>(p);
    else acu_fwd_step<2, false, false><<<grid, NTHREADS, 0, st>>>(p);
  } else {
    if (record) acu_fwd_step<4, true, false><<<grid, NTHREADS, 0, st>>>(p);
    else if (store) acu_fwd_step<4, false, true><<<grid, NTHREADS, 0, st>>>(p);
    else acu_fwd_step<4, false, false><<<grid, NTHREADS, 0, st>>>(p);
  }
  return cudaGetLastError();
}

cudaError_t launch_acu_adj(const AcuStep& p, cudaStream_t st) {
  dim3 grid(p.g.ntx, p.g.ntz, p.S);
  if (p.N == 2) acu_adj_step<2><<<grid, NTHREADS, sizeof(AdjSmem), st>>>(p);
  else acu_adj_step<4><<<grid, NTHREADS, sizeof(AdjSmem), st>>>(p);
  return cudaGetLastError();
}

// The adjoint step stages nine tiles (about 64 KB): opt in to more than the
// default 48 KB of dynamic shared memory once per device.
cudaError_t acu_kernels_init() {
  cudaError_t e = cudaFuncSetAttribute(acu_adj_step<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(AdjSmem));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(acu_adj_step<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sizeof(AdjSmem));
}

}  // namespace fwi
