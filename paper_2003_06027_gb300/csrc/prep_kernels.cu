// prep_kernels.cu - parameter preparation, source/receiver set-up, misfit and
// gradient reductions of the acoustic path (sm_103a).
//
// Steps served: padded model and CPML tables (the coefficient matrix A(theta)
// of Eq. forward), source weights (point source or the Gaussian
// re-parameterisation of the Earthquake Location section), receiver lookup,
// the L2 misfit (Method, J = 1/2 sum |U_k - U_k^obs|^2) in FP64, and the FP64
// folds of the gradient of Eq. adjoint-gradient over time segments and shots.
#include <cuda_runtime.h>

#include <cmath>

#include "fwi_internal.cuh"

namespace fwi {


// m/2 = c^2/2 on the padded grid with the CPML filled by edge replication
// (the half-point coefficient is then the sum of two neighbours); every
// allocated cell is written (zero outside the padded grid).
__global__ void k_pad_model_sq(const float* __restrict__ c, Grid g, float* __restrict__ m) {
  const long long total = (long long)g.rows * g.pitch;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(idx / g.pitch), col = (int)(idx - (long long)r * g.pitch);
    const int i = r - APRON, j = col - APRON;
    float v = 0.f;
    if (i >= 0 && i < g.Nz && j >= 0 && j < g.Nx) {
      const int ci = min(max(i - g.npml, 0), g.nz - 1), cj = min(max(j - g.npml, 0), g.nx - 1);
      const float cc = c[(long long)ci * g.nx + cj];
      v = 0.5f * cc * cc;
    }
    m[idx] = v;
  }
}

// CPML coefficients along one axis (Komatitsch & Martin 2007, cited in the
// paper's Implementation section): kappa = 1, d(l) = d0 (l/L)^2,
// d0 = -3 vmax ln R / (2 L), alpha = pi f0 (1 - l/L), b = exp(-(d + alpha) dt),
// a = d (b - 1) / (d + alpha); l = distance into the layer. Entries outside
// the padded axis (and half points past its last node) are a = 0, b = 1.
__global__ void k_cpml_tables(int n_phys, int npml, int Npad, int len, double h, double dt, double R,
                              double vmax, double f0, float* a, float* b, float* ah, float* bh) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= len) return;
  const int idx = k - TAB_OFF;
  for (int half = 0; half < 2; half++) {
    float av = 0.f, bv = 1.f;
    const bool inside = half ? (idx >= 0 && idx < Npad - 1) : (idx >= 0 && idx < Npad);
    if (inside && npml > 0) {
      const double x = idx + (half ? 0.5 : 0.0);
      double l = 0.0;
      if (npml - x > l) l = npml - x;
      if (x - (npml + n_phys - 1) > l) l = x - (npml + n_phys - 1);
      l *= h;
      if (l > 0.0) {
        const double L = npml * h;
        const double d0 = -3.0 * vmax * log(R) / (2.0 * L);
        const double d = d0 * (l / L) * (l / L);
        const double al = M_PI * f0 * (1.0 - l / L);
        const double bb = exp(-(d + al) * dt);
        bv = (float)bb;
        av = (float)(d * (bb - 1.0) / (d + al));
      }
    }
    if (half) {
      ah[k] = av;
      bh[k] = bv;
    } else {
      a[k] = av;
      b[k] = bv;
    }
  }
}

// Per-shot source box and weights. Point source: 1/(dx dz) on the nearest
// physical cell. Gaussian: g/(2 pi s^2) exp(-|x - x0|^2/(2 s^2)), s = dx/2, on
// the 7 x 7 cells around the nearest cell.
__global__ void k_src_prep(int S, int kind, const float* __restrict__ x0, Grid g, float dx, float dz,
                           int* box, float* w, int* status) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  const double xr = x0[2 * s], zr = x0[2 * s + 1];
  const int jc = (int)llround(xr / (double)dx) + g.npml;
  const int ic = (int)llround(zr / (double)dz) + g.npml;
  float* ws = w + s * SRC_W * SRC_W;
  for (int q = 0; q < SRC_W * SRC_W; q++) ws[q] = 0.f;
  bool ok;
  if (kind == 0) {
    ok = isfinite(xr) && isfinite(zr) && ic >= g.npml && ic < g.npml + g.nz && jc >= g.npml &&
         jc < g.npml + g.nx;
    if (ok) {
      box[2 * s] = ic;
      box[2 * s + 1] = jc;
      ws[0] = (float)(1.0 / ((double)dx * (double)dz));
    }
  } else {
    ok = isfinite(xr) && isfinite(zr) && ic - 3 >= 0 && ic + 3 < g.Nz && jc - 3 >= 0 && jc + 3 < g.Nx;
    if (ok) {
      box[2 * s] = ic - 3;
      box[2 * s + 1] = jc - 3;
      const double sg = 0.5 * (double)dx;
      for (int di = 0; di < SRC_W; di++)
        for (int dj = 0; dj < SRC_W; dj++) {
          const double xi = (double)(jc - 3 + dj - g.npml) * dx - xr;
          const double zi = (double)(ic - 3 + di - g.npml) * dz - zr;
          ws[di * SRC_W + dj] = (float)(exp(-(xi * xi + zi * zi) / (2.0 * sg * sg)) / (2.0 * M_PI * sg * sg));
        }
    }
  }
  if (!ok) {
    box[2 * s] = -1;
    box[2 * s + 1] = -1;
    atomicOr(status, ST_BADSRC);
  }
}

// Receiver cells and receiver lists per owning thread (one block of 1024
// threads). The step kernels give the 2 x 4 cells (rows 2ty..2ty+1, columns
// 4tx..4tx+3) of a 64 x 32 tile to thread ty*16 + tx, so a receiver belongs to
// key = (tile of one shot) * NTHREADS + thread; an entry packs the receiver
// index with the row and column inside that thread's cells. Receivers outside
// the physical grid are flagged and listed nowhere. Buckets are sorted by
// receiver index, so the result does not depend on atomic ordering.
__global__ void k_rec_csr(int nrec, const int* __restrict__ iz, const int* __restrict__ ix, Grid g,
                          int* rec_cell, int* rec_key, int* start, int* cursor, int* list, int* status) {
  __shared__ int ssum[1024];
  const int nkeys = g.ntx * g.ntz * NTHREADS;
  for (int k = threadIdx.x; k <= nkeys; k += blockDim.x) start[k] = 0;
  for (int k = threadIdx.x; k < nkeys; k += blockDim.x) cursor[k] = 0;
  __syncthreads();
  for (int r = threadIdx.x; r < nrec; r += blockDim.x) {
    const int i = iz[r], j = ix[r];
    if (i >= 0 && i < g.nz && j >= 0 && j < g.nx) {
      const int pi = i + g.npml, pj = j + g.npml;
      rec_cell[2 * r] = pi;
      rec_cell[2 * r + 1] = pj;
      const int lr = pi % TILE_Z, lc = pj % TILE_X;
      const int key = ((pi / TILE_Z) * g.ntx + pj / TILE_X) * NTHREADS + (lr >> 1) * 16 + (lc >> 2);
      rec_key[r] = key;
      atomicAdd(&start[key + 1], 1);
    } else {
      rec_cell[2 * r] = -1;
      rec_cell[2 * r + 1] = -1;
      rec_key[r] = -1;
      atomicOr(status, ST_BADREC);
    }
  }
  __syncthreads();
  // inclusive scan of start[1..nkeys]: per-thread chunk sums, then a scan of the sums
  const int chunk = (nkeys + blockDim.x - 1) / blockDim.x;
  const int lo = 1 + threadIdx.x * chunk, hi = min(nkeys + 1, lo + chunk);
  int acc = 0;
  for (int k = lo; k < hi; k++) acc += start[k];
  ssum[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int t = 1; t < (int)blockDim.x; t++) ssum[t] += ssum[t - 1];
  __syncthreads();
  int run = threadIdx.x == 0 ? 0 : ssum[threadIdx.x - 1];
  for (int k = lo; k < hi; k++) {
    run += start[k];
    start[k] = run;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < nrec; r += blockDim.x) {
    const int key = rec_key[r];
    if (key < 0) continue;
    const int pi = rec_cell[2 * r], pj = rec_cell[2 * r + 1];
    const int code = (r << 3) | (((pi % TILE_Z) & 1) << 2) | ((pj % TILE_X) & 3);
    list[start[key] + atomicAdd(&cursor[key], 1)] = code;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nkeys; k += blockDim.x) {
    const int b = start[k], e = start[k + 1];
    for (int a = b + 1; a < e; a++) {  // insertion sort of a (tiny) bucket
      const int v = list[a];
      int q = a - 1;
      while (q >= b && list[q] > v) {
        list[q + 1] = list[q];
        q--;
      }
      list[q + 1] = v;
    }
  }
}

// CFL: c_max dt sqrt(1/dx^2 + 1/dz^2) sum|a_k| <= 1, and c finite and > 0.
__global__ void k_model_check(const float* __restrict__ c, long long n, float coef, int* status) {
  __shared__ float smax[1024 / 32];
  __shared__ int sbad;
  if (threadIdx.x == 0) sbad = 0;
  __syncthreads();
  float mx = 0.f;
  int bad = 0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) {
    const float v = c[i];
    if (!(v > 0.f) || !isfinite(v)) bad = 1;
    else mx = fmaxf(mx, v);
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

// Residual r = d - d_obs (in place over the observed copy) and per-block
// FP64 partial sums of r^2 (fixed reduction tree: deterministic).
// VJP: the buffer already holds the cotangent v = dL/dd, which is the adjoint
// source as it stands (it is left unchanged); the partial sums are of d * v,
// so the scalar returned is <d, v>, the functional whose gradient the adjoint
// sweep then computes.
template <bool VJP>
__global__ void k_misfit(const float* __restrict__ seis, float* res, long long n, double* part) {
  __shared__ double sred[256 / 32];
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    if (VJP) {
      acc += (double)seis[i] * (double)res[i];
    } else {
      const float r = seis[i] - res[i];
      res[i] = r;
      acc += (double)r * (double)r;
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += sred[w];
    part[blockIdx.x] = s;
  }
}

// Superposed sources: r = sum_s d_s - d_obs over the S seismograms (summed in
// shot order), broadcast into cot[s] for every s (the adjoint source of each
// sub-source is the common residual), and per-block FP64 partial sums of r^2.
__global__ void k_superpose(const float* __restrict__ seis, int S, long long n, const float* __restrict__ obs,
                            float* __restrict__ cot, double* part) {
  __shared__ double sred[256 / 32];
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    float d = 0.f;
    for (int sh = 0; sh < S; sh++) d += seis[(long long)sh * n + i];
    const float r = d - obs[i];
    for (int sh = 0; sh < S; sh++) cot[(long long)sh * n + i] = r;
    acc += (double)r * (double)r;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) sum += sred[w];
    part[blockIdx.x] = sum;
  }
}

__global__ void k_misfit_final(const double* part, int nb, double scale, double* J, int* status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int b = 0; b < nb; b++) s += part[b];
  s *= scale;
  *J = s;
  if (!isfinite(s)) atomicOr(status, ST_NONFINITE);
}

__global__ void k_finite_check(const float* __restrict__ a, long long n, int* status) {
  int bad = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    if (!isfinite(a[i])) bad = 1;
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, ST_NONFINITE);
}

// Adjoint initial condition: lambda_{nt} = residual of the last sample at the
// receivers (in receiver order), and its source-parameter partial (index nt-1).
__global__ void k_adj_init(AcuStep p, float* lam, float* hx, float* hz, bool lap) {
  const int s = blockIdx.x;
  if (threadIdx.x != 0) return;
  const long long sh = (long long)s * p.g.slice + p.g.off0;
  for (int r = 0; r < p.nrec; r++) {
    const int ri = p.rec_cell[2 * r], rj = p.rec_cell[2 * r + 1];
    if (ri < 0) continue;
    const long long c = sh + (long long)ri * p.g.pitch + rj;
    const float rv = p.res[((long long)s * p.nrec + r) * p.nt + p.nt - 1];
    // hhat = lambda at a receiver (never inside the CPML layer); m lambda for the
    // Laplacian operator (m = 2 (m/2) at the cell)
    const float hv = lap ? 2.f * p.mh[p.g.off0 + (long long)ri * p.g.pitch + rj] * rv : rv;
    lam[c] += rv;
    hx[c] += hv;
    hz[c] += hv;
  }
  if (p.src_part == nullptr) return;
  const int i0 = p.src_box[2 * s], j0 = p.src_box[2 * s + 1], nb = p.src_n;
  float acc[3] = {0.f, 0.f, 0.f};
  if (i0 >= 0) {
    const float xs = p.x0[2 * s], zs = p.x0[2 * s + 1];
    for (int di = 0; di < nb; di++)
      for (int dj = 0; dj < nb; dj++) {
        const float l = lam[sh + (long long)(i0 + di) * p.g.pitch + j0 + dj];
        const float wl = p.src_w[s * SRC_W * SRC_W + di * SRC_W + dj] * l;
        acc[0] += wl;
        acc[1] += wl * ((float)(j0 + dj - p.g.npml) * p.dx - xs);
        acc[2] += wl * ((float)(i0 + di - p.g.npml) * p.dz - zs);
      }
  }
  float* dst = p.src_part + ((long long)s * p.nt + (p.nt - 1)) * SRC_SLOTS * 3;
  for (int q = 0; q < SRC_SLOTS * 3; q++) dst[q] = 0.f;
  dst[0] = acc[0];
  dst[1] = acc[1];
  dst[2] = acc[2];
}

// Segment fold: G (FP64, per padded cell) += sum over shots of the FP32
// segment partials (in shot order), which are reset for the next segment. A
// thread takes 4 consecutive cells (the slice is a multiple of 4 floats) and
// has the partials of 8 shots in flight before it adds them.
__global__ void k_fold(float* __restrict__ gpart, int S, long long slice, double* __restrict__ G) {
  const long long n4 = slice / 4;
  float4* __restrict__ p4 = reinterpret_cast<float4*>(gpart);
  double2* __restrict__ G2 = reinterpret_cast<double2*>(G);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4;
       i += (long long)gridDim.x * blockDim.x) {
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    for (int s0 = 0; s0 < S; s0 += 8) {
      const int m = min(8, S - s0);
      float4 v[8];
#pragma unroll
      for (int u = 0; u < 8; u++)
        if (u < m) v[u] = p4[(long long)(s0 + u) * n4 + i];
#pragma unroll
      for (int u = 0; u < 8; u++)
        if (u < m) {
          a0 += (double)v[u].x;
          a1 += (double)v[u].y;
          a2 += (double)v[u].z;
          a3 += (double)v[u].w;
          p4[(long long)(s0 + u) * n4 + i] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    double2 g0 = G2[2 * i], g1 = G2[2 * i + 1];
    g0.x += a0;
    g0.y += a1;
    g1.x += a2;
    g1.y += a3;
    G2[2 * i] = g0;
    G2[2 * i + 1] = g1;
  }
}

// dJ/dc = 2 c dJ/dm = c G, where G holds 2 dJ/dm (the step kernels add each
// half-point correlation to both neighbours without the factor 1/2) and a
// physical cell also collects the CPML cells that replicate it (transpose of
// the edge padding).
__global__ void k_grad_c(const double* __restrict__ G, Grid g, const float* __restrict__ c,
                         float* grad) {
  const long long n = (long long)g.nz * g.nx;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const int iz = (int)(idx / g.nx), ix = (int)(idx - (long long)iz * g.nx);
    const int i_lo = iz == 0 ? 0 : iz + g.npml;
    const int i_hi = iz == g.nz - 1 ? g.Nz - 1 : iz + g.npml;
    const int j_lo = ix == 0 ? 0 : ix + g.npml;
    const int j_hi = ix == g.nx - 1 ? g.Nx - 1 : ix + g.npml;
    double acc = 0.0;
    for (int i = i_lo; i <= i_hi; i++)
      for (int j = j_lo; j <= j_hi; j++) acc += G[g.off0 + (long long)i * g.pitch + j];
    grad[idx] = (float)((double)c[idx] * acc);
  }
}

// Source-parameter gradients from the per-step partials (nslots per step,
// each (sum w a, sum w a (x_i - x0), sum w a (z_i - z0)) of the adjoint field
// a at the source support): dJ/dg(t_n) = scale * sum_slots part0, and for
// Gaussian sources dJ/dx0 = sum_n g(t_n) scale sum_slots part1 / s^2 (z alike).
// Acoustic: scale = dt^2 (a = lambda_{n+1}); elastic: scale = -dt (a = M : sigma-bar^{n+1}).
__global__ void k_src_grad(const float* __restrict__ part, int S, int nt, int nslots, double scale,
                           const float* __restrict__ stf, double inv_sig2, int kind, float* gstf, float* gx0) {
  __shared__ double sred[256 / 32][2];
  const int s = blockIdx.x;
  double ax = 0.0, az = 0.0;
  for (int n = threadIdx.x; n < nt; n += blockDim.x) {
    const float* q = part + ((long long)s * nt + n) * nslots * 3;
    double w0 = 0.0, w1 = 0.0, w2 = 0.0;
    for (int k = 0; k < nslots; k++) {
      w0 += q[3 * k];
      w1 += q[3 * k + 1];
      w2 += q[3 * k + 2];
    }
    if (gstf) gstf[(long long)s * nt + n] = (float)(scale * w0);
    const double g = stf[(long long)s * nt + n];
    ax += g * scale * w1 * inv_sig2;
    az += g * scale * w2 * inv_sig2;
  }
  for (int o = 16; o > 0; o >>= 1) {
    ax += __shfl_xor_sync(0xffffffffu, ax, o);
    az += __shfl_xor_sync(0xffffffffu, az, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sred[threadIdx.x >> 5][0] = ax;
    sred[threadIdx.x >> 5][1] = az;
  }
  __syncthreads();
  if (threadIdx.x == 0 && gx0) {
    double sx = 0.0, sz = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
      sx += sred[w][0];
      sz += sred[w][1];
    }
    gx0[2 * s] = kind == 1 ? (float)sx : 0.f;
    gx0[2 * s + 1] = kind == 1 ? (float)sz : 0.f;
  }
}

// ---------------------------------------------------------------------------
// launchers
// Line sources (the paper's plane-wave sources: a row of L cells, each firing
// its own time function amp[s][n][q] with weight 1/(dx dz)). The step kernels
// see no source box for them (box = -1); the line is injected by its own small
// kernel after each step and read back by another after each adjoint step.
//
// k_line_prep: padded (row, first column) of each shot's line from x0 = (x of
// the first cell, z of the row) in metres; every cell must be physical.
__global__ void k_line_prep(int S, int L, const float* __restrict__ x0, Grid g, float dx, float dz, int* line_cell,
                            int* box, int* status) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  const double xr = x0[2 * s], zr = x0[2 * s + 1];
  const int j0 = (int)llround(xr / (double)dx) + g.npml;
  const int i0 = (int)llround(zr / (double)dz) + g.npml;
  const bool ok = isfinite(xr) && isfinite(zr) && i0 >= g.npml && i0 < g.npml + g.nz && j0 >= g.npml &&
                  j0 + L <= g.npml + g.nx;
  line_cell[2 * s] = ok ? i0 : -1;
  line_cell[2 * s + 1] = ok ? j0 : -1;
  box[2 * s] = -1;  // no box source for the step kernels
  box[2 * s + 1] = -1;
  if (!ok) atomicOr(status, ST_BADSRC);
}

// u^{n+1}(row, j0 + q) += scale * amp[s][n][q] for the S shots of a group
// (shot s of the group at u + s * slice); with `seis`, the samples already
// recorded from those cells at step n get the same increment (a receiver on
// the line records u^{n+1} with its source term, as the recursion defines it).
__global__ void k_line_inject(int S, int L, int n, int nt, float scale, const float* __restrict__ amp,
                              const int* __restrict__ line_cell, float* u, long long slice, long long off0, int pitch,
                              const int* __restrict__ rec_cell, int nrec, float* seis) {
  const int s = blockIdx.y;
  const int i0 = line_cell[2 * s], j0 = line_cell[2 * s + 1];
  if (i0 < 0) return;
  const float* a = amp + ((long long)s * nt + n) * L;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < L + (seis ? nrec : 0); k += gridDim.x * blockDim.x) {
    if (k < L) {
      u[(long long)s * slice + off0 + (long long)i0 * pitch + j0 + k] += scale * a[k];
    } else {
      const int r = k - L, ri = rec_cell[2 * r], rj = rec_cell[2 * r + 1];
      if (ri == i0 && rj >= j0 && rj < j0 + L) seis[((long long)s * nrec + r) * nt + n] += scale * a[rj - j0];
    }
  }
}

// gamp[s][n][q] = scale * lambda(row, j0 + q): the derivative of the misfit with
// respect to amp[s][n][q] (lambda the adjoint of u^{n+1}, complete).
__global__ void k_line_grad(int S, int L, int n, int nt, float scale, const int* __restrict__ line_cell,
                            const float* __restrict__ lam, long long slice, long long off0, int pitch, float* gamp) {
  const int s = blockIdx.y;
  const int i0 = line_cell[2 * s], j0 = line_cell[2 * s + 1];
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < L; k += gridDim.x * blockDim.x)
    gamp[((long long)s * nt + n) * L + k] =
        i0 < 0 ? 0.f : scale * lam[(long long)s * slice + off0 + (long long)i0 * pitch + j0 + k];
}

cudaError_t launch_pad_model(const float* c, const Grid& g, float* m, cudaStream_t st) {
  k_pad_model_sq<<<304, 256, 0, st>>>(c, g, m);
  return cudaGetLastError();
}
cudaError_t launch_cpml_tables(int n_phys, int npml, int Npad, int len, double h, double dt, double R,
                               double vmax, double f0, float* a, float* b, float* ah, float* bh,
                               cudaStream_t st) {
  k_cpml_tables<<<(len + 255) / 256, 256, 0, st>>>(n_phys, npml, Npad, len, h, dt, R, vmax, f0, a, b, ah, bh);
  return cudaGetLastError();
}
cudaError_t launch_line_prep(int S, int L, const float* x0, const Grid& g, float dx, float dz, int* line_cell,
                             int* box, int* status, cudaStream_t st) {
  k_line_prep<<<(S + 127) / 128, 128, 0, st>>>(S, L, x0, g, dx, dz, line_cell, box, status);
  return cudaGetLastError();
}
cudaError_t launch_line_inject(int S, int L, int n, int nt, float scale, const float* amp, const int* line_cell,
                               float* u, const Grid& g, const int* rec_cell, int nrec, float* seis, cudaStream_t st) {
  const int work = L + (seis ? nrec : 0);
  k_line_inject<<<dim3((work + 255) / 256, S), 256, 0, st>>>(S, L, n, nt, scale, amp, line_cell, u, g.slice, g.off0,
                                                           g.pitch, rec_cell, nrec, seis);
  return cudaGetLastError();
}
cudaError_t launch_line_grad(int S, int L, int n, int nt, float scale, const int* line_cell, const float* lam,
                             const Grid& g, float* gamp, cudaStream_t st) {
  k_line_grad<<<dim3((L + 255) / 256, S), 256, 0, st>>>(S, L, n, nt, scale, line_cell, lam, g.slice, g.off0, g.pitch,
                                                       gamp);
  return cudaGetLastError();
}
cudaError_t launch_src_prep(int S, int kind, const float* x0, const Grid& g, float dx, float dz, int* box,
                            float* w, int* status, cudaStream_t st) {
  k_src_prep<<<(S + 127) / 128, 128, 0, st>>>(S, kind, x0, g, dx, dz, box, w, status);
  return cudaGetLastError();
}
cudaError_t launch_rec_csr(int nrec, const int* iz, const int* ix, const Grid& g, int* rec_cell, int* rec_key,
                           int* start, int* cursor, int* list, int* status, cudaStream_t st) {
  k_rec_csr<<<1, 1024, 0, st>>>(nrec, iz, ix, g, rec_cell, rec_key, start, cursor, list, status);
  return cudaGetLastError();
}
cudaError_t launch_model_check(const float* c, long long n, float coef, int* status, cudaStream_t st) {
  k_model_check<<<1, 1024, 0, st>>>(c, n, coef, status);
  return cudaGetLastError();
}
cudaError_t launch_misfit(const float* seis, float* res, long long n, double* part, int nb, double* J,
                          int* status, bool vjp, cudaStream_t st) {
  if (vjp) k_misfit<true><<<nb, 256, 0, st>>>(seis, res, n, part);
  else k_misfit<false><<<nb, 256, 0, st>>>(seis, res, n, part);
  k_misfit_final<<<1, 32, 0, st>>>(part, nb, vjp ? 1.0 : 0.5, J, status);
  return cudaGetLastError();
}
cudaError_t launch_superpose(const float* seis, int S, long long n, const float* obs, float* cot, double* part,
                             int nb, double* J, int* status, cudaStream_t st) {
  k_superpose<<<nb, 256, 0, st>>>(seis, S, n, obs, cot, part);
  k_misfit_final<<<1, 32, 0, st>>>(part, nb, 0.5, J, status);
  return cudaGetLastError();
}
cudaError_t launch_finite_check(const float* a, long long n, int* status, cudaStream_t st) {
  k_finite_check<<<304, 256, 0, st>>>(a, n, status);
  return cudaGetLastError();
}
cudaError_t launch_adj_init(const AcuStep& p, float* lam, float* hx, float* hz, cudaStream_t st, bool lap) {
  k_adj_init<<<p.S, 32, 0, st>>>(p, lam, hx, hz, lap);
  return cudaGetLastError();
}
// Copies of a descriptor table: block row y copies descriptor y.
__global__ void k_copy_table(const CopyDesc* __restrict__ d) {
  const CopyDesc c = d[blockIdx.y];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < c.n4; i += (long long)gridDim.x * blockDim.x)
    c.dst[i] = c.src[i];
}
cudaError_t launch_copy_table(const CopyDesc* d, int n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_copy_table<<<dim3(64, n), 256, 0, st>>>(d);
  return cudaGetLastError();
}
cudaError_t launch_fold(float* gpart, int S, long long slice, double* G, cudaStream_t st) {
  k_fold<<<608, 256, 0, st>>>(gpart, S, slice, G);
  return cudaGetLastError();
}
cudaError_t launch_grad_c(const double* G, const Grid& g, const float* c, float* grad, cudaStream_t st) {
  k_grad_c<<<304, 256, 0, st>>>(G, g, c, grad);
  return cudaGetLastError();
}
cudaError_t launch_src_grad(const float* part, int S, int nt, int nslots, double scale, const float* stf,
                            double inv_sig2, int kind, float* gstf, float* gx0, cudaStream_t st) {
  k_src_grad<<<S, 256, 0, st>>>(part, S, nt, nslots, scale, stf, inv_sig2, kind, gstf, gx0);
  return cudaGetLastError();
}

}  // namespace fwi
