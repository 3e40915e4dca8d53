// acoustic_lap.cu - the acoustic recursion with the c^2 Laplacian operator,
// u_tt = c^2 (D-x (D+x u + psi_x) + zeta_x + D-z (D+z u + psi_z) + zeta_z) + f,
// beside the paper's divergence form div(c^2 grad u) (Implementation, Eq.
// acoustic) of acoustic_kernels.cu: the same staggered first derivatives and
// CPML, with the coefficient m = c^2 multiplying the whole operator at the cell
// instead of the fluxes at the half points. One forward step is two plain
// kernels (fluxes at the half points, then the update at the cells) and one
// adjoint step three (the transpose of the update, of the fluxes, and of the
// divergence), each thread owning one point; the gradient correlation is
// dJ/dm += dt^2 lambda_{n+1} r^n at the cells, with r^n stored by the recompute.
// These kernels favour plainness over speed: the divergence form is the path
// the library optimises.
//
// Layout as every field of the library: [shot][rows][pitch] with a zero apron,
// cell (i, j) of shot s at s*slice + off0 + i*pitch + j. Grids: blockIdx.z =
// shot, blockIdx.y = row, threads along the row.
#include <cuda_runtime.h>

#include "fwi_internal.cuh"

namespace fwi {

struct LapStep {
  Grid g;
  int N;
  float c1x[4], c1z[4];  // a_k / dx, a_k / dz
  float dt2;
  const float* mh;  // c^2 / 2 at the cells (the library's padded coefficient field)
  const float *ax, *bx, *axh, *bxh, *az, *bz, *azh, *bzh;  // CPML tables, indexed [h + TAB_OFF]
};

namespace {

__device__ __forceinline__ long long cell_index(const Grid& g, int s, int i, int j) {
  return (long long)s * g.slice + g.off0 + (long long)i * g.pitch + j;
}

// p = D+u + psi at the half points (i, j+1/2) and (i+1/2, j), psi updated in
// place; zero at the half points outside [0, N-1).
template <int N>
__global__ void k_lap_flux(const LapStep p, const float* __restrict__ u, float* psix, float* psiz, float* qx,
                           float* qz) {
  const Grid& g = p.g;
  const int s = blockIdx.z, i = blockIdx.y, j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= g.Nx) return;
  const long long id = cell_index(g, s, i, j);
  float vx = 0.f, vz = 0.f;
  if (j < g.Nx - 1) {
    float d = 0.f;
#pragma unroll
    for (int k = 1; k <= N; k++) d += p.c1x[k - 1] * (u[id + k] - u[id - k + 1]);
    const float ps = p.bxh[j + TAB_OFF] * psix[id] + p.axh[j + TAB_OFF] * d;
    psix[id] = ps;
    vx = d + ps;
  }
  if (i < g.Nz - 1) {
    float d = 0.f;
#pragma unroll
    for (int k = 1; k <= N; k++) d += p.c1z[k - 1] * (u[id + (long long)k * g.pitch] - u[id - (long long)(k - 1) * g.pitch]);
    const float ps = p.bzh[i + TAB_OFF] * psiz[id] + p.azh[i + TAB_OFF] * d;
    psiz[id] = ps;
    vz = d + ps;
  }
  qx[id] = vx;
  qz[id] = vz;
}

// r = D-x qx + zeta_x + D-z qz + zeta_z (zeta updated in place);
// u^{n+1} = 2 u^n - u^{n-1} + dt^2 m r + dt^2 w g(t_n), written over u^{n-1};
// rstore (if not null) keeps r for the gradient.
template <int N>
__global__ void k_lap_update(const LapStep p, const float* __restrict__ u, float* uprev, const float* __restrict__ qx,
                             const float* __restrict__ qz, float* zetx, float* zetz, const int* __restrict__ box,
                             const float* __restrict__ w, int nb, const float* __restrict__ stf, int nt, int n,
                             float* rstore) {
  const Grid& g = p.g;
  const int s = blockIdx.z, i = blockIdx.y, j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= g.Nx) return;
  const long long id = cell_index(g, s, i, j);
  float hx = 0.f, hz = 0.f;
#pragma unroll
  for (int k = 1; k <= N; k++) {
    hx += p.c1x[k - 1] * (qx[id + k - 1] - qx[id - k]);
    hz += p.c1z[k - 1] * (qz[id + (long long)(k - 1) * g.pitch] - qz[id - (long long)k * g.pitch]);
  }
  const float zx = p.bx[j + TAB_OFF] * zetx[id] + p.ax[j + TAB_OFF] * hx;
  const float zz = p.bz[i + TAB_OFF] * zetz[id] + p.az[i + TAB_OFF] * hz;
  zetx[id] = zx;
  zetz[id] = zz;
  const float r = hx + zx + hz + zz;
  if (rstore) rstore[id] = r;
  float v = 2.f * u[id] - uprev[id] + p.dt2 * (2.f * p.mh[id - (long long)s * g.slice]) * r;
  const int i0 = box[2 * s], j0 = box[2 * s + 1];
  if (i0 >= 0 && i >= i0 && i < i0 + nb && j >= j0 && j < j0 + nb)
    v += p.dt2 * stf[(long long)s * nt + n] * w[s * SRC_W * SRC_W + (i - i0) * SRC_W + (j - j0)];
  uprev[id] = v;
}

// seis[s][r][n] = u^{n+1}(receiver cell r), one thread per (shot, receiver)
__global__ void k_lap_record(const float* __restrict__ u, const Grid g, int S, int nrec, int nt, int n,
                             const int* __restrict__ rec_cell, float* seis) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= S * nrec) return;
  const int s = k / nrec, r = k - s * nrec;
  const int i = rec_cell[2 * r], j = rec_cell[2 * r + 1];
  seis[((long long)s * nrec + r) * nt + n] = i < 0 ? 0.f : u[cell_index(g, s, i, j)];  // -1: outside the grid
}

// lam(receiver cell r) += res[s][r][n], one thread per (receiver, shot): the
// residual of sample n enters lambda_{n+1} (the adjoint seed, and the adjoint
// sweep's source). Receivers that share a cell are added by the first of them, in receiver
// order, so the sum is the sequential one and the kernel deterministic. The
// block scans the receiver cells in ascending chunks staged in shared memory:
// every earlier receiver is seen before any later one. Receivers outside the
// grid (cell -1, reported through the status word) are skipped.
constexpr int INJ_THREADS = 128;
__global__ void __launch_bounds__(INJ_THREADS) k_lap_inject_res(float* lam, const Grid g, int S, int nrec, int nt,
                                                                int n, const int* __restrict__ rec_cell,
                                                                const float* __restrict__ res) {
  __shared__ int2 cells[INJ_THREADS];
  const int s = blockIdx.y, r = blockIdx.x * INJ_THREADS + threadIdx.x;
  const int2* rc = reinterpret_cast<const int2*>(rec_cell);
  const int2 c = r < nrec ? rc[r] : make_int2(-1, -1);
  bool first = c.x >= 0;
  const float* rs = res + (long long)s * nrec * nt + n;
  const long long id = first ? cell_index(g, s, c.x, c.y) : 0;
  float v = first ? lam[id] + rs[(long long)r * nt] : 0.f;
  for (int q0 = 0; q0 < nrec; q0 += INJ_THREADS) {
    __syncthreads();  // the previous chunk is no longer read
    if (q0 + (int)threadIdx.x < nrec) cells[threadIdx.x] = rc[q0 + threadIdx.x];
    __syncthreads();
    const int m = min(INJ_THREADS, nrec - q0);
    for (int t = 0; t < m; t++) {
      const int2 o = cells[t];
      if (o.x == c.x && o.y == c.y) {
        const int q = q0 + t;
        if (q < r) first = false;                      // an earlier receiver adds this cell's samples
        else if (q > r && first) v += rs[(long long)q * nt];
      }
    }
  }
  if (first) lam[id] = v;
}

// Adjoint of the update at the cells, given lambda_{n+1} (complete):
//   dJ/dm += dt^2 lambda r^n (the FP32 partial holds 2 dJ/dm),
//   rbar = dt^2 m lambda; hbar = rbar + a (Z + rbar), Z <- b (Z + rbar) per axis.
__global__ void k_lap_adj_update(const LapStep p, const float* __restrict__ lam1, const float* __restrict__ rst,
                                 float* gpart, float* Zx, float* Zz, float* hbx, float* hbz) {
  const Grid& g = p.g;
  const int s = blockIdx.z, i = blockIdx.y, j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= g.Nx) return;
  const long long id = cell_index(g, s, i, j);
  const float l = lam1[id];
  gpart[id] += 2.f * p.dt2 * l * rst[id];
  const float rb = p.dt2 * (2.f * p.mh[id - (long long)s * g.slice]) * l;
  float t = Zx[id] + rb;
  hbx[id] = rb + p.ax[j + TAB_OFF] * t;
  Zx[id] = p.bx[j + TAB_OFF] * t;
  t = Zz[id] + rb;
  hbz[id] = rb + p.az[i + TAB_OFF] * t;
  Zz[id] = p.bz[i + TAB_OFF] * t;
}

// Adjoint of the divergence and of the fluxes at the half points:
//   qbar = -D+ hbar, gbar = qbar + a_h (P + qbar), P <- b_h (P + qbar); zero outside [0, N-1).
template <int N>
__global__ void k_lap_adj_flux(const LapStep p, const float* __restrict__ hbx, const float* __restrict__ hbz,
                               float* Px, float* Pz, float* gbx, float* gbz) {
  const Grid& g = p.g;
  const int s = blockIdx.z, i = blockIdx.y, j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= g.Nx) return;
  const long long id = cell_index(g, s, i, j);
  float vx = 0.f, vz = 0.f;
  if (j < g.Nx - 1) {
    float q = 0.f;
#pragma unroll
    for (int k = 1; k <= N; k++) q += p.c1x[k - 1] * (hbx[id - k + 1] - hbx[id + k]);
    const float t = Px[id] + q;
    vx = q + p.axh[j + TAB_OFF] * t;
    Px[id] = p.bxh[j + TAB_OFF] * t;
  }
  if (i < g.Nz - 1) {
    float q = 0.f;
#pragma unroll
    for (int k = 1; k <= N; k++) q += p.c1z[k - 1] * (hbz[id - (long long)(k - 1) * g.pitch] - hbz[id + (long long)k * g.pitch]);
    const float t = Pz[id] + q;
    vz = q + p.azh[i + TAB_OFF] * t;
    Pz[id] = p.bzh[i + TAB_OFF] * t;
  }
  gbx[id] = vx;
  gbz[id] = vz;
}

// lambda_n = 2 lambda_{n+1} - lambda_{n+2} + D+^T gbar, written over lambda_{n+2}
template <int N>
__global__ void k_lap_adj_lambda(const LapStep p, const float* __restrict__ lam1, float* lam2,
                                 const float* __restrict__ gbx, const float* __restrict__ gbz) {
  const Grid& g = p.g;
  const int s = blockIdx.z, i = blockIdx.y, j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= g.Nx) return;
  const long long id = cell_index(g, s, i, j);
  float acc = 0.f;
#pragma unroll
  for (int k = 1; k <= N; k++) {
    acc += p.c1x[k - 1] * (gbx[id - k] - gbx[id + k - 1]);
    acc += p.c1z[k - 1] * (gbz[id - (long long)k * g.pitch] - gbz[id + (long long)(k - 1) * g.pitch]);
  }
  lam2[id] = 2.f * lam1[id] - lam2[id] + acc;
}

// Source partials of time index n from lambda_{n+1} over the box: slot 0 of
// part[s][n] gets (sum w lambda, sum w lambda (x_i - x0), sum w lambda (z_i - z0)).
__global__ void k_lap_src_part(const float* __restrict__ lam1, const Grid g, int S, int nt, int n,
                               const int* __restrict__ box, const float* __restrict__ w, int nb,
                               const float* __restrict__ x0, float dx, float dz, float* part) {
  const int s = blockIdx.x;
  const int i0 = box[2 * s], j0 = box[2 * s + 1];
  float a[3] = {0.f, 0.f, 0.f};
  if (i0 >= 0) {
    for (int q = threadIdx.x; q < nb * nb; q += 32) {
      const int di = q / nb, dj = q - di * nb;
      const float wl = w[s * SRC_W * SRC_W + di * SRC_W + dj] * lam1[cell_index(g, s, i0 + di, j0 + dj)];
      a[0] += wl;
      a[1] += wl * ((float)(j0 + dj - g.npml) * dx - x0[2 * s]);
      a[2] += wl * ((float)(i0 + di - g.npml) * dz - x0[2 * s + 1]);
    }
  }
  for (int k = 0; k < 3; k++)
    for (int o = 16; o > 0; o >>= 1) a[k] += __shfl_xor_sync(0xffffffffu, a[k], o);
  if (threadIdx.x == 0)
    for (int k = 0; k < 3; k++) part[(((long long)s * nt + n) * SRC_SLOTS + 0) * 3 + k] = a[k];
}

dim3 grid_of(const Grid& g, int S) { return dim3((unsigned)((g.Nx + 127) / 128), (unsigned)g.Nz, (unsigned)S); }

}  // namespace

cudaError_t launch_lap_forward_step(const LapStep& p, int S, const float* u, float* uprev, float* psix, float* psiz,
                                    float* qx, float* qz, float* zetx, float* zetz, const int* box, const float* w,
                                    int nb, const float* stf, int nt, int n, float* rstore, cudaStream_t st) {
  if (p.N == 2) {
    k_lap_flux<2><<<grid_of(p.g, S), 128, 0, st>>>(p, u, psix, psiz, qx, qz);
    k_lap_update<2><<<grid_of(p.g, S), 128, 0, st>>>(p, u, uprev, qx, qz, zetx, zetz, box, w, nb, stf, nt, n, rstore);
  } else {
    k_lap_flux<4><<<grid_of(p.g, S), 128, 0, st>>>(p, u, psix, psiz, qx, qz);
    k_lap_update<4><<<grid_of(p.g, S), 128, 0, st>>>(p, u, uprev, qx, qz, zetx, zetz, box, w, nb, stf, nt, n, rstore);
  }
  return cudaGetLastError();
}
cudaError_t launch_lap_record(const float* u, const Grid& g, int S, int nrec, int nt, int n, const int* rec_cell,
                              float* seis, cudaStream_t st) {
  if (S * nrec == 0) return cudaSuccess;
  k_lap_record<<<(S * nrec + 127) / 128, 128, 0, st>>>(u, g, S, nrec, nt, n, rec_cell, seis);
  return cudaGetLastError();
}
cudaError_t launch_lap_inject_res(float* lam, const Grid& g, int S, int nrec, int nt, int n, const int* rec_cell,
                                  const float* res, cudaStream_t st) {
  if (S * nrec == 0) return cudaSuccess;
  k_lap_inject_res<<<dim3((unsigned)((nrec + INJ_THREADS - 1) / INJ_THREADS), (unsigned)S), INJ_THREADS, 0, st>>>(
      lam, g, S, nrec, nt, n, rec_cell, res);
  return cudaGetLastError();
}
cudaError_t launch_lap_adjoint_step(const LapStep& p, int S, const float* lam1, float* lam2, const float* rst,
                                    float* gpart, float* Zx, float* Zz, float* Px, float* Pz, float* hbx, float* hbz,
                                    float* gbx, float* gbz, cudaStream_t st) {
  k_lap_adj_update<<<grid_of(p.g, S), 128, 0, st>>>(p, lam1, rst, gpart, Zx, Zz, hbx, hbz);
  if (p.N == 2) {
    k_lap_adj_flux<2><<<grid_of(p.g, S), 128, 0, st>>>(p, hbx, hbz, Px, Pz, gbx, gbz);
    k_lap_adj_lambda<2><<<grid_of(p.g, S), 128, 0, st>>>(p, lam1, lam2, gbx, gbz);
  } else {
    k_lap_adj_flux<4><<<grid_of(p.g, S), 128, 0, st>>>(p, hbx, hbz, Px, Pz, gbx, gbz);
    k_lap_adj_lambda<4><<<grid_of(p.g, S), 128, 0, st>>>(p, lam1, lam2, gbx, gbz);
  }
  return cudaGetLastError();
}
cudaError_t launch_lap_src_part(const float* lam1, const Grid& g, int S, int nt, int n, const int* box,
                                const float* w, int nb, const float* x0, float dx, float dz, float* part,
                                cudaStream_t st) {
  k_lap_src_part<<<S, 32, 0, st>>>(lam1, g, S, nt, n, box, w, nb, x0, dx, dz, part);
  return cudaGetLastError();
}

}  // namespace fwi
