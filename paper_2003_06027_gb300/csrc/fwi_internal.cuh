// fwi_internal.cuh - device-side layout and parameter blocks shared by the
// kernels of libfwi (not part of the public ABI).
//
// HBM layout of every per-shot field (wavefields, CPML memory variables,
// gradient partials, stored fluxes): [shot][rows][pitch] FP32 with a zero
// apron of APRON cells on every side, so that the halo of a tile is always
// inside the allocation (TMA boxes and float4 loads need no bounds checks).
// Cell (i, j) of the padded grid (physical + CPML) of shot s lives at
//   base + s*slice + off0 + i*pitch + j,   off0 = APRON*pitch + APRON.
// Rows are padded to a multiple of the tile height and pitch to a multiple
// of the tile width; cells outside the padded grid are never written.
#pragma once
#include <cuda.h>
#include <cstdint>

namespace fwi {

constexpr int APRON = 8;     // >= stencil radius 2N-1 (7 at 8th order), float4 aligned
constexpr int TILE_X = 64;   // cells per tile along x (16 threads x float4)
constexpr int TILE_Z = 32;   // rows per tile (16 threads x 2 rows)
constexpr int NTHREADS = 256;
constexpr int TAB_OFF = 8;   // 1D CPML tables are indexed [h + TAB_OFF]
constexpr int SRC_W = 7;     // Gaussian source support (7 x 7)
constexpr int SRC_SLOTS = 4; // a 7 x 7 box touches at most 2 x 2 tiles
// Rows of the acoustic field layout are padded to a multiple of the tallest
// tile of its step kernels (the forward step also runs on 64 x 64 tiles), so
// that every tile of either height, with its halo, lies inside the allocation.
constexpr int ROW_ALIGN = 64;

// status bits written by device kernels
enum : int { ST_CFL = 1, ST_BADREC = 2, ST_BADSRC = 4, ST_NONFINITE = 8, ST_BADMODEL = 16, ST_TIMEOUT = 32 };

struct Grid {
  int nz, nx, npml;   // physical grid and CPML width
  int Nz, Nx;         // padded grid
  int ntx, ntz;       // tiles
  int pitch;          // floats per row
  int rows;           // allocated rows per shot
  long long slice;    // floats per shot per field
  long long off0;     // offset of padded cell (0,0)
};

// L2 policy for data that is streamed once per sweep (the segment slots: written
// by the recompute step, read back once by the adjoint step): such lines are
// evicted first, so they do not push the step's resident fields (wavefield
// pairs, gradient partials, CPML memory) out of L2.
__device__ __forceinline__ uint64_t l2_evict_first() {
  uint64_t pol;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ float4 ld4_stream(const float* ptr, uint64_t pol) {
  float4 v;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
      : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
      : "l"(ptr), "l"(pol));
  return v;
}
__device__ __forceinline__ void st4_stream(float* ptr, float4 v, uint64_t pol) {
  asm volatile("st.global.L1::no_allocate.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(ptr), "f"(v.x),
               "f"(v.y), "f"(v.z), "f"(v.w), "l"(pol));  // no later reader in the same kernel
}

// Tile t of a persistent walk over all shots: t = (s * ntz + tz) * ntx + tx.
struct TileId {
  int s, x0, z0, tx, tz;
};
__device__ __forceinline__ TileId tile_decode(const Grid& g, int t) {
  TileId r;
  r.tx = t % g.ntx;
  const int q = t / g.ntx;
  r.tz = q % g.ntz;
  r.s = q / g.ntz;
  r.x0 = r.tx * TILE_X;
  r.z0 = r.tz * TILE_Z;
  return r;
}

// TMA descriptors of one elastic call: 3D maps over [S][rows][pitch] of each
// field, with the box each kernel stages.
struct EleMaps {
  CUtensorMap sxx, szz, sxz, vx, vz;   // forward fields
  CUtensorMap Sxx, Szz, Sxz, Vx, Vz;   // adjoint fields
};

// TMA descriptors of one call: the wavefield pair [2][S] (forward), the
// half-coefficient field m/2, and the adjoint operand pairs [2][S].
struct AcuMaps {
  CUtensorMap u;
  CUtensorMap m;
  CUtensorMap u64, m64;  // the same fields with the boxes of 64-row forward tiles
  CUtensorMap lx, lz;   // adjoint: lambda pair, x-operand and z-operand boxes
  CUtensorMap hx, hz;   // adjoint: hhat pairs (CPML tiles)
};

// Everything one acoustic step kernel needs (passed by value).
struct AcuStep {
  Grid g;
  int S, N, n, nt, nrec;   // S: shots of this launch (one shot group)
  int S_pair, s0;         // shots per half of the u / lambda pairs, and this group's first shot there
  int cur;                // pair index holding u^n (forward) or lambda_{n+1} (adjoint)
  int ntiles;             // S * ntx * ntz
  float c1x[4], c1z[4];   // stage-1 weights (flux):  fwd a_k/dx;  adj -a_k dt^2/dx
  float c2x[4], c2z[4];   // stage-2 weights (div.):  fwd a_k dt^2/dx;  adj a_k/dx
  float dt2;
  const float* mh;        // [slice] c^2 / 2, zero in the apron (m_half = mh_i + mh_{i+1})
  const float *ax, *bx, *axh, *bxh, *az, *bz, *azh, *bzh;  // CPML tables
  // forward state
  float* u;               // [2][S][slice]
  const float *psix_in, *psiz_in;
  float *psix_out, *psiz_out;
  float *zetx, *zetz;     // dt^2 * zeta, cell-local, updated in place
  // sources: box origin (padded cell indices) and weights, per shot
  const int* src_box;     // [S][2] (i0, j0), -1 if invalid
  const float* src_w;     // [S][49]
  int src_n;              // box side: 1 (point) or 7 (Gaussian)
  const float* stf;       // [S][nt]
  // receivers, indexed by the thread that owns their cell: key =
  // (tile of one shot) * NTHREADS + thread; entries (r << 3) | (row << 2) | column
  const int* thr_rec_start;   // [ntx * ntz * NTHREADS + 1]
  const int* thr_rec;         // [nrec]
  const int* rec_cell;        // [nrec][2] padded (i, j)
  float* seis;                // [S][nrec][nt]
  // fluxes of step n kept for the reverse sweep (STORE): p = D+u + psi
  float *slot_px, *slot_pz;
  // adjoint state
  float* lam;             // [2][S][slice]
  const float *zx_in, *zz_in, *px_in, *pz_in;   // Z (scaled by 1/dt^2) and P
  float *zx_out, *zz_out, *px_out, *pz_out;
  float *hx_out, *hz_out;  // hhat of the next (earlier) step, written near the CPML: [S][slice]
  const float* res;       // [S][nrec][nt] residual seis - observed
  float* gpart;           // [S][slice] FP32 partial of 2 dJ/dm per padded cell
  float* src_part;        // [S][nt][SRC_SLOTS][3]
  const float* x0;        // [S][2] metres (physical)
  float dx, dz;
  int* status;
};

// One inversion instance of a multi-instance launch (fwi_batch_*): one work
// table, in device memory, lists the tiles of every instance taking part, and
// each tile finds its instance here. `p` holds the instance's static step
// parameters (all shots, S_pair = S, s0 = 0); the fields that depend on the
// time step n (pair halves, segment slots) are filled in by the kernel from
// the buffers below. Instances of one launch share the discretisation (order,
// dx, dz, dt), so the stencil weights come from the launch arguments.
struct AcuInst {
  CUtensorMap mu, mm;          // forward: wavefield pair, m/2
  CUtensorMap lx, lz, hx, hz;  // adjoint operand maps (lambda pair, hhat pairs)
  AcuStep p;
  float *psix[2], *psiz[2];    // forward CPML memory pairs
  float *zx[2], *zz[2], *px[2], *pz[2];  // adjoint CPML memory pairs
  float *hxp, *hzp;            // hhat pairs [2][S][slice]
  float* slot;                 // [K][2][S][slice] stored fluxes of one segment
  long long field;             // S * slice
  int nt;                      // time steps of this instance
  int nlast;                   // first step of its last segment (the forward sweep stores from there on)
};

// Arguments of one multi-instance launch. Instances are sorted by nt (longest
// first), so the ones taking part in any step form a prefix [0, n_active).
struct BatchArgs {
  const AcuInst* inst;    // [n_inst] device table
  const int* tile_start;  // [n_inst + 1] first tile of each instance (S * ntx * ntz tiles each)
  int n_active;           // instances of this launch
  int ntiles;             // tile_start[n_active]
  int n;                  // time step
  int K;                  // checkpoint interval: segment slot of step n is n - (n / K) * K
};

// One device-to-device copy of a batched copy launch (checkpoint saves and
// restores of several instances at once): n4 float4 from src to dst.
struct CopyDesc {
  const float4* src;
  float4* dst;
  long long n4;
};

// Stencil weights of a step launch (kernel parameters, so they stay in the
// constant bank): forward stage 1 a_k/dx (flux) and stage 2 a_k dt^2/dx
// (divergence); adjoint stage 1 -a_k dt^2/dx and stage 2 a_k/dx.
struct AcuCoef {
  float c1x[4], c1z[4], c2x[4], c2z[4];
  float dt2;
};

// Everything one elastic step kernel needs (passed by value). Node sets on the
// padded grid (index (i, j) of each field's storage): normal stresses and
// lambda, lambda+2mu at (i, j); vx and bx at (i, j+1/2); vz and bz at
// (i+1/2, j); sxz and mu_xz at (i+1/2, j+1/2).
constexpr int ELA_SLOTS = 8;  // source partial slots: 4 tiles x (normal box, shear box)
struct EleStep {
  Grid g;
  int S, N, n, nt, nrec;
  float cx[4], cz[4];     // a_k/dx, a_k/dz
  float dt;
  const float *bx, *bz, *lam, *lp2m, *mxz;   // [slice] medium on the nodes (zero outside)
  const float *ax, *bxt, *axh, *bxh, *az, *bzt, *azh, *bzh;  // CPML tables
  // forward state ([S][slice] each)
  float *vx, *vz, *sxx, *szz, *sxz;
  float* psi[8];          // CPML memory variables, node-local, updated in place
  // moment-tensor sources: boxes on the normal and shear grids
  const int *box_n, *box_s;   // [S][2], -1 if invalid
  const float *w_n, *w_s;     // [S][49]
  int src_n;
  const float* stf;           // [S][nt]
  const float* mt;            // [S][3] (Mxx, Mzz, Mxz)
  // receivers (vx, vz nodes of the receiver cell), per owning thread
  const int *thr_rec_start, *thr_rec;
  float* seis;                // [S][2][nrec][nt]
  // forward values kept for the reverse sweep (STORE): fx, fz, ex, ez, exz
  float* slot[5];
  // adjoint state
  float *Vx, *Vz, *Sxx, *Szz, *Sxz;
  const float* Min[8];
  float* Mout[8];
  const float* res;           // [S][2][nrec][nt]
  float *g_lam, *g_mu, *g_mxz, *g_bx, *g_bz;  // [S][slice] FP32 segment partials
  float* src_part;            // [S][nt][ELA_SLOTS][3]
  const float* x0;
  float dx, dz;
  int* status;                // ST_* bits (a timed-out tile wait sets ST_TIMEOUT)
};

}  // namespace fwi
