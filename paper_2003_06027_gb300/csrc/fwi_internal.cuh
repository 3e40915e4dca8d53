// fwi_internal.cuh - device-side layout and parameter blocks shared by the
// kernels of libfwi (not part of the public ABI).
//
// HBM layout of every per-shot field (wavefields, CPML memory variables,
// gradient partials, stored wavefields): [shot][rows][pitch] FP32 with a zero
// apron of APRON cells on every side, so that the halo loads of a tile never
// need bounds checks. Cell (i, j) of the padded grid (physical + CPML) of
// shot s lives at  base + s*slice + off0 + i*pitch + j,
// off0 = APRON*pitch + APRON.  Rows are padded to a multiple of the tile
// height and pitch to a multiple of the tile width; cells outside the padded
// grid are never written and stay zero.
#pragma once
#include <cstdint>

namespace fwi {

constexpr int APRON = 8;     // >= stencil radius 2N-1 (7 at 8th order), float4 aligned
constexpr int TILE_X = 64;   // cells per tile along x (16 threads x float4)
constexpr int TILE_Z = 16;   // rows per tile
constexpr int NTHREADS = 256;
constexpr int TAB_OFF = 8;   // 1D CPML tables are indexed [h + TAB_OFF]
constexpr int SRC_W = 7;     // Gaussian source support (7 x 7)
constexpr int SRC_SLOTS = 4; // a 7 x 7 box touches at most 2 x 2 tiles

struct Grid {
  int nz, nx, npml;   // physical grid and CPML width
  int Nz, Nx;         // padded grid
  int ntx, ntz;       // tiles
  int pitch;          // floats per row
  int rows;           // allocated rows per shot
  long long slice;    // floats per shot per field
  long long off0;     // offset of padded cell (0,0)
};

// Everything one acoustic step kernel needs (passed by value).
struct AcuStep {
  Grid g;
  int S, N, n, nt, nrec;
  float inv_dx, inv_dz, dt2;
  float a[4];
  const float* m;                                    // [slice] c^2, zero in the apron
  const float *ax, *bx, *axh, *bxh, *az, *bz, *azh, *bzh;  // CPML tables
  // forward state
  const float* u_cur;     // u^n
  float* u_prev;          // u^{n-1} in, u^{n+1} out (in place)
  const float *psix_in, *psiz_in;
  float *psix_out, *psiz_out;
  float *zetx, *zetz;     // in place (cell-local in the forward step)
  // sources: box origin (padded cell indices) and weights, per shot
  const int* src_box;     // [S][2] (i0, j0)
  const float* src_w;     // [S][49]
  int src_n;              // box side: 1 (point) or 7 (Gaussian)
  const float* stf;       // [S][nt]
  // receivers: per-tile lists
  const int* tile_rec_start;  // [ntiles + 1]
  const int* tile_rec;        // receiver indices grouped by tile
  const int* rec_cell;        // [nrec][2] padded (i, j)
  float* seis;                // [S][nrec][nt]
  // stored wavefields for the reverse sweep (one slot = one step)
  float *slot_u, *slot_psix, *slot_psiz;
  // adjoint state
  const float* l_cur;     // lambda_{n+1}
  float* l_prev;          // lambda_{n+2} in, lambda_n out
  const float *zx_in, *zz_in, *px_in, *pz_in;
  float *zx_out, *zz_out, *px_out, *pz_out;
  const float* res;       // [S][nrec][nt] residual seis - observed
  float* gpart;           // [S][slice] FP32 gradient partial (dJ/dm per padded cell)
  float* src_part;        // [S][nt][SRC_SLOTS][3]
  float src_x0_cells;     // unused placeholder for alignment
  const float* x0;        // [S][2] metres (physical)
  float dx, dz;
};

}  // namespace fwi
