// fwi_capi.cu - the C ABI of libfwi (declared in include/fwi.h): context,
// device workspace, validation, and the orchestration of the time loops.
//
// fwi_forward runs the explicit recursion of Eq. forward; fwi_misfit_grad
// adds the L2 misfit and the reverse sweep of Eqs. adjoint-backward /
// adjoint-gradient. The reverse sweep needs U_{k-1} at every step; instead of
// keeping all nt wavefields (the memory limit the paper's Limitations section
// names), the forward sweep saves the full state every K steps and the
// reverse sweep recomputes one K-step segment at a time into a slot buffer.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <string>
#include <vector>

#include "../../include/fwi.h"
#include "fwi_host.h"
#include "fwi_internal.cuh"

namespace fwi {
cudaError_t launch_acu_fwd(const AcuStep& p, const AcuMaps& maps, bool record, bool store, cudaStream_t st);
cudaError_t launch_acu_fwd_tz(const AcuStep& p, const AcuMaps& maps, bool record, bool store, int tz, cudaStream_t st,
                              bool lap);
cudaError_t launch_acu_adj(const AcuStep& p, const AcuMaps& maps, cudaStream_t st, bool lap);
cudaError_t launch_acu_fwd_batch(const BatchArgs& b, const AcuCoef& cf, int N, bool record, cudaStream_t st);
cudaError_t launch_acu_adj_batch(const BatchArgs& b, const AcuCoef& cf, int N, cudaStream_t st);
cudaError_t launch_copy_table(const CopyDesc* d, int n, cudaStream_t st);
cudaError_t acu_kernels_init();
cudaError_t ela_kernels_init();
cudaError_t acu_make_maps(AcuMaps* maps, const Grid& g, int S, float* u_pair, const float* mh);
cudaError_t acu_make_adj_maps(AcuMaps* maps, const Grid& g, int S, float* lam_pair, float* hx_pair, float* hz_pair);
cudaError_t launch_pad_model(const float* c, const Grid& g, float* m, cudaStream_t st);
cudaError_t launch_cpml_tables(int n_phys, int npml, int Npad, int len, double h, double dt, double R,
                               double vmax, double f0, float* a, float* b, float* ah, float* bh,
                               cudaStream_t st);
cudaError_t launch_src_prep(int S, int kind, const float* x0, const Grid& g, float dx, float dz, int* box,
                            float* w, int* status, cudaStream_t st);
cudaError_t launch_rec_csr(int nrec, const int* iz, const int* ix, const Grid& g, int* rec_cell, int* rec_key,
                           int* start, int* cursor, int* list, int* status, cudaStream_t st);
cudaError_t launch_model_check(const float* c, long long n, float coef, int* status, cudaStream_t st);
cudaError_t launch_misfit(const float* seis, float* res, long long n, double* part, int nb, double* J,
                          int* status, bool vjp, cudaStream_t st);
cudaError_t launch_finite_check(const float* a, long long n, int* status, cudaStream_t st);
cudaError_t launch_superpose(const float* seis, int S, long long n, const float* obs, float* cot, double* part,
                             int nb, double* J, int* status, cudaStream_t st);
cudaError_t launch_selftest_wait(int* status, unsigned long long* waited_ns, cudaStream_t st);
cudaError_t launch_ela_velocity_grad(const float* vp, const float* vs, const float* rho, const float* gin,
                                     float* gout, long long n, cudaStream_t st);
cudaError_t launch_adj_init(const AcuStep& p, float* lam, float* hx, float* hz, cudaStream_t st, bool lap = false);
cudaError_t launch_line_prep(int S, int L, const float* x0, const Grid& g, float dx, float dz, int* line_cell,
                             int* box, int* status, cudaStream_t st);
cudaError_t launch_line_inject(int S, int L, int n, int nt, float scale, const float* amp, const int* line_cell,
                               float* u, const Grid& g, const int* rec_cell, int nrec, float* seis, cudaStream_t st);
cudaError_t launch_line_grad(int S, int L, int n, int nt, float scale, const int* line_cell, const float* lam,
                             const Grid& g, float* gamp, cudaStream_t st);
cudaError_t launch_fold(float* gpart, int S, long long slice, double* G, cudaStream_t st);
cudaError_t launch_grad_c(const double* G, const Grid& g, const float* c, float* grad, cudaStream_t st);
cudaError_t launch_src_grad(const float* part, int S, int nt, int nslots, double scale, const float* stf,
                            double inv_sig2, int kind, float* gstf, float* gx0, cudaStream_t st);
void set_last_error(const std::string& msg);
}  // namespace fwi

using namespace fwi;

namespace {
thread_local std::string g_err;
}  // namespace

// Lets the other translation units of the library set fwi_last_error().
void fwi::set_last_error(const std::string& msg) { g_err = msg; }

namespace {

fwi_status fail(fwi_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

constexpr int MISFIT_BLOCKS = 512;

// Staggered first-derivative weights (the Taylor moment conditions
// sum_k a_k (2k-1)^(2j-1) = delta_{j1}); exact rationals for orders 4 and 8.
bool fd_coeffs(int order, float a[4]) {
  for (int k = 0; k < 4; k++) a[k] = 0.f;
  if (order == 4) {
    a[0] = (float)(9.0 / 8.0);
    a[1] = (float)(-1.0 / 24.0);
    return true;
  }
  if (order == 8) {
    a[0] = (float)(1225.0 / 1024.0);
    a[1] = (float)(-245.0 / 3072.0);
    a[2] = (float)(49.0 / 5120.0);
    a[3] = (float)(-5.0 / 7168.0);
    return true;
  }
  return false;
}

struct Plan {
  Grid g{};
  int S = 0, nt = 0, nrec = 0, K = 0, nseg = 0, N = 0, kind = 0;
  int L = 0;  // cells of a line source (FWI_SRC_LINE), else 0
  bool grad = false;
  int tablen = 0;
  int slot_fields = 2;  // fields a segment slot keeps per step: p_x, p_z (divergence form) or r (c^2 Laplacian)
  // base
  float *m = nullptr, *tab = nullptr, *c = nullptr, *stf = nullptr, *x0 = nullptr, *src_w = nullptr;
  int *src_box = nullptr, *rec_in = nullptr, *rec_cell = nullptr, *rec_key = nullptr, *tstart = nullptr;
  int *tcursor = nullptr, *tlist = nullptr;
  int* line_cell = nullptr;  // [S][2] padded (row, first column) of a line source
  float *u = nullptr;  // [2][S][slice]: pair of wavefield buffers
  float *psix[2] = {}, *psiz[2] = {}, *zetx = nullptr, *zetz = nullptr, *seis = nullptr;
  int* status = nullptr;
  // gradient
  float *res = nullptr, *ckpt = nullptr, *slot = nullptr, *lam = nullptr, *zx[2] = {}, *zz[2] = {};
  float *px[2] = {}, *pz[2] = {}, *gpart = nullptr, *src_part = nullptr, *grad_c = nullptr;
  float *hx = nullptr, *hz = nullptr;  // [2][S][slice] hhat pairs of the adjoint CPML tiles
  float *gstf = nullptr, *gx0 = nullptr;
  double *G = nullptr, *Jpart = nullptr, *J = nullptr;
  size_t bytes = 0;
  size_t zero_lo = 0, zero_hi = 0;  // byte range re-zeroed on every call
};

// Lay the plan out over an arena starting at `base` (nullptr: size only).
void layout(Plan& P, char* base) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    off = (off + 255) & ~size_t(255);
    char* p = base ? base + off : nullptr;
    off += bytes;
    return p;
  };
  const size_t field = (size_t)P.S * (size_t)P.g.slice * sizeof(float);
  const int ntiles = P.g.ntx * P.g.ntz;
  P.status = (int*)take(64);
  P.m = (float*)take((size_t)P.g.slice * 4);
  P.tab = (float*)take((size_t)8 * P.tablen * 4);
  P.c = (float*)take((size_t)P.g.nz * P.g.nx * 4);
  const size_t stf_len = (size_t)P.S * P.nt * (size_t)std::max(1, P.L);  // [S][nt] or [S][nt][L]
  P.stf = (float*)take(stf_len * 4);
  P.line_cell = (int*)take((size_t)P.S * 2 * 4);
  P.x0 = (float*)take((size_t)P.S * 2 * 4);
  P.src_w = (float*)take((size_t)P.S * SRC_W * SRC_W * 4);
  P.src_box = (int*)take((size_t)P.S * 2 * 4);
  P.rec_in = (int*)take((size_t)(P.nrec + 1) * 2 * 4);
  P.rec_cell = (int*)take((size_t)(P.nrec + 1) * 2 * 4);
  P.rec_key = (int*)take((size_t)(P.nrec + 1) * 4);
  P.tstart = (int*)take((size_t)(ntiles * NTHREADS + 1) * 4);
  P.tcursor = (int*)take((size_t)(ntiles * NTHREADS + 1) * 4);
  P.tlist = (int*)take((size_t)(P.nrec + 1) * 4);
  P.seis = (float*)take((size_t)P.S * P.nrec * P.nt * 4 + 4);
  // fields zeroed on every call (initial conditions)
  off = (off + 255) & ~size_t(255);
  P.zero_lo = off;
  P.u = (float*)take(2 * field);
  for (int k = 0; k < 2; k++) P.psix[k] = (float*)take(field);
  for (int k = 0; k < 2; k++) P.psiz[k] = (float*)take(field);
  P.zetx = (float*)take(field);
  P.zetz = (float*)take(field);
  if (P.grad) {
    P.lam = (float*)take(2 * field);
    for (int k = 0; k < 2; k++) P.zx[k] = (float*)take(field);
    for (int k = 0; k < 2; k++) P.zz[k] = (float*)take(field);
    for (int k = 0; k < 2; k++) P.px[k] = (float*)take(field);
    for (int k = 0; k < 2; k++) P.pz[k] = (float*)take(field);
    P.hx = (float*)take(2 * field);
    P.hz = (float*)take(2 * field);
    P.gpart = (float*)take(field);
    P.G = (double*)take((size_t)P.g.slice * 8);
    P.src_part = (float*)take((size_t)P.S * P.nt * SRC_SLOTS * 3 * 4);
  }
  off = (off + 255) & ~size_t(255);
  P.zero_hi = off;
  if (P.grad) {
    P.res = (float*)take((size_t)P.S * P.nrec * P.nt * 4 + 4);
    P.Jpart = (double*)take((size_t)MISFIT_BLOCKS * 8);
    P.J = (double*)take(8);
    P.grad_c = (float*)take((size_t)P.g.nz * P.g.nx * 4);
    P.gstf = (float*)take(stf_len * 4);
    P.gx0 = (float*)take((size_t)P.S * 2 * 4);
    P.ckpt = (float*)take(field * 6 * (size_t)P.nseg);
    P.slot = (float*)take(field * (size_t)P.slot_fields * (size_t)P.K);  // per step: p_x, p_z, or r
  }
  P.bytes = (off + 255) & ~size_t(255);
}

}  // namespace

namespace {

// LK: a checked kernel launch, counted (n kernels per launcher call)
#define LK(n, call)      \
  do {                   \
    CK(call);            \
    ctx->launches += (n); \
  } while (0)

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(FWI_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));         \
  } while (0)

fwi_status validate(const fwi_model* M, const fwi_sources* Sv, const fwi_receivers* R, int nt, float dt) {
  if (!M || !Sv || !R) return fail(FWI_EINVAL, "model, sources and receivers must not be NULL");
  if (M->physics != FWI_ACOUSTIC) return fail(FWI_ENOTIMPL, "only FWI_ACOUSTIC is implemented in this call");
  if (M->nz < 1 || M->nx < 1) return fail(FWI_EINVAL, "nz and nx must be >= 1");
  if (!(M->dz > 0.f) || !(M->dx > 0.f)) return fail(FWI_EINVAL, "dz and dx must be > 0");
  if (M->order != 4 && M->order != 8) return fail(FWI_EINVAL, "order must be 4 or 8");
  if (M->npml < 0) return fail(FWI_EINVAL, "npml must be >= 0");
  if (M->npml > 0 && (!(M->pml_R > 0.f && M->pml_R < 1.f) || !(M->pml_vmax > 0.f) || !(M->pml_f0 >= 0.f)))
    return fail(FWI_EINVAL, "CPML needs 0 < pml_R < 1, pml_vmax > 0, pml_f0 >= 0");
  if (!M->vp) return fail(FWI_EINVAL, "vp must not be NULL");
  if (M->op != FWI_OP_DIVERGENCE && M->op != FWI_OP_LAPLACIAN)
    return fail(FWI_EINVAL, "op must be FWI_OP_DIVERGENCE or FWI_OP_LAPLACIAN");
  if (Sv->nshots < 1) return fail(FWI_EINVAL, "nshots must be >= 1");
  if (Sv->kind != FWI_SRC_POINT && Sv->kind != FWI_SRC_GAUSSIAN && Sv->kind != FWI_SRC_LINE)
    return fail(FWI_EINVAL, "acoustic sources are FWI_SRC_POINT, FWI_SRC_GAUSSIAN or FWI_SRC_LINE");
  if (Sv->kind == FWI_SRC_LINE && (Sv->line_len < 1 || Sv->line_len > M->nx))
    return fail(FWI_EINVAL, "a line source needs 1 <= line_len <= nx");
  if (!Sv->x0 || !Sv->stf) return fail(FWI_EINVAL, "x0 and stf must not be NULL");
  if (R->nrec < 0 || (R->nrec > 0 && (!R->iz || !R->ix))) return fail(FWI_EINVAL, "bad receiver arrays");
  if (nt < 1) return fail(FWI_EINVAL, "nt must be >= 1");
  if (!(dt > 0.f)) return fail(FWI_EINVAL, "dt must be > 0");
  const long long Nz = (long long)M->nz + 2LL * M->npml, Nx = (long long)M->nx + 2LL * M->npml;
  if (Nz > (1 << 20) || Nx > (1 << 20) || Nz * Nx > (1LL << 31)) return fail(FWI_EINVAL, "grid too large");
  return FWI_OK;
}

void make_plan(Plan& P, const fwi_model* M, const fwi_sources* Sv, const fwi_receivers* R, int nt, int K,
               bool grad) {
  Grid& g = P.g;
  g.nz = M->nz;
  g.nx = M->nx;
  g.npml = M->npml;
  g.Nz = M->nz + 2 * M->npml;
  g.Nx = M->nx + 2 * M->npml;
  g.ntx = (g.Nx + TILE_X - 1) / TILE_X;
  g.ntz = (g.Nz + TILE_Z - 1) / TILE_Z;
  g.pitch = g.ntx * TILE_X + 2 * APRON;
  g.rows = (g.Nz + ROW_ALIGN - 1) / ROW_ALIGN * ROW_ALIGN + 2 * APRON;
  g.slice = (long long)g.rows * g.pitch;
  g.off0 = (long long)APRON * g.pitch + APRON;
  P.S = Sv->nshots;
  P.nt = nt;
  P.nrec = R->nrec;
  P.N = M->order / 2;
  P.kind = Sv->kind;
  P.L = Sv->kind == FWI_SRC_LINE ? Sv->line_len : 0;
  P.grad = grad;
  P.K = grad ? K : 0;
  P.nseg = grad ? (nt + K - 1) / K : 0;
  P.tablen = std::max(g.ntx * TILE_X, g.rows - 2 * APRON) + 2 * APRON + 2 * TAB_OFF;
  P.slot_fields = M->op == FWI_OP_LAPLACIAN ? 1 : 2;
}

std::string plan_key(const Plan& P) {
  char b[256];
  snprintf(b, sizeof b, "%d %d %d %d %lld %d %d %d %d %d %d %d %d", P.g.Nz, P.g.Nx, P.g.pitch, P.g.rows, P.g.slice,
           P.S, P.nt, P.nrec, P.K, (int)P.grad, P.tablen, P.L, P.slot_fields);
  return b;
}

fwi_status ensure_arena(fwi_ctx* ctx, Plan& P, cudaStream_t st) {
  layout(P, nullptr);
  const std::string key = "acoustic " + plan_key(P);
  fwi_status v = arena_acquire(ctx, P.bytes, key, P.zero_lo, P.zero_hi, st);
  if (v != FWI_OK) return v;
  layout(P, ctx->arena);
  return FWI_OK;
}

void fill_step(const Plan& P, const fwi_model* M, float dt, AcuStep& p);

// Copy inputs into the workspace and build m, CPML tables, source weights,
// receiver lists; queue the model checks.
fwi_status prepare(fwi_ctx* ctx, Plan& P, const fwi_model* M, const fwi_sources* Sv, const fwi_receivers* R,
                   float dt, cudaStream_t st, AcuStep& p) {
  const Grid& g = P.g;
  CK(cudaMemcpyAsync(P.c, M->vp, (size_t)g.nz * g.nx * 4, cudaMemcpyDefault, st));
  CK(cudaMemcpyAsync(P.stf, Sv->stf, (size_t)P.S * P.nt * std::max(1, P.L) * 4, cudaMemcpyDefault, st));
  CK(cudaMemcpyAsync(P.x0, Sv->x0, (size_t)P.S * 2 * 4, cudaMemcpyDefault, st));
  if (P.nrec > 0) {
    CK(cudaMemcpyAsync(P.rec_in, R->iz, (size_t)P.nrec * 4, cudaMemcpyDefault, st));
    CK(cudaMemcpyAsync(P.rec_in + P.nrec, R->ix, (size_t)P.nrec * 4, cudaMemcpyDefault, st));
  }
  float a[4];
  fd_coeffs(M->order, a);
  float sa = 0.f;
  for (int k = 0; k < 4; k++) sa += fabsf(a[k]);
  const float coef = dt * sqrtf(1.f / (M->dx * M->dx) + 1.f / (M->dz * M->dz)) * sa;
  LK(1, launch_model_check(P.c, (long long)g.nz * g.nx, coef, P.status, st));
  LK(1, launch_pad_model(P.c, g, P.m, st));
  const int L = P.tablen;
  float* T = P.tab;
  LK(1, launch_cpml_tables(g.nx, g.npml, g.Nx, L, M->dx, dt, M->pml_R, M->pml_vmax, M->pml_f0, T, T + L, T + 2 * L,
                        T + 3 * L, st));
  LK(1, launch_cpml_tables(g.nz, g.npml, g.Nz, L, M->dz, dt, M->pml_R, M->pml_vmax, M->pml_f0, T + 4 * L, T + 5 * L,
                        T + 6 * L, T + 7 * L, st));
  if (P.L > 0)
    LK(1, launch_line_prep(P.S, P.L, P.x0, g, M->dx, M->dz, P.line_cell, P.src_box, P.status, st));
  else
    LK(1, launch_src_prep(P.S, P.kind, P.x0, g, M->dx, M->dz, P.src_box, P.src_w, P.status, st));
  LK(1, launch_rec_csr(P.nrec, P.rec_in, P.rec_in + P.nrec, g, P.rec_cell, P.rec_key, P.tstart, P.tcursor, P.tlist,
                       P.status, st));
  fill_step(P, M, dt, p);
  (void)ctx;
  return FWI_OK;
}

// The step parameters of a call (everything but the fields of one time step),
// from the plan's layout alone: no device work.
void fill_step(const Plan& P, const fwi_model* M, float dt, AcuStep& p) {
  const Grid& g = P.g;
  float a[4];
  fd_coeffs(M->order, a);
  const int L = P.tablen;
  float* T = P.tab;
  memset(&p, 0, sizeof p);
  p.g = g;
  p.S = P.S;
  p.S_pair = P.S;
  p.s0 = 0;
  p.N = P.N;
  p.nt = P.nt;
  p.nrec = P.nrec;
  p.dt2 = dt * dt;
  // forward weights: stage 1 a_k/dx (flux), stage 2 a_k dt^2/dx (dt^2 folded in)
  for (int k = 0; k < 4; k++) {
    p.c1x[k] = a[k] / M->dx;
    p.c1z[k] = a[k] / M->dz;
    p.c2x[k] = a[k] * p.dt2 / M->dx;
    p.c2z[k] = a[k] * p.dt2 / M->dz;
  }
  p.ntiles = P.S * g.ntx * g.ntz;
  p.mh = P.m;
  p.u = P.u;
  p.lam = P.lam;
  p.status = P.status;
  p.ax = T; p.bx = T + L; p.axh = T + 2 * L; p.bxh = T + 3 * L;
  p.az = T + 4 * L; p.bz = T + 5 * L; p.azh = T + 6 * L; p.bzh = T + 7 * L;
  p.zetx = P.zetx;
  p.zetz = P.zetz;
  p.src_box = P.src_box;
  p.src_w = P.src_w;
  p.src_n = P.kind == FWI_SRC_GAUSSIAN ? SRC_W : 1;
  p.stf = P.stf;
  p.thr_rec_start = P.tstart;
  p.thr_rec = P.tlist;
  p.rec_cell = P.rec_cell;
  p.seis = P.seis;
  p.x0 = P.x0;
  p.dx = M->dx;
  p.dz = M->dz;
}

// Adjoint weights: stage 1 -a_k dt^2/dx (qbar = -dt^2 D+ hhat), stage 2 a_k/dx.
void set_adjoint_weights(AcuStep& q, const AcuStep& fwd) {
  for (int k = 0; k < 4; k++) {
    q.c1x[k] = -fwd.c2x[k];
    q.c1z[k] = -fwd.c2z[k];
    q.c2x[k] = fwd.c1x[k];
    q.c2z[k] = fwd.c1z[k];
  }
}

void set_fwd_state(const Plan& P, AcuStep& p, int n) {
  p.n = n;
  p.cur = n & 1;
  p.psix_in = P.psix[n & 1];
  p.psix_out = P.psix[(n + 1) & 1];
  p.psiz_in = P.psiz[n & 1];
  p.psiz_out = P.psiz[(n + 1) & 1];
}

fwi_status finish_status(fwi_ctx* ctx, const Plan& P, cudaStream_t st) { return finish_status_dev(ctx, P.status, st); }

// ---------------------------------------------------------------------------
// Shot groups: the shots are split into up to MAX_GROUPS contiguous groups whose
// step launches run on separate streams. Each step kernel is a persistent walk
// over its tiles, and its last partial wave leaves SMs idle; concurrent groups
// fill them. Everything that couples shots (misfit, folds, source gradients)
// runs on the call's stream after a join.
constexpr int MAX_GROUPS = 4;
// The adjoint step kernel runs fewer, larger groups: measured on 16 shots of the
// 201 x 601 problem, 2 groups gave 26.8 us per step against 27.2 with 4 (the
// forward kernels prefer 4: 16.4 against 18.6 us).
constexpr int ADJ_GROUPS = 2;

struct Groups {
  int G = 1;
  int s0[MAX_GROUPS] = {0, 0, 0, 0};
  int n[MAX_GROUPS] = {0, 0, 0, 0};
  cudaStream_t st[MAX_GROUPS] = {};
};

fwi_status make_groups(fwi_ctx* ctx, int S, cudaStream_t main, Groups& gr, int max_groups = MAX_GROUPS) {
  gr.G = std::max(1, std::min(std::min(max_groups, MAX_GROUPS), S));
  for (int g = 0, s0 = 0; g < gr.G; g++) {
    gr.n[g] = S / gr.G + (g < S % gr.G ? 1 : 0);
    gr.s0[g] = s0;
    s0 += gr.n[g];
  }
  if (gr.G == 1) {
    gr.st[0] = main;
    return FWI_OK;
  }
  for (int g = 0; g < gr.G; g++) {
    if (!ctx->gstream[g]) CK(cudaStreamCreateWithFlags(&ctx->gstream[g], cudaStreamNonBlocking));
    if (!ctx->join_ev[g]) CK(cudaEventCreateWithFlags(&ctx->join_ev[g], cudaEventDisableTiming));
    gr.st[g] = ctx->gstream[g];
  }
  if (!ctx->fork_ev) CK(cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming));
  return FWI_OK;
}

fwi_status fork(fwi_ctx* ctx, const Groups& gr, cudaStream_t main) {
  if (gr.G == 1) return FWI_OK;
  CK(cudaEventRecord(ctx->fork_ev, main));
  for (int g = 0; g < gr.G; g++) CK(cudaStreamWaitEvent(gr.st[g], ctx->fork_ev, 0));
  return FWI_OK;
}

fwi_status join(fwi_ctx* ctx, const Groups& gr, cudaStream_t main) {
  if (gr.G == 1) return FWI_OK;
  for (int g = 0; g < gr.G; g++) {
    CK(cudaEventRecord(ctx->join_ev[g], gr.st[g]));
    CK(cudaStreamWaitEvent(main, ctx->join_ev[g], 0));
  }
  return FWI_OK;
}

// Tile height of the context's acoustic forward steps.
int fwd_tz(const fwi_ctx* ctx) { return ctx->fwd_tile_rows == 64 ? 64 : TILE_Z; }

// The step parameters of one group: shots [s0, s0 + Sg). Per-shot arrays are
// offset to the group's first shot; the u and lambda pairs keep their base and
// the kernels index them with (pair * S_pair + s0 + s).
AcuStep group_view(const AcuStep& p, const Plan& P, int s0, int Sg) {
  AcuStep q = p;
  const long long sl = P.g.slice, ns = (long long)p.nrec * p.nt;
  auto off = [&](auto* ptr, long long per) { return ptr ? ptr + s0 * per : ptr; };
  q.S = Sg;
  q.s0 = s0;
  q.ntiles = Sg * P.g.ntx * P.g.ntz;
  q.psix_in = off(p.psix_in, sl);
  q.psix_out = off(p.psix_out, sl);
  q.psiz_in = off(p.psiz_in, sl);
  q.psiz_out = off(p.psiz_out, sl);
  q.zetx = off(p.zetx, sl);
  q.zetz = off(p.zetz, sl);
  q.src_box = off(p.src_box, 2);
  q.src_w = off(p.src_w, SRC_W * SRC_W);
  q.stf = off(p.stf, p.nt);
  q.x0 = off(p.x0, 2);
  q.seis = off(p.seis, ns);
  q.slot_px = off(p.slot_px, sl);
  q.slot_pz = off(p.slot_pz, sl);
  q.zx_in = off(p.zx_in, sl);
  q.zx_out = off(p.zx_out, sl);
  q.zz_in = off(p.zz_in, sl);
  q.zz_out = off(p.zz_out, sl);
  q.px_in = off(p.px_in, sl);
  q.px_out = off(p.px_out, sl);
  q.pz_in = off(p.pz_in, sl);
  q.pz_out = off(p.pz_out, sl);
  q.hx_out = off(p.hx_out, sl);
  q.hz_out = off(p.hz_out, sl);
  q.res = off(p.res, ns);
  q.gpart = off(p.gpart, sl);
  q.src_part = off(p.src_part, (long long)p.nt * SRC_SLOTS * 3);
  return q;
}

}  // namespace

// ---------------------------------------------------------------------------
// host helpers shared with the elastic orchestration (fwi_host.h)
fwi_status fwi::host_fail(fwi_status st, const std::string& msg) { return fail(st, msg); }

// Make the context arena at least `bytes` large. A new layout (key) zeroes the
// whole arena (aprons and never-written cells must read as zero); the same
// layout re-zeroes only [zero_lo, zero_hi) (the initial conditions) and the
// status word at offset 0.
fwi_status fwi::arena_acquire(fwi_ctx* ctx, size_t bytes, const std::string& key, size_t zero_lo, size_t zero_hi,
                              cudaStream_t st) {
  if (bytes > ctx->arena_bytes) {
    if (ctx->arena) {
      CK(cudaStreamSynchronize(st));
      CK(cudaFree(ctx->arena));
      ctx->arena = nullptr;
      ctx->arena_bytes = 0;
    }
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(FWI_ENOMEM, "cannot allocate " + std::to_string(bytes) + " bytes of workspace: " +
                                  cudaGetErrorString(e));
    }
    ctx->arena = (char*)p;
    ctx->arena_bytes = bytes;
    ctx->layout_key.clear();
    ctx->arena_epoch++;
  }
  if (ctx->layout_key != key) {
    CK(cudaMemsetAsync(ctx->arena, 0, bytes, st));
    ctx->layout_key = key;
    ctx->arena_epoch++;
  } else {
    CK(cudaMemsetAsync(ctx->arena + zero_lo, 0, zero_hi - zero_lo, st));
    CK(cudaMemsetAsync(ctx->arena, 0, 64, st));
  }
  return FWI_OK;
}

// Read the device status word (one sync) and turn it into a status code.
fwi_status fwi::finish_status_dev(fwi_ctx* ctx, const int* d_status, cudaStream_t st) {
  CK(cudaMemcpyAsync(ctx->h_status, d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return decode_status(*ctx->h_status, "");
}

// The status code of a device status word (FWI_OK when no bit is set).
fwi_status fwi::decode_status(int s, const std::string& where) {
  if (s & ST_TIMEOUT) return fail(FWI_ETIMEOUT, where + "a step kernel gave up waiting for its tile fetch");  // first: later results are invalid
  if (s & ST_BADMODEL) return fail(FWI_EINVAL, where + "the medium must be finite with vp > 0, rho > 0, vp^2 >= 2 vs^2");
  if (s & ST_BADREC) return fail(FWI_EINVAL, where + "a receiver lies outside the physical grid");
  if (s & ST_BADSRC) return fail(FWI_EINVAL, where + "a source (or its 7x7 Gaussian support) lies outside the grid");
  if (s & ST_CFL) return fail(FWI_ECFL, where + "CFL condition violated: c_max dt sqrt(1/dx^2+1/dz^2) sum|a_k| > 1");
  if (s & ST_NONFINITE) return fail(FWI_EUNSTABLE, where + "non-finite value in the seismograms or the misfit");
  return FWI_OK;
}

void fwi::ensure_events(fwi_ctx* ctx, size_t nseg) {
  for (auto& e : ctx->ev)
    if (!e) cudaEventCreate(&e);
  while (ctx->seg_ev.size() < 4 * nseg) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    ctx->seg_ev.push_back(e);
  }
}

extern "C" {

fwi_status fwi_create(fwi_ctx** out, int device) {
  if (!out) return fail(FWI_EINVAL, "ctx must not be NULL");
  *out = nullptr;
  int n = 0;
  CK(cudaGetDeviceCount(&n));
  if (device < 0 || device >= n) return fail(FWI_EINVAL, "no such CUDA device");
  CK(cudaSetDevice(device));
  CK(acu_kernels_init());
  CK(ela_kernels_init());
  fwi_ctx* c = new fwi_ctx();
  c->device = device;
  if (cudaMallocHost((void**)&c->h_status, 64) != cudaSuccess) {
    delete c;
    return fail(FWI_ENOMEM, "cannot allocate pinned status word");
  }
  *out = c;
  g_err.clear();
  return FWI_OK;
}

fwi_status fwi_destroy(fwi_ctx* ctx) {
  if (!ctx) return FWI_OK;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  if (ctx->arena) cudaFree(ctx->arena);
  if (ctx->h_status) cudaFreeHost(ctx->h_status);
  for (auto& e : ctx->ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : ctx->seg_ev) cudaEventDestroy(e);
  for (int g = 0; g < 4; g++) {
    if (ctx->gstream[g]) cudaStreamDestroy(ctx->gstream[g]);
    if (ctx->join_ev[g]) cudaEventDestroy(ctx->join_ev[g]);
  }
  if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  delete ctx;
  return FWI_OK;
}

const char* fwi_last_error(void) { return g_err.c_str(); }

fwi_status fwi_elastic_velocity_grad(const float* vp, const float* vs, const float* rho, const float* grad_lame,
                                     float* grad_vel, int64_t n, void* stream) {
  if (n < 0) return fail(FWI_EINVAL, "n must be >= 0");
  if (n > 0 && (!vp || !vs || !rho || !grad_lame || !grad_vel))
    return fail(FWI_EINVAL, "vp, vs, rho, grad_lame and grad_vel must not be NULL");
  CK(launch_ela_velocity_grad(vp, vs, rho, grad_lame, grad_vel, n, (cudaStream_t)stream));
  g_err.clear();
  return FWI_OK;
}

fwi_status fwi_selftest_wait_timeout(fwi_ctx* ctx, int64_t* waited_ns) {
  if (!ctx) return fail(FWI_EINVAL, "ctx must not be NULL");
  CK(cudaSetDevice(ctx->device));
  void* buf = nullptr;
  CK(cudaMalloc(&buf, 16));
  int* dst = reinterpret_cast<int*>(buf);
  unsigned long long* dns = reinterpret_cast<unsigned long long*>(static_cast<char*>(buf) + 8);
  cudaError_t e = launch_selftest_wait(dst, dns, 0);
  int st = 0;
  unsigned long long ns = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&st, dst, sizeof st, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&ns, dns, sizeof ns, cudaMemcpyDeviceToHost);
  cudaFree(buf);
  if (e != cudaSuccess) return fail(FWI_ECUDA, std::string("selftest: ") + cudaGetErrorString(e));
  if (waited_ns) *waited_ns = (int64_t)ns;
  if (st & ST_TIMEOUT) return fail(FWI_ETIMEOUT, "device wait gave up as designed (self-test)");
  return fail(FWI_ECUDA, "self-test: a wait that cannot complete reported completion");
}

fwi_status fwi_set_shot_groups(fwi_ctx* ctx, int32_t forward_groups, int32_t adjoint_groups) {
  if (!ctx) return fail(FWI_EINVAL, "ctx must not be NULL");
  if (forward_groups < 0 || forward_groups > MAX_GROUPS || adjoint_groups < 0 || adjoint_groups > MAX_GROUPS)
    return fail(FWI_EINVAL, "shot groups must be in [0, " + std::to_string(MAX_GROUPS) + "] (0: default)");
  ctx->fwd_groups = forward_groups;
  ctx->adj_groups = adjoint_groups;
  return FWI_OK;
}

fwi_status fwi_set_tile_shape(fwi_ctx* ctx, int32_t forward_tile_rows) {
  if (!ctx) return fail(FWI_EINVAL, "ctx must not be NULL");
  if (forward_tile_rows != 0 && forward_tile_rows != 32 && forward_tile_rows != 64)
    return fail(FWI_EINVAL, "forward_tile_rows must be 0, 32 or 64");
  ctx->fwd_tile_rows = forward_tile_rows;
  g_err.clear();
  return FWI_OK;
}

fwi_status fwi_last_timing(const fwi_ctx* ctx, float* phase_ms3, float* kernel_ms3, int64_t* launches) {
  if (!ctx) return fail(FWI_EINVAL, "ctx must not be NULL");
  for (int k = 0; k < 3; k++) {
    if (phase_ms3) phase_ms3[k] = ctx->phase_ms[k];
    if (kernel_ms3) kernel_ms3[k] = ctx->kernel_ms[k];
  }
  if (launches) *launches = ctx->launches;
  return FWI_OK;
}

fwi_status fwi_forward(fwi_ctx* ctx, const fwi_model* M, const fwi_sources* Sv, const fwi_receivers* R,
                       int32_t nt, float dt, float* seis, void* stream) {
  if (!ctx) return fail(FWI_EINVAL, "ctx must not be NULL");
  if (M && M->physics == FWI_ELASTIC) return ela_forward(ctx, M, Sv, R, nt, dt, seis, stream);
  fwi_status v = validate(M, Sv, R, nt, dt);
  if (v != FWI_OK) return v;
  if (!seis && R->nrec > 0) return fail(FWI_EINVAL, "seis must not be NULL");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  const bool lap = M->op == FWI_OP_LAPLACIAN;
  Plan P;
  make_plan(P, M, Sv, R, nt, 0, false);
  v = ensure_arena(ctx, P, st);
  if (v != FWI_OK) return v;
  AcuStep p;
  ctx->launches = 0;
  v = prepare(ctx, P, M, Sv, R, dt, st, p);
  if (v != FWI_OK) return v;
  AcuMaps maps;
  CK(acu_make_maps(&maps, P.g, P.S, P.u, P.m));
  ensure_events(ctx, 0);
  Groups gr;
  if ((v = make_groups(ctx, P.S, st, gr, ctx->fwd_groups ? ctx->fwd_groups : MAX_GROUPS)) != FWI_OK) return v;
  CK(cudaEventRecord(ctx->ev[0], st));
  if ((v = fork(ctx, gr, st)) != FWI_OK) return v;
  const size_t fieldf = (size_t)P.S * P.g.slice;
  const float lscale = (float)((double)dt * dt / ((double)M->dx * M->dz));
  for (int n = 0; n < nt; n++) {
    set_fwd_state(P, p, n);
    for (int g = 0; g < gr.G; g++) {
      LK(1, launch_acu_fwd_tz(group_view(p, P, gr.s0[g], gr.n[g]), maps, true, false, fwd_tz(ctx), gr.st[g], lap));
      if (P.L > 0)
        LK(1, launch_line_inject(gr.n[g], P.L, n, nt, lscale, P.stf + (size_t)gr.s0[g] * nt * P.L,
                                 P.line_cell + 2 * gr.s0[g], P.u + ((n + 1) & 1) * fieldf + gr.s0[g] * P.g.slice,
                                 P.g, P.rec_cell, P.nrec, P.seis + (size_t)gr.s0[g] * P.nrec * nt, gr.st[g]));
    }
  }
  if ((v = join(ctx, gr, st)) != FWI_OK) return v;
  CK(cudaEventRecord(ctx->ev[1], st));
  const long long ns = (long long)P.S * P.nrec * nt;
  if (ns > 0) {
    LK(1, launch_finite_check(P.seis, ns, P.status, st));
    CK(cudaMemcpyAsync(seis, P.seis, (size_t)ns * 4, cudaMemcpyDefault, st));
  }
  CK(cudaEventRecord(ctx->ev[3], st));
  v = finish_status(ctx, P, st);
  float t = 0.f;
  cudaEventElapsedTime(&t, ctx->ev[0], ctx->ev[1]);
  ctx->phase_ms[0] = t;
  ctx->phase_ms[1] = 0.f;
  cudaEventElapsedTime(&t, ctx->ev[0], ctx->ev[3]);
  ctx->phase_ms[2] = t;
  ctx->kernel_ms[0] = ctx->phase_ms[0] / nt;
  ctx->kernel_ms[1] = 0.f;
  ctx->kernel_ms[2] = 0.f;
  if (v == FWI_OK) g_err.clear();
  return v;
}

}  // extern "C"

namespace {

// A phase mark: a plain event record on a direct call; inside a recording, an
// external event-record node, so that every replay of the graph records it
// and the replay's phases can be timed like a direct call's.
cudaError_t mark(cudaEvent_t e, cudaStream_t st, bool capture) {
  return capture ? cudaEventRecordWithFlags(e, st, cudaEventRecordExternal) : cudaEventRecord(e, st);
}

// Phase and per-step kernel times of the last gradient call (or graph replay)
// of nt steps with a checkpoint every K steps, from its completed phase marks:
// ev[0..3] (forward sweep start and end, reverse sweep end, call end) and per
// segment seg_ev[4 seg + 0..2] (recompute start, adjoint start, adjoint end).
void grad_timings(fwi_ctx* ctx, int nt, int K) {
  const int nseg = (nt + K - 1) / K, nlast = (nseg - 1) * K;
  float t = 0.f;
  cudaEventElapsedTime(&t, ctx->ev[0], ctx->ev[1]);
  ctx->phase_ms[0] = t;
  cudaEventElapsedTime(&t, ctx->ev[1], ctx->ev[2]);
  ctx->phase_ms[1] = t;
  cudaEventElapsedTime(&t, ctx->ev[0], ctx->ev[3]);
  ctx->phase_ms[2] = t;
  ctx->kernel_ms[0] = ctx->phase_ms[0] / nt;
  float rec = 0.f, adj = 0.f;
  for (int seg = 0; seg < nseg; seg++) {
    float ta = 0.f;
    cudaEventElapsedTime(&ta, ctx->seg_ev[4 * seg + 0], ctx->seg_ev[4 * seg + 1]);
    rec += ta;
    cudaEventElapsedTime(&ta, ctx->seg_ev[4 * seg + 1], ctx->seg_ev[4 * seg + 2]);
    adj += ta;
  }
  ctx->kernel_ms[1] = nlast > 0 ? rec / nlast : 0.f;  // per recomputed step
  ctx->kernel_ms[2] = adj / nt;
}

// The acoustic misfit/gradient call. With `capture` the device work is being
// recorded into a graph: the arena is already sized and laid out by an earlier
// call with the same problem, and the ending synchronisation (status read,
// phase timings) is left out.
fwi_status acu_misfit_grad(fwi_ctx* ctx, const fwi_model* M, const fwi_sources* Sv, const fwi_receivers* R,
                           int32_t nt, float dt, const float* observed, int32_t K, double* misfit, float* grad,
                           float* grad_stf, float* grad_x0, float* seis_out, cudaStream_t st, bool capture,
                           int** status_out) {
  fwi_status v = validate(M, Sv, R, nt, dt);
  if (v != FWI_OK) return v;
  if (!observed && R->nrec > 0) return fail(FWI_EINVAL, "observed must not be NULL");
  if (!misfit) return fail(FWI_EINVAL, "misfit must not be NULL");
  if (K < 1 || K > nt) return fail(FWI_EINVAL, "ckpt_every must be in [1, nt]");
  if (Sv->kind == FWI_SRC_LINE && grad_x0) return fail(FWI_EINVAL, "a line source has no position gradient");
  CK(cudaSetDevice(ctx->device));
  const bool lap = M->op == FWI_OP_LAPLACIAN;
  const float lscale = (float)((double)dt * dt / ((double)M->dx * M->dz));
  Plan P;
  make_plan(P, M, Sv, R, nt, K, true);
  v = ensure_arena(ctx, P, st);
  if (v != FWI_OK) return v;
  AcuStep p;
  ctx->launches = 0;
  v = prepare(ctx, P, M, Sv, R, dt, st, p);
  if (v != FWI_OK) return v;
  const long long ns = (long long)P.S * P.nrec * nt;
  if (ns > 0) CK(cudaMemcpyAsync(P.res, observed, (size_t)ns * 4, cudaMemcpyDefault, st));
  const size_t field = (size_t)P.S * P.g.slice;
  AcuMaps maps;
  CK(acu_make_maps(&maps, P.g, P.S, P.u, P.m));
  CK(acu_make_adj_maps(&maps, P.g, P.S, P.lam, P.hx, P.hz));
  ensure_events(ctx, P.nseg);

  Groups gr, gra;
  if ((v = make_groups(ctx, P.S, st, gr, ctx->fwd_groups ? ctx->fwd_groups : MAX_GROUPS)) != FWI_OK) return v;
  if ((v = make_groups(ctx, P.S, st, gra, ctx->adj_groups ? ctx->adj_groups : ADJ_GROUPS)) != FWI_OK) return v;
  const size_t sl = (size_t)P.g.slice;

  // forward sweep with a full-state checkpoint at the start of every segment
  // but the last: the sweep itself keeps the last segment's fluxes (recording
  // and storing in one launch), so that segment is never recomputed
  const int nlast = (P.nseg - 1) * K;
  CK(mark(ctx->ev[0], st, capture));
  if ((v = fork(ctx, gr, st)) != FWI_OK) return v;
  for (int n = 0; n < nt; n++) {
    if (n % K == 0 && n < nlast) {
      float* ck = P.ckpt + (size_t)(n / K) * 6 * field;
      const float* src[6] = {P.u + (n & 1) * field, P.u + ((n + 1) & 1) * field, P.psix[n & 1], P.psiz[n & 1],
                             P.zetx, P.zetz};
      for (int g = 0; g < gr.G; g++)
        for (int f = 0; f < 6; f++)
          CK(cudaMemcpyAsync(ck + f * field + gr.s0[g] * sl, src[f] + gr.s0[g] * sl, gr.n[g] * sl * 4,
                             cudaMemcpyDeviceToDevice, gr.st[g]));
    }
    set_fwd_state(P, p, n);
    const bool keep = n >= nlast;
    if (keep) {
      p.slot_px = P.slot + (size_t)(n - nlast) * P.slot_fields * field;
      p.slot_pz = lap ? nullptr : p.slot_px + field;
    }
    for (int g = 0; g < gr.G; g++) {
      LK(1, launch_acu_fwd_tz(group_view(p, P, gr.s0[g], gr.n[g]), maps, true, keep, fwd_tz(ctx), gr.st[g], lap));
      if (P.L > 0)
        LK(1, launch_line_inject(gr.n[g], P.L, n, nt, lscale, P.stf + (size_t)gr.s0[g] * nt * P.L,
                                 P.line_cell + 2 * gr.s0[g], P.u + ((n + 1) & 1) * field + gr.s0[g] * sl, P.g,
                                 P.rec_cell, P.nrec, P.seis + (size_t)gr.s0[g] * P.nrec * nt, gr.st[g]));
    }
  }
  if ((v = join(ctx, gr, st)) != FWI_OK) return v;
  CK(mark(ctx->ev[1], st, capture));
  if (ns > 0) LK(2, launch_misfit(P.seis, P.res, ns, P.Jpart, MISFIT_BLOCKS, P.J, P.status, ctx->vjp, st));
  else CK(cudaMemsetAsync(P.J, 0, 8, st));

  // reverse sweep, segment by segment
  p.res = P.res;
  p.gpart = P.gpart;
  p.src_part = P.src_part;
  AcuStep pa = p;
  set_adjoint_weights(pa, p);
  LK(1, launch_adj_init(pa, P.lam + (nt & 1) * field, P.hx + (nt & 1) * field, P.hz + (nt & 1) * field, st, lap));
  if (P.L > 0) LK(1, launch_line_grad(P.S, P.L, nt - 1, nt, lscale, P.line_cell, P.lam + (nt & 1) * field, P.g, P.gstf, st));
  for (int seg = P.nseg - 1; seg >= 0; seg--) {
    const int n0 = seg * K, n1 = std::min(nt, n0 + K);
    const float* ck = P.ckpt + (size_t)seg * 6 * field;
    float* dst[6] = {P.u + (n0 & 1) * field, P.u + ((n0 + 1) & 1) * field, P.psix[n0 & 1], P.psiz[n0 & 1], P.zetx,
                     P.zetz};
    // recompute (from the checkpoint) on the group streams; the last segment's
    // fluxes are already stored by the forward sweep
    CK(mark(ctx->seg_ev[4 * seg + 0], st, capture));
    if (seg < P.nseg - 1) {
      if ((v = fork(ctx, gr, st)) != FWI_OK) return v;
      for (int g = 0; g < gr.G; g++)
        for (int f = 0; f < 6; f++)
          CK(cudaMemcpyAsync(dst[f] + gr.s0[g] * sl, ck + f * field + gr.s0[g] * sl, gr.n[g] * sl * 4,
                             cudaMemcpyDeviceToDevice, gr.st[g]));
      for (int n = n0; n < n1; n++) {
        set_fwd_state(P, p, n);
        p.slot_px = P.slot + (size_t)(n - n0) * P.slot_fields * field;
        p.slot_pz = lap ? nullptr : p.slot_px + field;
        for (int g = 0; g < gr.G; g++) {
          LK(1, launch_acu_fwd_tz(group_view(p, P, gr.s0[g], gr.n[g]), maps, false, true, fwd_tz(ctx), gr.st[g], lap));
          if (P.L > 0)
            LK(1, launch_line_inject(gr.n[g], P.L, n, nt, lscale, P.stf + (size_t)gr.s0[g] * nt * P.L,
                                     P.line_cell + 2 * gr.s0[g], P.u + ((n + 1) & 1) * field + gr.s0[g] * sl, P.g,
                                     P.rec_cell, P.nrec, nullptr, gr.st[g]));
        }
      }
      if ((v = join(ctx, gr, st)) != FWI_OK) return v;
    }
    CK(mark(ctx->seg_ev[4 * seg + 1], st, capture));
    if ((v = fork(ctx, gra, st)) != FWI_OK) return v;
    for (int n = n1 - 1; n >= n0; n--) {
      pa.n = n;
      pa.cur = (n + 1) & 1;  // lambda_{n+1}; lambda_{n+2} -> lambda_n in the other buffer
      pa.slot_px = P.slot + (size_t)(n - n0) * P.slot_fields * field;
      pa.slot_pz = lap ? nullptr : pa.slot_px + field;
      pa.zx_in = P.zx[(n + 1) & 1];
      pa.zx_out = P.zx[n & 1];
      pa.zz_in = P.zz[(n + 1) & 1];
      pa.zz_out = P.zz[n & 1];
      pa.px_in = P.px[(n + 1) & 1];
      pa.px_out = P.px[n & 1];
      pa.pz_in = P.pz[(n + 1) & 1];
      pa.pz_out = P.pz[n & 1];
      pa.hx_out = P.hx + (n & 1) * field;
      pa.hz_out = P.hz + (n & 1) * field;
      for (int g = 0; g < gra.G; g++) {
        LK(1, launch_acu_adj(group_view(pa, P, gra.s0[g], gra.n[g]), maps, gra.st[g], lap));
        if (P.L > 0 && n >= 1)  // lambda_n is complete: the derivative for amp[n - 1]
          LK(1, launch_line_grad(gra.n[g], P.L, n - 1, nt, lscale, P.line_cell + 2 * gra.s0[g],
                                 P.lam + (n & 1) * field + gra.s0[g] * sl, P.g, P.gstf + (size_t)gra.s0[g] * nt * P.L,
                                 gra.st[g]));
      }
    }
    if ((v = join(ctx, gra, st)) != FWI_OK) return v;
    CK(mark(ctx->seg_ev[4 * seg + 2], st, capture));
    LK(1, launch_fold(P.gpart, P.S, P.g.slice, P.G, st));
  }
  CK(mark(ctx->ev[2], st, capture));
  if (grad) {
    LK(1, launch_grad_c(P.G, P.g, P.c, P.grad_c, st));
    CK(cudaMemcpyAsync(grad, P.grad_c, (size_t)P.g.nz * P.g.nx * 4, cudaMemcpyDefault, st));
  }
  if (P.L > 0) {
    if (grad_stf) CK(cudaMemcpyAsync(grad_stf, P.gstf, (size_t)P.S * nt * P.L * 4, cudaMemcpyDefault, st));
  } else if (grad_stf || grad_x0) {
    LK(1, launch_src_grad(P.src_part, P.S, nt, SRC_SLOTS, (double)dt * dt, P.stf, 1.0 / (0.25 * (double)M->dx * M->dx), P.kind,
                       P.gstf, P.gx0, st));
    if (grad_stf) CK(cudaMemcpyAsync(grad_stf, P.gstf, (size_t)P.S * nt * 4, cudaMemcpyDefault, st));
    if (grad_x0) CK(cudaMemcpyAsync(grad_x0, P.gx0, (size_t)P.S * 2 * 4, cudaMemcpyDefault, st));
  }
  if (seis_out && ns > 0) CK(cudaMemcpyAsync(seis_out, P.seis, (size_t)ns * 4, cudaMemcpyDefault, st));
  CK(cudaMemcpyAsync(misfit, P.J, 8, cudaMemcpyDefault, st));
  CK(mark(ctx->ev[3], st, capture));
  if (status_out) *status_out = P.status;
  if (capture) return FWI_OK;
  v = finish_status(ctx, P, st);
  grad_timings(ctx, nt, K);
  if (v == FWI_OK) g_err.clear();
  return v;
}

bool is_device_ptr(const void* p, bool or_pinned_host = false) {
  if (!p) return true;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged ||
         (or_pinned_host && a.type == cudaMemoryTypeHost);
}

}  // namespace

struct fwi_graph {
  fwi_ctx* ctx = nullptr;
  cudaGraphExec_t exec = nullptr;
  int* status = nullptr;  // device status word inside ctx's arena
  unsigned long long epoch = 0;
  int nt = 0, K = 1;       // the recorded call's steps and checkpoint interval (for its phase times)
  long long launches = 0;  // kernels of one replay
};

extern "C" {

fwi_status fwi_misfit_grad(fwi_ctx* ctx, const fwi_model* M, const fwi_sources* Sv, const fwi_receivers* R,
                           int32_t nt, float dt, const float* observed, int32_t K, double* misfit, float* grad,
                           float* grad_stf, float* grad_x0, float* seis_out, void* stream) {
  if (!ctx) return fail(FWI_EINVAL, "ctx must not be NULL");
  if (M && M->physics == FWI_ELASTIC)
    return ela_misfit_grad(ctx, M, Sv, R, nt, dt, observed, K, misfit, grad, grad_stf, grad_x0, seis_out, stream);
  return acu_misfit_grad(ctx, M, Sv, R, nt, dt, observed, K, misfit, grad, grad_stf, grad_x0, seis_out,
                         (cudaStream_t)stream, false, nullptr);
}

fwi_status fwi_forward_vjp(fwi_ctx* ctx, const fwi_model* M, const fwi_sources* Sv, const fwi_receivers* R,
                           int32_t nt, float dt, const float* cotangent, int32_t K, double* value, float* grad,
                           float* grad_stf, float* grad_x0, float* seis_out, void* stream) {
  if (!ctx) return fail(FWI_EINVAL, "ctx must not be NULL");
  if (R && R->nrec > 0 && !cotangent) return fail(FWI_EINVAL, "cotangent must not be NULL");
  // the misfit call with its residual replaced by the cotangent: the adjoint
  // sweep is the same, seeded with v instead of d - d_obs
  double local = 0.0;  // <d, v> when the caller does not want it (the call synchronises before returning)
  struct Flag {
    fwi_ctx* c;
    ~Flag() { c->vjp = false; }
  } flag{ctx};
  ctx->vjp = true;
  return fwi_misfit_grad(ctx, M, Sv, R, nt, dt, cotangent, K, value ? value : &local, grad, grad_stf, grad_x0,
                         seis_out, stream);
}

fwi_status fwi_superposed_misfit_grad(fwi_ctx* ctx, const fwi_model* M, const fwi_sources* Sv,
                                      const fwi_receivers* R, int32_t nt, float dt, const float* observed, int32_t K,
                                      double* misfit, float* grad, float* grad_stf, float* grad_x0, void* stream) {
  if (!ctx) return fail(FWI_EINVAL, "ctx must not be NULL");
  if (M && M->physics != FWI_ACOUSTIC) return fail(FWI_ENOTIMPL, "superposed sources are acoustic only");
  fwi_status v = validate(M, Sv, R, nt, dt);
  if (v != FWI_OK) return v;
  if (!misfit) return fail(FWI_EINVAL, "misfit must not be NULL");
  if (!observed && R->nrec > 0) return fail(FWI_EINVAL, "observed must not be NULL");
  if (K < 1 || K > nt) return fail(FWI_EINVAL, "ckpt_every must be in [1, nt]");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  const int S = Sv->nshots;
  const long long n = (long long)R->nrec * nt;
  // stream-ordered scratch: the S seismograms, the common residual for every
  // sub-source, the observed data, the misfit's partial sums and status word
  struct Scratch {
    cudaStream_t st;
    void* p[5] = {};
    ~Scratch() {
      for (void* q : p)
        if (q) cudaFreeAsync(q, st);
    }
  } sc{st};
  const size_t bytes[5] = {(size_t)S * n * 4 + 4, (size_t)S * n * 4 + 4, (size_t)n * 4 + 4,
                           (size_t)MISFIT_BLOCKS * 8 + 8, sizeof(int)};
  for (int k = 0; k < 5; k++)
    if (cudaMallocAsync(&sc.p[k], bytes[k], st) != cudaSuccess) {
      cudaGetLastError();
      return fail(FWI_ENOMEM, "superposed misfit: scratch allocation failed");
    }
  float *seis = (float*)sc.p[0], *cot = (float*)sc.p[1], *obs = (float*)sc.p[2];
  double* part = (double*)sc.p[3];
  double* J = part + MISFIT_BLOCKS;
  int* status = (int*)sc.p[4];
  // the S sub-source seismograms, each in its own wavefield (the equation is linear in the source)
  if ((v = fwi_forward(ctx, M, Sv, R, nt, dt, seis, stream)) != FWI_OK) return v;
  CK(cudaMemsetAsync(status, 0, sizeof(int), st));
  if (n > 0) CK(cudaMemcpyAsync(obs, observed, (size_t)n * 4, cudaMemcpyDefault, st));
  if (n > 0) LK(2, launch_superpose(seis, S, n, obs, cot, part, MISFIT_BLOCKS, J, status, st));
  else CK(cudaMemsetAsync(J, 0, 8, st));
  CK(cudaMemcpyAsync(misfit, J, 8, cudaMemcpyDefault, st));
  // the gradient: the adjoint sweep of every sub-source seeded with the common residual
  double inner = 0.0;
  if ((v = fwi_forward_vjp(ctx, M, Sv, R, nt, dt, cot, K, &inner, grad, grad_stf, grad_x0, nullptr, stream)) !=
      FWI_OK)
    return v;
  if ((v = finish_status_dev(ctx, status, st)) != FWI_OK) return v;
  g_err.clear();
  return FWI_OK;
}

fwi_status fwi_misfit_grad_graph(fwi_ctx* ctx, const fwi_model* M, const fwi_sources* Sv, const fwi_receivers* R,
                                 int32_t nt, float dt, const float* observed, int32_t K, double* misfit,
                                 float* grad, float* grad_stf, float* grad_x0, fwi_graph** out) {
  if (!ctx || !out) return fail(FWI_EINVAL, "ctx and graph must not be NULL");
  *out = nullptr;
  if (!M || M->physics != FWI_ACOUSTIC) return fail(FWI_ENOTIMPL, "graphs are recorded for the acoustic gradient only");
  fwi_status v = validate(M, Sv, R, nt, dt);
  if (v != FWI_OK) return v;
  const void* ptrs[] = {M->vp, Sv->x0, Sv->stf, R->iz, R->ix, observed, misfit, grad, grad_stf, grad_x0};
  for (const void* p : ptrs)
    if (!is_device_ptr(p, true))
      return fail(FWI_EINVAL, "every buffer of a recorded call must be device memory or page-locked host memory");
  CK(cudaSetDevice(ctx->device));
  if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
  cudaStream_t cs = ctx->cap_stream;
  // one ordinary call first: it validates the inputs on the device, sizes and
  // lays out the arena, and creates the group streams and events
  v = acu_misfit_grad(ctx, M, Sv, R, nt, dt, observed, K, misfit, grad, grad_stf, grad_x0, nullptr, cs, false,
                      nullptr);
  if (v != FWI_OK) return v;
  const unsigned long long epoch = ctx->arena_epoch;
  CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
  int* dstatus = nullptr;
  v = acu_misfit_grad(ctx, M, Sv, R, nt, dt, observed, K, misfit, grad, grad_stf, grad_x0, nullptr, cs, true,
                      &dstatus);
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(cs, &graph);
  if (v == FWI_OK && (e != cudaSuccess || ctx->arena_epoch != epoch))
    v = fail(FWI_ECUDA, std::string("graph capture: ") + (e != cudaSuccess ? cudaGetErrorString(e) : "arena changed"));
  cudaGraphExec_t exec = nullptr;
  if (v == FWI_OK) {
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    if (ei != cudaSuccess) v = fail(FWI_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ei));
  }
  if (graph) cudaGraphDestroy(graph);
  if (v != FWI_OK) {
    cudaGetLastError();
    return v;
  }
  fwi_graph* g = new fwi_graph;
  g->ctx = ctx;
  g->exec = exec;
  g->status = dstatus;
  g->epoch = epoch;
  g->nt = nt;
  g->K = K;
  g->launches = ctx->launches;
  *out = g;
  g_err.clear();
  return FWI_OK;
}

fwi_status fwi_graph_launch(fwi_graph* g, void* stream) {
  if (!g) return fail(FWI_EINVAL, "graph must not be NULL");
  if (g->ctx->arena_epoch != g->epoch)
    return fail(FWI_EINVAL, "the context's workspace was reallocated or relaid out since the graph was recorded");
  CK(cudaSetDevice(g->ctx->device));
  CK(cudaGraphLaunch(g->exec, (cudaStream_t)stream));
  return FWI_OK;
}

fwi_status fwi_graph_status(fwi_graph* g, void* stream) {
  if (!g) return fail(FWI_EINVAL, "graph must not be NULL");
  CK(cudaSetDevice(g->ctx->device));
  fwi_status v = finish_status_dev(g->ctx, g->status, (cudaStream_t)stream);
  // the replay's phase marks are complete: its timings replace the context's
  grad_timings(g->ctx, g->nt, g->K);
  g->ctx->launches = g->launches;
  if (v == FWI_OK) g_err.clear();
  return v;
}

fwi_status fwi_graph_destroy(fwi_graph* g) {
  if (!g) return FWI_OK;
  cudaSetDevice(g->ctx->device);
  if (g->exec) cudaGraphExecDestroy(g->exec);
  delete g;
  return FWI_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched gradients of several acoustic instances (fwi_batch_*). Every
// instance keeps the layout of its own single call (one plan per instance in
// one arena); a device table describes the instances, and each time step is
// ONE persistent launch over the tiles of all instances that take part in it.
// Instances are sorted by nt, longest first, so that at any step those that
// take part form a prefix. The checkpoint interval K is common, so segment
// boundaries line up across instances: every instance recomputes, stores and
// runs the adjoint of a segment in the same launches. The whole sweep (inputs,
// preparation, forward sweep, misfits, reverse sweep, folds, outputs) is
// recorded as one CUDA graph.
struct fwi_batch {
  fwi_ctx* ctx = nullptr;
  int n = 0, K = 0, N = 0, max_nt = 0;
  float dt = 0.f;
  std::vector<int> order;  // sorted position -> caller's index
  std::vector<Plan> P;
  std::vector<fwi_model> M;
  std::vector<fwi_sources> Sv;
  std::vector<fwi_receivers> R;
  std::vector<const float*> obs;
  std::vector<float*> grad;  // caller's order
  double* misfit = nullptr;  // device [n], caller's order
  std::vector<int> ts;       // first tile of each sorted instance, [n + 1]
  AcuCoef cf_fwd{}, cf_adj{};
  AcuInst* d_inst = nullptr;
  int* d_ts = nullptr;
  CopyDesc* d_copy = nullptr;
  std::vector<int> sv0, sv1, rs0, rs1;  // per checkpoint index: descriptor ranges of the saves and restores
  int* h_status = nullptr;              // pinned [n]
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap = nullptr;
};

namespace {

void batch_free(fwi_batch* B) {
  if (!B) return;
  if (B->ctx) cudaSetDevice(B->ctx->device);
  if (B->exec) cudaGraphExecDestroy(B->exec);
  if (B->cap) cudaStreamDestroy(B->cap);
  if (B->h_status) cudaFreeHost(B->h_status);
  if (B->ctx) fwi_destroy(B->ctx);
  delete B;
}

// Instances taking part in step n (nt > n): a prefix of the sorted list.
int batch_active(const fwi_batch* B, int n) {
  int a = 0;
  while (a < B->n && B->P[a].nt > n) a++;
  return a;
}

// Enqueue one whole sweep on `st` (the recorded graph is this, captured).
fwi_status batch_enqueue(fwi_batch* B, cudaStream_t st) {
  fwi_ctx* ctx = B->ctx;
  const int n = B->n, K = B->K;
  ctx->launches = 0;
  for (int i = 0; i < n; i++) {
    Plan& P = B->P[i];
    char* base = reinterpret_cast<char*>(P.status);  // the plan's layout starts with its status word
    CK(cudaMemsetAsync(base, 0, 64, st));
    CK(cudaMemsetAsync(base + P.zero_lo, 0, P.zero_hi - P.zero_lo, st));
    AcuStep p;
    fwi_status v = prepare(ctx, P, &B->M[i], &B->Sv[i], &B->R[i], B->dt, st, p);
    if (v != FWI_OK) return v;
    const long long ns = (long long)P.S * P.nrec * P.nt;
    if (ns > 0) CK(cudaMemcpyAsync(P.res, B->obs[i], (size_t)ns * 4, cudaMemcpyDefault, st));
  }
  BatchArgs b;
  memset(&b, 0, sizeof b);
  b.inst = B->d_inst;
  b.tile_start = B->d_ts;
  b.K = K;
  // forward sweep: checkpoints at segment starts, one launch per step
  for (int nn = 0; nn < B->max_nt; nn++) {
    if (nn % K == 0) {
      const int k = nn / K;
      LK(1, launch_copy_table(B->d_copy + B->sv0[k], B->sv1[k] - B->sv0[k], st));
    }
    b.n = nn;
    b.n_active = batch_active(B, nn);
    b.ntiles = B->ts[b.n_active];
    LK(1, launch_acu_fwd_batch(b, B->cf_fwd, B->N, true, st));
  }
  for (int i = 0; i < n; i++) {
    Plan& P = B->P[i];
    const long long ns = (long long)P.S * P.nrec * P.nt;
    if (ns > 0) LK(2, launch_misfit(P.seis, P.res, ns, P.Jpart, MISFIT_BLOCKS, P.J, P.status, false, st));
    else CK(cudaMemsetAsync(P.J, 0, 8, st));
  }
  // reverse sweep, segment by segment
  const int max_nseg = (B->max_nt + K - 1) / K;
  for (int seg = max_nseg - 1; seg >= 0; seg--) {
    const int n0 = seg * K, n1 = std::min(B->max_nt, n0 + K);
    int r = 0;  // instances with a later segment: they recompute this one (the forward sweep kept their last)
    while (r < n && B->P[r].nt > n0 + K) r++;
    if (r > 0) {
      LK(1, launch_copy_table(B->d_copy + B->rs0[seg], B->rs1[seg] - B->rs0[seg], st));
      for (int nn = n0; nn < n0 + K; nn++) {
        b.n = nn;
        b.n_active = r;
        b.ntiles = B->ts[r];
        LK(1, launch_acu_fwd_batch(b, B->cf_fwd, B->N, false, st));
      }
    }
    for (int nn = n1 - 1; nn >= n0; nn--) {
      for (int i = 0; i < n; i++) {
        Plan& P = B->P[i];
        if (P.nt - 1 != nn) continue;
        // adjoint seed of instance i: lambda_nt = residual of its last sample
        AcuStep pa;
        fill_step(P, &B->M[i], B->dt, pa);
        pa.res = P.res;
        pa.gpart = P.gpart;
        pa.src_part = nullptr;
        const size_t field = (size_t)P.S * P.g.slice;
        LK(1, launch_adj_init(pa, P.lam + (P.nt & 1) * field, P.hx + (P.nt & 1) * field, P.hz + (P.nt & 1) * field,
                              st));
      }
      b.n = nn;
      b.n_active = batch_active(B, nn);
      b.ntiles = B->ts[b.n_active];
      LK(1, launch_acu_adj_batch(b, B->cf_adj, B->N, st));
    }
    for (int i = 0; i < n; i++)
      if (B->P[i].nt > n0) LK(1, launch_fold(B->P[i].gpart, B->P[i].S, B->P[i].g.slice, B->P[i].G, st));
  }
  for (int i = 0; i < n; i++) {
    Plan& P = B->P[i];
    LK(1, launch_grad_c(P.G, P.g, P.c, P.grad_c, st));
    CK(cudaMemcpyAsync(B->grad[B->order[i]], P.grad_c, (size_t)P.g.nz * P.g.nx * 4, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(B->misfit + B->order[i], P.J, 8, cudaMemcpyDeviceToDevice, st));
  }
  return FWI_OK;
}

// Read every instance's status word (one synchronisation); the first failing
// instance (caller's index) in *bad.
fwi_status batch_read_status(fwi_batch* B, cudaStream_t st, int32_t* bad) {
  for (int i = 0; i < B->n; i++)
    CK(cudaMemcpyAsync(B->h_status + i, B->P[i].status, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (bad) *bad = -1;
  int first = -1, word = 0;
  for (int i = 0; i < B->n; i++)
    if (B->h_status[i] && (first < 0 || B->order[i] < first)) {
      first = B->order[i];
      word = B->h_status[i];
    }
  if (first < 0) return FWI_OK;
  if (bad) *bad = first;
  return decode_status(word, "instance " + std::to_string(first) + ": ");
}

}  // namespace

extern "C" {

fwi_status fwi_batch_create(int32_t device, int32_t n, const fwi_model* models, const fwi_sources* srcs,
                            const fwi_receivers* recs, const int32_t* nts, float dt, const float* const* observed,
                            int32_t K, double* misfit, float* const* grads, fwi_batch** out) {
  if (!out) return fail(FWI_EINVAL, "batch must not be NULL");
  *out = nullptr;
  if (n < 1 || !models || !srcs || !recs || !nts || !observed || !grads || !misfit)
    return fail(FWI_EINVAL, "a batch needs n >= 1 and non-NULL arrays");
  if (K < 1) return fail(FWI_EINVAL, "ckpt_every must be >= 1");
  for (int i = 0; i < n; i++) {
    const fwi_model* M = &models[i];
    fwi_status v = validate(M, &srcs[i], &recs[i], nts[i], dt);
    if (v != FWI_OK) return fail(v, "instance " + std::to_string(i) + ": " + g_err);
    if (M->op != FWI_OP_DIVERGENCE || srcs[i].kind == FWI_SRC_LINE)
      return fail(FWI_ENOTIMPL, "a batch takes the divergence-form operator with point or Gaussian sources");
    if (M->order != models[0].order || M->dx != models[0].dx || M->dz != models[0].dz)
      return fail(FWI_EINVAL, "the instances of a batch share order, dx and dz");
    if (recs[i].nrec > 0 && !observed[i]) return fail(FWI_EINVAL, "observed must not be NULL");
    if (!grads[i]) return fail(FWI_EINVAL, "every instance needs a gradient buffer");
    const void* ptrs[] = {M->vp, srcs[i].x0, srcs[i].stf, recs[i].iz, recs[i].ix, observed[i], grads[i]};
    for (const void* p : ptrs)
      if (!is_device_ptr(p)) return fail(FWI_EINVAL, "every buffer of a batch must be device memory");
  }
  if (!is_device_ptr(misfit)) return fail(FWI_EINVAL, "every buffer of a batch must be device memory");
  fwi_batch* B = new fwi_batch;
  fwi_status v = fwi_create(&B->ctx, device);
  if (v != FWI_OK) {
    delete B;
    return v;
  }
  auto bail = [&](fwi_status st) {
    const std::string msg = g_err;
    batch_free(B);
    g_err = msg;
    return st;
  };
#define BCK(call)                                                                                   \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess) return bail(fail(FWI_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_))); \
  } while (0)
  BCK(cudaSetDevice(device));
  BCK(cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking));
  B->n = n;
  B->K = K;
  B->N = models[0].order / 2;
  B->dt = dt;
  B->misfit = misfit;
  B->order.resize(n);
  for (int i = 0; i < n; i++) B->order[i] = i;
  std::stable_sort(B->order.begin(), B->order.end(), [&](int a, int c) { return nts[a] > nts[c]; });
  B->P.resize(n);
  size_t off = 0;
  std::vector<size_t> offs(n);
  for (int i = 0; i < n; i++) {
    const int j = B->order[i];
    B->M.push_back(models[j]);
    B->Sv.push_back(srcs[j]);
    B->R.push_back(recs[j]);
    B->obs.push_back(observed[j]);
    Plan& P = B->P[i];
    make_plan(P, &models[j], &srcs[j], &recs[j], nts[j], std::min(K, nts[j]), true);
    layout(P, nullptr);
    offs[i] = off;
    off += (P.bytes + 255) & ~size_t(255);
  }
  for (int i = 0; i < n; i++) B->grad.push_back(grads[i]);
  B->max_nt = B->P[0].nt;
  // tables after the plans: instances, tile starts, copy descriptors
  const int max_nseg = (B->max_nt + K - 1) / K;
  std::vector<CopyDesc> cp;
  B->sv0.assign(max_nseg, 0);
  B->sv1.assign(max_nseg, 0);
  B->rs0.assign(max_nseg, 0);
  B->rs1.assign(max_nseg, 0);
  const size_t o_inst = off;
  off += (sizeof(AcuInst) * n + 255) & ~size_t(255);
  const size_t o_ts = off;
  off += ((size_t)(n + 1) * 4 + 255) & ~size_t(255);
  const size_t o_copy = off;
  size_t ncopy = 0;
  for (int i = 0; i < n; i++) ncopy += 12 * (size_t)std::max(0, B->P[i].nseg - 1);
  off += (sizeof(CopyDesc) * std::max<size_t>(ncopy, 1) + 255) & ~size_t(255);
  v = arena_acquire(B->ctx, off, "batch", 0, 0, B->cap);
  if (v != FWI_OK) return bail(v);
  char* arena = B->ctx->arena;
  std::vector<AcuInst> inst(n);
  B->ts.assign(n + 1, 0);
  for (int i = 0; i < n; i++) {
    Plan& P = B->P[i];
    layout(P, arena + offs[i]);
    AcuInst& in = inst[i];
    memset(&in, 0, sizeof in);
    AcuMaps mp;
    BCK(acu_make_maps(&mp, P.g, P.S, P.u, P.m));
    BCK(acu_make_adj_maps(&mp, P.g, P.S, P.lam, P.hx, P.hz));
    in.mu = mp.u;
    in.mm = mp.m;
    in.lx = mp.lx;
    in.lz = mp.lz;
    in.hx = mp.hx;
    in.hz = mp.hz;
    fill_step(P, &B->M[i], dt, in.p);
    in.p.res = P.res;
    in.p.gpart = P.gpart;
    in.p.src_part = nullptr;
    for (int k = 0; k < 2; k++) {
      in.psix[k] = P.psix[k];
      in.psiz[k] = P.psiz[k];
      in.zx[k] = P.zx[k];
      in.zz[k] = P.zz[k];
      in.px[k] = P.px[k];
      in.pz[k] = P.pz[k];
    }
    in.hxp = P.hx;
    in.hzp = P.hz;
    in.slot = P.slot;
    in.field = (long long)P.S * P.g.slice;
    in.nt = P.nt;
    in.nlast = (P.nseg - 1) * P.K;
    B->ts[i + 1] = B->ts[i] + P.S * P.g.ntx * P.g.ntz;
    if (i == 0) {
      B->cf_fwd = AcuCoef{};
      for (int k = 0; k < 4; k++) {
        B->cf_fwd.c1x[k] = in.p.c1x[k];
        B->cf_fwd.c1z[k] = in.p.c1z[k];
        B->cf_fwd.c2x[k] = in.p.c2x[k];
        B->cf_fwd.c2z[k] = in.p.c2z[k];
        // adjoint: stage 1 -a_k dt^2/dx, stage 2 a_k/dx
        B->cf_adj.c1x[k] = -in.p.c2x[k];
        B->cf_adj.c1z[k] = -in.p.c2z[k];
        B->cf_adj.c2x[k] = in.p.c1x[k];
        B->cf_adj.c2z[k] = in.p.c1z[k];
      }
      B->cf_fwd.dt2 = B->cf_adj.dt2 = in.p.dt2;
    }
  }
  // checkpoint k (step kK) of every instance whose last segment starts later
  for (int k = 0; k < max_nseg; k++) {
    for (int pass = 0; pass < 2; pass++) {  // 0: saves, 1: restores
      (pass == 0 ? B->sv0 : B->rs0)[k] = (int)cp.size();
      const int nn = k * K;
      for (int i = 0; i < n; i++) {
        const Plan& P = B->P[i];
        if (nn >= (P.nseg - 1) * P.K) continue;
        const size_t field = (size_t)P.S * P.g.slice;
        float* ck = P.ckpt + (size_t)k * 6 * field;
        float* st6[6] = {P.u + (nn & 1) * field, P.u + ((nn + 1) & 1) * field, P.psix[nn & 1], P.psiz[nn & 1], P.zetx,
                         P.zetz};
        for (int f = 0; f < 6; f++) {
          CopyDesc d;
          d.src = reinterpret_cast<const float4*>(pass == 0 ? st6[f] : ck + f * field);
          d.dst = reinterpret_cast<float4*>(pass == 0 ? ck + f * field : st6[f]);
          d.n4 = (long long)field / 4;
          cp.push_back(d);
        }
      }
      (pass == 0 ? B->sv1 : B->rs1)[k] = (int)cp.size();
    }
  }
  B->d_inst = reinterpret_cast<AcuInst*>(arena + o_inst);
  B->d_ts = reinterpret_cast<int*>(arena + o_ts);
  B->d_copy = reinterpret_cast<CopyDesc*>(arena + o_copy);
  BCK(cudaMemcpyAsync(B->d_inst, inst.data(), sizeof(AcuInst) * n, cudaMemcpyHostToDevice, B->cap));
  BCK(cudaMemcpyAsync(B->d_ts, B->ts.data(), (size_t)(n + 1) * 4, cudaMemcpyHostToDevice, B->cap));
  if (!cp.empty())
    BCK(cudaMemcpyAsync(B->d_copy, cp.data(), sizeof(CopyDesc) * cp.size(), cudaMemcpyHostToDevice, B->cap));
  BCK(cudaStreamSynchronize(B->cap));  // the host tables are released below
  BCK(cudaMallocHost((void**)&B->h_status, sizeof(int) * n));
  // one ordinary sweep validates the inputs on the device, then the sweep is recorded
  if ((v = batch_enqueue(B, B->cap)) != FWI_OK) return bail(v);
  int32_t bad = -1;
  if ((v = batch_read_status(B, B->cap, &bad)) != FWI_OK) return bail(v);
  BCK(cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeRelaxed));
  v = batch_enqueue(B, B->cap);
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(B->cap, &graph);
  if (v == FWI_OK && e != cudaSuccess) v = fail(FWI_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  if (v == FWI_OK) {
    const cudaError_t ei = cudaGraphInstantiate(&B->exec, graph, 0);
    if (ei != cudaSuccess) v = fail(FWI_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ei));
  }
  if (graph) cudaGraphDestroy(graph);
  if (v != FWI_OK) {
    cudaGetLastError();
    return bail(v);
  }
#undef BCK
  *out = B;
  g_err.clear();
  return FWI_OK;
}

fwi_status fwi_batch_launch(fwi_batch* B, void* stream) {
  if (!B) return fail(FWI_EINVAL, "batch must not be NULL");
  CK(cudaSetDevice(B->ctx->device));
  CK(cudaGraphLaunch(B->exec, (cudaStream_t)stream));
  return FWI_OK;
}

fwi_status fwi_batch_status(fwi_batch* B, void* stream, int32_t* instance) {
  if (!B) return fail(FWI_EINVAL, "batch must not be NULL");
  CK(cudaSetDevice(B->ctx->device));
  fwi_status v = batch_read_status(B, (cudaStream_t)stream, instance);
  if (v == FWI_OK) g_err.clear();
  return v;
}

int64_t fwi_batch_launches(const fwi_batch* B) { return B ? B->ctx->launches : 0; }

fwi_status fwi_batch_destroy(fwi_batch* B) {
  batch_free(B);
  return FWI_OK;
}

}  // extern "C"

namespace {

// Workspace of one call, sized by the layout the call itself uses; the model
// and geometry must already be valid.
uint64_t workspace_of(const fwi_model* M, const fwi_sources* Sv, const fwi_receivers* R, int nt, int K) {
  if (M->physics == FWI_ELASTIC) {
    uint64_t b = 0;
    return ela_workspace_bytes(M, Sv, R, nt, K, &b) == FWI_OK ? b : UINT64_MAX;
  }
  Plan P;
  make_plan(P, M, Sv, R, nt, K, K > 0);
  layout(P, nullptr);
  return (uint64_t)P.bytes;
}

}  // namespace

extern "C" {

fwi_status fwi_workspace_bytes(const fwi_model* M, const fwi_sources* Sv, const fwi_receivers* R, int32_t nt,
                               int32_t ckpt_every, uint64_t* bytes) {
  if (!bytes) return fail(FWI_EINVAL, "bytes must not be NULL");
  if (M && M->physics == FWI_ELASTIC) {
    const fwi_status v = ela_workspace_bytes(M, Sv, R, nt, ckpt_every, bytes);
    if (v == FWI_OK) g_err.clear();
    return v;
  }
  const fwi_status v = validate(M, Sv, R, nt, 1.f);
  if (v != FWI_OK) return v;
  if (ckpt_every < 0 || ckpt_every > nt) return fail(FWI_EINVAL, "ckpt_every must be in [0, nt] (0: the forward call)");
  *bytes = workspace_of(M, Sv, R, nt, ckpt_every);
  g_err.clear();
  return FWI_OK;
}

fwi_status fwi_choose_ckpt(fwi_ctx* ctx, const fwi_model* M, const fwi_sources* Sv, const fwi_receivers* R,
                           int32_t nt, uint64_t budget_bytes, int32_t* ckpt_every) {
  if (!ckpt_every) return fail(FWI_EINVAL, "ckpt_every must not be NULL");
  uint64_t w = 0;
  fwi_status v = fwi_workspace_bytes(M, Sv, R, nt, 0, &w);  // validates the call
  if (v != FWI_OK) return v;
  uint64_t budget = budget_bytes;
  if (budget == 0) {
    if (!ctx) return fail(FWI_EINVAL, "a zero budget (the device's free memory) needs a context");
    CK(cudaSetDevice(ctx->device));
    size_t fr = 0, tot = 0;
    CK(cudaMemGetInfo(&fr, &tot));
    // the context's own arena is freed before a larger one is allocated
    const uint64_t avail = (uint64_t)fr + (uint64_t)ctx->arena_bytes;
    const uint64_t margin = std::max<uint64_t>(1ull << 30, (uint64_t)tot / 50);
    budget = avail > margin ? avail - margin : 0;
  }
  int best = 0, best_seg = 0;
  long long best_rec = 0;
  uint64_t best_w = 0, min_w = UINT64_MAX;
  int min_k = 1;
  for (int K = nt; K >= 1; K--) {
    w = workspace_of(M, Sv, R, nt, K);
    if (w < min_w) {
      min_w = w;
      min_k = K;
    }
    if (w > budget) continue;
    const int nseg = (nt + K - 1) / K;
    // recomputed forward steps: the forward sweep stores the last segment itself
    const long long rec = (long long)(nseg - 1) * K;
    if (!best || rec < best_rec || (rec == best_rec && (nseg < best_seg || (nseg == best_seg && w < best_w)))) {
      best = K;
      best_rec = rec;
      best_seg = nseg;
      best_w = w;
    }
  }
  if (!best)
    return fail(FWI_ENOMEM, "the smallest gradient workspace (" + std::to_string(min_w) + " bytes, ckpt_every = " +
                                std::to_string(min_k) + ") exceeds the budget of " + std::to_string(budget) +
                                " bytes");
  *ckpt_every = best;
  g_err.clear();
  return FWI_OK;
}

}  // extern "C"
