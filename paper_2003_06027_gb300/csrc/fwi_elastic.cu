// fwi_elastic.cu - elastic paths of fwi_forward and fwi_misfit_grad.
//
// The velocity-stress recursion (Implementation, Eq. elastic; Eq. forward)
// with a moment-tensor source, receivers recording (vx, vz) of v^{n+1/2};
// the L2 misfit and its exact gradient with respect to lambda, mu, rho (the
// paper's elastic inversion parameters), the source time function and the
// Gaussian source position (Eqs. adjoint-backward, adjoint-gradient). Like the
// acoustic path, the forward sweep saves the full state every K steps and the
// reverse sweep recomputes each segment, keeping the five forward quantities
// the correlations need (the forces on vx, vz and the strains ex, ez, exz,
// CPML terms included).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "../../include/fwi.h"
#include "fwi_host.h"
#include "fwi_internal.cuh"

namespace fwi {
cudaError_t ela_make_maps(EleMaps* maps, const Grid& g, int S, float* const* f, float* const* a);
cudaError_t launch_ela_vel(const EleStep& p, const EleMaps& m, bool record, bool store, cudaStream_t st);
cudaError_t launch_ela_str(const EleStep& p, const EleMaps& m, bool store, cudaStream_t st);
cudaError_t launch_ela_adj(const EleStep& p, const EleMaps& m, cudaStream_t st);
cudaError_t launch_ela_medium(const float* vp, const float* vs, const float* rho, const Grid& g, float* lam,
                              float* lp2m, float* bx, float* bz, float* mxz, float* mu_pad, cudaStream_t st);
cudaError_t launch_ela_src_prep(int S, int kind, const float* x0, const Grid& g, float dx, float dz, int* box_n,
                                int* box_s, float* w_n, float* w_s, int* status, cudaStream_t st);
cudaError_t launch_ela_model_check(const float* vp, const float* vs, const float* rho, long long n, float coef,
                                   int* status, cudaStream_t st);
cudaError_t launch_ela_fold(float* const* parts, int S, long long slice, double* G, cudaStream_t st);
cudaError_t launch_ela_grad(const double* G, const Grid& g, const float* mxz, const float* mu_pad, const float* bx,
                            const float* bz, float* out, cudaStream_t st);
cudaError_t launch_cpml_tables(int n_phys, int npml, int Npad, int len, double h, double dt, double R,
                               double vmax, double f0, float* a, float* b, float* ah, float* bh,
                               cudaStream_t st);
cudaError_t launch_rec_csr(int nrec, const int* iz, const int* ix, const Grid& g, int* rec_cell, int* rec_key,
                           int* start, int* cursor, int* list, int* status, cudaStream_t st);
cudaError_t launch_misfit(const float* seis, float* res, long long n, double* part, int nb, double* J,
                          int* status, bool vjp, cudaStream_t st);
cudaError_t launch_finite_check(const float* a, long long n, int* status, cudaStream_t st);
cudaError_t launch_src_grad(const float* part, int S, int nt, int nslots, double scale, const float* stf,
                            double inv_sig2, int kind, float* gstf, float* gx0, cudaStream_t st);
}  // namespace fwi

using namespace fwi;

namespace {

constexpr int MISFIT_BLOCKS = 512;
constexpr int NSTATE = 13;  // vx, vz, sxx, szz, sxz, psi0..psi7

#define ECK(call)                                                                          \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return host_fail(FWI_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));     \
  } while (0)
#define ELK(n, call)      \
  do {                    \
    ECK(call);            \
    ctx->launches += (n); \
  } while (0)

struct EPlan {
  Grid g{};
  int S = 0, nt = 0, nrec = 0, K = 0, nseg = 0, N = 0, kind = 0, tablen = 0;
  bool grad = false;
  int* status = nullptr;
  float *lam = nullptr, *lp2m = nullptr, *bx = nullptr, *bz = nullptr, *mxz = nullptr, *mu = nullptr;
  float *tab = nullptr, *vp = nullptr, *vs = nullptr, *rho = nullptr, *stf = nullptr, *x0 = nullptr, *mt = nullptr;
  float *w_n = nullptr, *w_s = nullptr, *seis = nullptr;
  int *box_n = nullptr, *box_s = nullptr, *rec_in = nullptr, *rec_cell = nullptr, *rec_key = nullptr;
  int *tstart = nullptr, *tcursor = nullptr, *tlist = nullptr;
  float* f[NSTATE] = {};
  float* a[5] = {};
  float* M[2][8] = {};
  float* gp[5] = {};
  double* G = nullptr;
  float *src_part = nullptr, *res = nullptr, *gout = nullptr, *gstf = nullptr, *gx0 = nullptr;
  float *ckpt = nullptr, *slot = nullptr;
  double *Jpart = nullptr, *J = nullptr;
  size_t bytes = 0, zero_lo = 0, zero_hi = 0;
};

void ela_layout(EPlan& P, char* base) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    off = (off + 255) & ~size_t(255);
    char* p = base ? base + off : nullptr;
    off += bytes;
    return p;
  };
  const size_t field = (size_t)P.S * (size_t)P.g.slice * 4;
  const size_t sl = (size_t)P.g.slice * 4;
  const int nkeys = P.g.ntx * P.g.ntz * NTHREADS;
  const size_t ncell = (size_t)P.g.nz * P.g.nx * 4;
  P.status = (int*)take(64);
  P.lam = (float*)take(sl);
  P.lp2m = (float*)take(sl);
  P.bx = (float*)take(sl);
  P.bz = (float*)take(sl);
  P.mxz = (float*)take(sl);
  P.mu = (float*)take(sl);
  P.tab = (float*)take((size_t)8 * P.tablen * 4);
  P.vp = (float*)take(ncell);
  P.vs = (float*)take(ncell);
  P.rho = (float*)take(ncell);
  P.stf = (float*)take((size_t)P.S * P.nt * 4);
  P.x0 = (float*)take((size_t)P.S * 2 * 4);
  P.mt = (float*)take((size_t)P.S * 3 * 4);
  P.w_n = (float*)take((size_t)P.S * SRC_W * SRC_W * 4);
  P.w_s = (float*)take((size_t)P.S * SRC_W * SRC_W * 4);
  P.box_n = (int*)take((size_t)P.S * 2 * 4);
  P.box_s = (int*)take((size_t)P.S * 2 * 4);
  P.rec_in = (int*)take((size_t)(P.nrec + 1) * 2 * 4);
  P.rec_cell = (int*)take((size_t)(P.nrec + 1) * 2 * 4);
  P.rec_key = (int*)take((size_t)(P.nrec + 1) * 4);
  P.tstart = (int*)take((size_t)(nkeys + 1) * 4);
  P.tcursor = (int*)take((size_t)(nkeys + 1) * 4);
  P.tlist = (int*)take((size_t)(P.nrec + 1) * 4);
  P.seis = (float*)take((size_t)P.S * 2 * P.nrec * P.nt * 4 + 4);
  off = (off + 255) & ~size_t(255);
  P.zero_lo = off;
  for (int k = 0; k < NSTATE; k++) P.f[k] = (float*)take(field);
  if (P.grad) {
    for (int k = 0; k < 5; k++) P.a[k] = (float*)take(field);
    for (int b = 0; b < 2; b++)
      for (int k = 0; k < 8; k++) P.M[b][k] = (float*)take(field);
    for (int k = 0; k < 5; k++) P.gp[k] = (float*)take(field);
    P.G = (double*)take((size_t)5 * P.g.slice * 8);
    P.src_part = (float*)take((size_t)P.S * P.nt * ELA_SLOTS * 3 * 4);
  }
  off = (off + 255) & ~size_t(255);
  P.zero_hi = off;
  if (P.grad) {
    P.res = (float*)take((size_t)P.S * 2 * P.nrec * P.nt * 4 + 4);
    P.Jpart = (double*)take((size_t)MISFIT_BLOCKS * 8);
    P.J = (double*)take(8);
    P.gout = (float*)take(3 * ncell);
    P.gstf = (float*)take((size_t)P.S * P.nt * 4);
    P.gx0 = (float*)take((size_t)P.S * 2 * 4);
    P.ckpt = (float*)take(field * NSTATE * (size_t)P.nseg);
    P.slot = (float*)take(field * 5 * (size_t)P.K);
  }
  P.bytes = (off + 255) & ~size_t(255);
}

fwi_status ela_validate(const fwi_model* M, const fwi_sources* Sv, const fwi_receivers* R, int nt, float dt) {
  if (!M || !Sv || !R) return host_fail(FWI_EINVAL, "model, sources and receivers must not be NULL");
  if (M->nz < 1 || M->nx < 1) return host_fail(FWI_EINVAL, "nz and nx must be >= 1");
  if (!(M->dz > 0.f) || !(M->dx > 0.f)) return host_fail(FWI_EINVAL, "dz and dx must be > 0");
  if (M->order != 4 && M->order != 8) return host_fail(FWI_EINVAL, "order must be 4 or 8");
  if (M->npml < 0) return host_fail(FWI_EINVAL, "npml must be >= 0");
  if (M->npml > 0 && (!(M->pml_R > 0.f && M->pml_R < 1.f) || !(M->pml_vmax > 0.f) || !(M->pml_f0 >= 0.f)))
    return host_fail(FWI_EINVAL, "CPML needs 0 < pml_R < 1, pml_vmax > 0, pml_f0 >= 0");
  if (!M->vp || !M->vs || !M->rho) return host_fail(FWI_EINVAL, "elastic models need vp, vs and rho");
  if (Sv->nshots < 1) return host_fail(FWI_EINVAL, "nshots must be >= 1");
  if (Sv->kind != FWI_SRC_POINT && Sv->kind != FWI_SRC_GAUSSIAN && Sv->kind != FWI_SRC_MOMENT)
    return host_fail(FWI_EINVAL, "bad source kind");
  if (!Sv->x0 || !Sv->stf || !Sv->mt) return host_fail(FWI_EINVAL, "elastic sources need x0, stf and mt");
  if (R->nrec < 0 || (R->nrec > 0 && (!R->iz || !R->ix))) return host_fail(FWI_EINVAL, "bad receiver arrays");
  if (nt < 1 || !(dt > 0.f)) return host_fail(FWI_EINVAL, "nt must be >= 1 and dt > 0");
  const long long Nz = (long long)M->nz + 2LL * M->npml, Nx = (long long)M->nx + 2LL * M->npml;
  if (Nz > (1 << 20) || Nx > (1 << 20) || Nz * Nx > (1LL << 31)) return host_fail(FWI_EINVAL, "grid too large");
  return FWI_OK;
}

void ela_make_plan(EPlan& P, const fwi_model* M, const fwi_sources* Sv, const fwi_receivers* R, int nt, int K,
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
  g.rows = g.ntz * TILE_Z + 2 * APRON;
  g.slice = (long long)g.rows * g.pitch;
  g.off0 = (long long)APRON * g.pitch + APRON;
  P.S = Sv->nshots;
  P.nt = nt;
  P.nrec = R->nrec;
  P.N = M->order / 2;
  P.kind = Sv->kind == FWI_SRC_POINT ? 0 : 1;  // FWI_SRC_MOMENT uses the Gaussian weights
  P.grad = grad;
  P.K = grad ? K : 0;
  P.nseg = grad ? (nt + K - 1) / K : 0;
  P.tablen = std::max(g.ntx * TILE_X, g.ntz * TILE_Z) + 2 * APRON + 2 * TAB_OFF;
}

}  // namespace

// Device workspace of an elastic call: the forward call (K = 0) or the
// gradient with checkpoint interval K; the plan's own layout, sized only.
fwi_status ela_workspace_bytes(const fwi_model* M, const fwi_sources* Sv, const fwi_receivers* R, int32_t nt,
                               int32_t K, uint64_t* bytes) {
  const fwi_status v = ela_validate(M, Sv, R, nt, 1.f);
  if (v != FWI_OK) return v;
  if (K < 0 || K > nt) return host_fail(FWI_EINVAL, "ckpt_every must be in [0, nt] (0: the forward call)");
  EPlan P;
  ela_make_plan(P, M, Sv, R, nt, K, K > 0);
  ela_layout(P, nullptr);
  *bytes = (uint64_t)P.bytes;
  return FWI_OK;
}

namespace {

fwi_status ela_acquire(fwi_ctx* ctx, EPlan& P, cudaStream_t st) {
  ela_layout(P, nullptr);
  char key[256];
  snprintf(key, sizeof key, "elastic %d %d %d %d %lld %d %d %d %d %d %d", P.g.Nz, P.g.Nx, P.g.pitch, P.g.rows,
           P.g.slice, P.S, P.nt, P.nrec, P.K, (int)P.grad, P.tablen);
  fwi_status v = arena_acquire(ctx, P.bytes, key, P.zero_lo, P.zero_hi, st);
  if (v != FWI_OK) return v;
  ela_layout(P, ctx->arena);
  return FWI_OK;
}

fwi_status ela_prepare(fwi_ctx* ctx, EPlan& P, const fwi_model* M, const fwi_sources* Sv, const fwi_receivers* R,
                       float dt, cudaStream_t st, EleStep& p) {
  const Grid& g = P.g;
  const size_t ncell = (size_t)g.nz * g.nx * 4;
  ECK(cudaMemcpyAsync(P.vp, M->vp, ncell, cudaMemcpyDefault, st));
  ECK(cudaMemcpyAsync(P.vs, M->vs, ncell, cudaMemcpyDefault, st));
  ECK(cudaMemcpyAsync(P.rho, M->rho, ncell, cudaMemcpyDefault, st));
  ECK(cudaMemcpyAsync(P.stf, Sv->stf, (size_t)P.S * P.nt * 4, cudaMemcpyDefault, st));
  ECK(cudaMemcpyAsync(P.x0, Sv->x0, (size_t)P.S * 2 * 4, cudaMemcpyDefault, st));
  ECK(cudaMemcpyAsync(P.mt, Sv->mt, (size_t)P.S * 3 * 4, cudaMemcpyDefault, st));
  if (P.nrec > 0) {
    ECK(cudaMemcpyAsync(P.rec_in, R->iz, (size_t)P.nrec * 4, cudaMemcpyDefault, st));
    ECK(cudaMemcpyAsync(P.rec_in + P.nrec, R->ix, (size_t)P.nrec * 4, cudaMemcpyDefault, st));
  }
  float a[4] = {0.f, 0.f, 0.f, 0.f};
  if (M->order == 4) {
    a[0] = (float)(9.0 / 8.0);
    a[1] = (float)(-1.0 / 24.0);
  } else {
    a[0] = (float)(1225.0 / 1024.0);
    a[1] = (float)(-245.0 / 3072.0);
    a[2] = (float)(49.0 / 5120.0);
    a[3] = (float)(-5.0 / 7168.0);
  }
  const float sa = fabsf(a[0]) + fabsf(a[1]) + fabsf(a[2]) + fabsf(a[3]);
  const float coef = dt * sqrtf(1.f / (M->dx * M->dx) + 1.f / (M->dz * M->dz)) * sa;
  ELK(1, launch_ela_model_check(P.vp, P.vs, P.rho, (long long)g.nz * g.nx, coef, P.status, st));
  ELK(1, launch_ela_medium(P.vp, P.vs, P.rho, g, P.lam, P.lp2m, P.bx, P.bz, P.mxz, P.mu, st));
  const int L = P.tablen;
  float* T = P.tab;
  ELK(1, launch_cpml_tables(g.nx, g.npml, g.Nx, L, M->dx, dt, M->pml_R, M->pml_vmax, M->pml_f0, T, T + L, T + 2 * L,
                            T + 3 * L, st));
  ELK(1, launch_cpml_tables(g.nz, g.npml, g.Nz, L, M->dz, dt, M->pml_R, M->pml_vmax, M->pml_f0, T + 4 * L,
                            T + 5 * L, T + 6 * L, T + 7 * L, st));
  ELK(1, launch_ela_src_prep(P.S, P.kind, P.x0, g, M->dx, M->dz, P.box_n, P.box_s, P.w_n, P.w_s, P.status, st));
  ELK(1, launch_rec_csr(P.nrec, P.rec_in, P.rec_in + P.nrec, g, P.rec_cell, P.rec_key, P.tstart, P.tcursor, P.tlist,
                        P.status, st));
  memset(&p, 0, sizeof p);
  p.g = g;
  p.S = P.S;
  p.N = P.N;
  p.nt = P.nt;
  p.nrec = P.nrec;
  for (int k = 0; k < 4; k++) {
    p.cx[k] = a[k] / M->dx;
    p.cz[k] = a[k] / M->dz;
  }
  p.dt = dt;
  p.bx = P.bx;
  p.bz = P.bz;
  p.lam = P.lam;
  p.lp2m = P.lp2m;
  p.mxz = P.mxz;
  p.ax = T; p.bxt = T + L; p.axh = T + 2 * L; p.bxh = T + 3 * L;
  p.az = T + 4 * L; p.bzt = T + 5 * L; p.azh = T + 6 * L; p.bzh = T + 7 * L;
  p.vx = P.f[0];
  p.vz = P.f[1];
  p.sxx = P.f[2];
  p.szz = P.f[3];
  p.sxz = P.f[4];
  for (int k = 0; k < 8; k++) p.psi[k] = P.f[5 + k];
  p.box_n = P.box_n;
  p.box_s = P.box_s;
  p.w_n = P.w_n;
  p.w_s = P.w_s;
  p.src_n = P.kind == 1 ? SRC_W : 1;
  p.stf = P.stf;
  p.mt = P.mt;
  p.thr_rec_start = P.tstart;
  p.thr_rec = P.tlist;
  p.seis = P.seis;
  p.x0 = P.x0;
  p.dx = M->dx;
  p.dz = M->dz;
  p.status = P.status;
  (void)ctx;
  return FWI_OK;
}

}  // namespace

fwi_status ela_forward(fwi_ctx* ctx, const fwi_model* M, const fwi_sources* Sv, const fwi_receivers* R, int32_t nt,
                       float dt, float* seis, void* stream) {
  fwi_status v = ela_validate(M, Sv, R, nt, dt);
  if (v != FWI_OK) return v;
  if (!seis && R->nrec > 0) return host_fail(FWI_EINVAL, "seis must not be NULL");
  ECK(cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  EPlan P;
  ela_make_plan(P, M, Sv, R, nt, 0, false);
  v = ela_acquire(ctx, P, st);
  if (v != FWI_OK) return v;
  EleStep p;
  ctx->launches = 0;
  v = ela_prepare(ctx, P, M, Sv, R, dt, st, p);
  if (v != FWI_OK) return v;
  EleMaps maps;
  ECK(ela_make_maps(&maps, P.g, P.S, P.f, nullptr));
  ensure_events(ctx, 0);
  ECK(cudaEventRecord(ctx->ev[0], st));
  for (int n = 0; n < nt; n++) {
    p.n = n;
    ELK(1, launch_ela_vel(p, maps, true, false, st));
    ELK(1, launch_ela_str(p, maps, false, st));
  }
  ECK(cudaEventRecord(ctx->ev[1], st));
  const long long ns = (long long)P.S * 2 * P.nrec * nt;
  if (ns > 0) {
    ELK(1, launch_finite_check(P.seis, ns, P.status, st));
    ECK(cudaMemcpyAsync(seis, P.seis, (size_t)ns * 4, cudaMemcpyDefault, st));
  }
  ECK(cudaEventRecord(ctx->ev[3], st));
  v = finish_status_dev(ctx, P.status, st);
  float t = 0.f;
  cudaEventElapsedTime(&t, ctx->ev[0], ctx->ev[1]);
  ctx->phase_ms[0] = t;
  ctx->phase_ms[1] = 0.f;
  cudaEventElapsedTime(&t, ctx->ev[0], ctx->ev[3]);
  ctx->phase_ms[2] = t;
  ctx->kernel_ms[0] = ctx->phase_ms[0] / nt;  // one velocity + one stress launch per step
  ctx->kernel_ms[1] = 0.f;
  ctx->kernel_ms[2] = 0.f;
  if (v == FWI_OK) host_fail(FWI_OK, "");
  return v;
}

fwi_status ela_misfit_grad(fwi_ctx* ctx, const fwi_model* M, const fwi_sources* Sv, const fwi_receivers* R,
                           int32_t nt, float dt, const float* observed, int32_t K, double* misfit, float* grad,
                           float* grad_stf, float* grad_x0, float* seis_out, void* stream) {
  fwi_status v = ela_validate(M, Sv, R, nt, dt);
  if (v != FWI_OK) return v;
  if (!observed && R->nrec > 0) return host_fail(FWI_EINVAL, "observed must not be NULL");
  if (!misfit) return host_fail(FWI_EINVAL, "misfit must not be NULL");
  if (K < 1 || K > nt) return host_fail(FWI_EINVAL, "ckpt_every must be in [1, nt]");
  ECK(cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  EPlan P;
  ela_make_plan(P, M, Sv, R, nt, K, true);
  v = ela_acquire(ctx, P, st);
  if (v != FWI_OK) return v;
  EleStep p;
  ctx->launches = 0;
  v = ela_prepare(ctx, P, M, Sv, R, dt, st, p);
  if (v != FWI_OK) return v;
  EleMaps maps;
  ECK(ela_make_maps(&maps, P.g, P.S, P.f, P.a));
  const long long ns = (long long)P.S * 2 * P.nrec * nt;
  if (ns > 0) ECK(cudaMemcpyAsync(P.res, observed, (size_t)ns * 4, cudaMemcpyDefault, st));
  const size_t field = (size_t)P.S * P.g.slice;
  ensure_events(ctx, P.nseg);

  // forward sweep with a full-state checkpoint at the start of every segment
  // but the last: over the last segment the sweep stores the forces and
  // strains itself (recording and storing in one launch), so that segment is
  // never recomputed
  const int nlast = (P.nseg - 1) * K;
  ECK(cudaEventRecord(ctx->ev[0], st));
  for (int n = 0; n < nt; n++) {
    if (n % K == 0 && n < nlast) {
      float* ck = P.ckpt + (size_t)(n / K) * NSTATE * field;
      for (int f = 0; f < NSTATE; f++)
        ECK(cudaMemcpyAsync(ck + f * field, P.f[f], field * 4, cudaMemcpyDeviceToDevice, st));
    }
    p.n = n;
    const bool keep = n >= nlast;
    if (keep)
      for (int k = 0; k < 5; k++) p.slot[k] = P.slot + ((size_t)(n - nlast) * 5 + k) * field;
    ELK(1, launch_ela_vel(p, maps, true, keep, st));
    ELK(1, launch_ela_str(p, maps, keep, st));
  }
  ECK(cudaEventRecord(ctx->ev[1], st));
  if (ns > 0) ELK(2, launch_misfit(P.seis, P.res, ns, P.Jpart, MISFIT_BLOCKS, P.J, P.status, ctx->vjp, st));
  else ECK(cudaMemsetAsync(P.J, 0, 8, st));

  // reverse sweep
  p.Vx = P.a[0];
  p.Vz = P.a[1];
  p.Sxx = P.a[2];
  p.Szz = P.a[3];
  p.Sxz = P.a[4];
  p.res = P.res;
  p.g_lam = P.gp[0];
  p.g_mu = P.gp[1];
  p.g_mxz = P.gp[2];
  p.g_bx = P.gp[3];
  p.g_bz = P.gp[4];
  p.src_part = P.src_part;
  for (int seg = P.nseg - 1; seg >= 0; seg--) {
    const int n0 = seg * K, n1 = std::min(nt, n0 + K);
    ECK(cudaEventRecord(ctx->seg_ev[4 * seg + 0], st));
    if (seg < P.nseg - 1) {  // the last segment's slots are already filled by the forward sweep
      const float* ck = P.ckpt + (size_t)seg * NSTATE * field;
      for (int f = 0; f < NSTATE; f++)
        ECK(cudaMemcpyAsync(P.f[f], ck + f * field, field * 4, cudaMemcpyDeviceToDevice, st));
      for (int n = n0; n < n1; n++) {
        p.n = n;
        for (int k = 0; k < 5; k++) p.slot[k] = P.slot + ((size_t)(n - n0) * 5 + k) * field;
        ELK(1, launch_ela_vel(p, maps, false, true, st));
        ELK(1, launch_ela_str(p, maps, true, st));
      }
    }
    ECK(cudaEventRecord(ctx->seg_ev[4 * seg + 1], st));
    for (int n = n1 - 1; n >= n0; n--) {
      p.n = n;
      for (int k = 0; k < 5; k++) p.slot[k] = P.slot + ((size_t)(n - n0) * 5 + k) * field;
      const int in = (n + 1) & 1, out = n & 1;
      for (int k = 0; k < 8; k++) {
        p.Min[k] = P.M[in][k];
        p.Mout[k] = P.M[out][k];
      }
      ELK(2, launch_ela_adj(p, maps, st));
    }
    ECK(cudaEventRecord(ctx->seg_ev[4 * seg + 2], st));
    ELK(1, launch_ela_fold(P.gp, P.S, P.g.slice, P.G, st));
  }
  ECK(cudaEventRecord(ctx->ev[2], st));
  if (grad) {
    ELK(1, launch_ela_grad(P.G, P.g, P.mxz, P.mu, P.bx, P.bz, P.gout, st));
    ECK(cudaMemcpyAsync(grad, P.gout, (size_t)3 * P.g.nz * P.g.nx * 4, cudaMemcpyDefault, st));
  }
  if (grad_stf || grad_x0) {
    ELK(1, launch_src_grad(P.src_part, P.S, nt, ELA_SLOTS, -(double)dt, P.stf, 1.0 / (0.25 * (double)M->dx * M->dx),
                           P.kind, P.gstf, P.gx0, st));
    if (grad_stf) ECK(cudaMemcpyAsync(grad_stf, P.gstf, (size_t)P.S * nt * 4, cudaMemcpyDefault, st));
    if (grad_x0) ECK(cudaMemcpyAsync(grad_x0, P.gx0, (size_t)P.S * 2 * 4, cudaMemcpyDefault, st));
  }
  if (seis_out && ns > 0) ECK(cudaMemcpyAsync(seis_out, P.seis, (size_t)ns * 4, cudaMemcpyDefault, st));
  ECK(cudaMemcpyAsync(misfit, P.J, 8, cudaMemcpyDefault, st));
  ECK(cudaEventRecord(ctx->ev[3], st));
  v = finish_status_dev(ctx, P.status, st);
  float t = 0.f;
  cudaEventElapsedTime(&t, ctx->ev[0], ctx->ev[1]);
  ctx->phase_ms[0] = t;
  cudaEventElapsedTime(&t, ctx->ev[1], ctx->ev[2]);
  ctx->phase_ms[1] = t;
  cudaEventElapsedTime(&t, ctx->ev[0], ctx->ev[3]);
  ctx->phase_ms[2] = t;
  ctx->kernel_ms[0] = ctx->phase_ms[0] / nt;
  float rec = 0.f, adj = 0.f;
  for (int seg = 0; seg < P.nseg; seg++) {
    float ta = 0.f;
    cudaEventElapsedTime(&ta, ctx->seg_ev[4 * seg + 0], ctx->seg_ev[4 * seg + 1]);
    rec += ta;
    cudaEventElapsedTime(&ta, ctx->seg_ev[4 * seg + 1], ctx->seg_ev[4 * seg + 2]);
    adj += ta;
  }
  ctx->kernel_ms[1] = nlast > 0 ? rec / nlast : 0.f;  // per recomputed step (checkpoint restores included)
  ctx->kernel_ms[2] = adj / nt;
  if (v == FWI_OK) host_fail(FWI_OK, "");
  return v;
}
