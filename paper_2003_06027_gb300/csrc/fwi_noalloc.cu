// fwi_noalloc.cu - forward modelling that allocates no device memory.
//
// Some callers cannot let a library call cudaMalloc: applications that give
// all device memory to their own allocator and account for every byte (a
// library allocation would fail or break their budget), and latency-sensitive
// loops that cannot afford the device-wide synchronisation cudaMalloc and
// cudaFree may cause. fwi_forward_noalloc serves them: it runs the same
// kernels as fwi_forward, but its working memory (wavefields, CPML memory
// variables, padded model, tables, source and receiver lists, status word) is
// one fixed, statically sized device array declared in this file.
//
// Costs and rules of that array:
//   - it is NOALLOC_SCRATCH_BYTES (32 MiB); every GPU on which a process loads
//     libfwi holds it until the process exits, whether or not this call is used;
//   - a problem that needs more is rejected with FWI_EINVAL and a message
//     giving the bytes it needs;
//   - every call on a device shares the same array and it keeps the previous
//     call's contents, so each call clears the part it uses before running;
//     calls whose work overlaps on the GPU (other streams, other host threads)
//     race on it and must be serialised by the caller;
//   - the first call on a device resolves the array's device address
//     (cudaGetSymbolAddress, with that device current); make that first call
//     before any stream capture is started on the device. Later calls resolve
//     it again (cheap), so a context torn down and created again (for example
//     after cudaDeviceReset) never gets a stale address; only a call made
//     while its stream is capturing reuses the address resolved earlier.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/fwi.h"
#include "fwi_internal.cuh"

namespace fwi {
cudaError_t launch_acu_fwd(const AcuStep& p, const AcuMaps& maps, bool record, bool store, cudaStream_t st);
cudaError_t acu_make_maps(AcuMaps* maps, const Grid& g, int S, float* u_pair, const float* mh);
cudaError_t launch_pad_model(const float* c, const Grid& g, float* m, cudaStream_t st);
cudaError_t launch_cpml_tables(int n_phys, int npml, int Npad, int len, double h, double dt, double R,
                               double vmax, double f0, float* a, float* b, float* ah, float* bh,
                               cudaStream_t st);
cudaError_t launch_src_prep(int S, int kind, const float* x0, const Grid& g, float dx, float dz, int* box,
                            float* w, int* status, cudaStream_t st);
cudaError_t launch_rec_csr(int nrec, const int* iz, const int* ix, const Grid& g, int* rec_cell, int* rec_key,
                           int* start, int* cursor, int* list, int* status, cudaStream_t st);
cudaError_t launch_model_check(const float* c, long long n, float coef, int* status, cudaStream_t st);
cudaError_t launch_finite_check(const float* a, long long n, int* status, cudaStream_t st);
void set_last_error(const std::string& msg);
}  // namespace fwi

using namespace fwi;

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(32) << 20;
constexpr int MAX_DEVICES = 64;

// The fixed working memory. In host code `g_scratch` is only a host-side
// stand-in for the symbol, never a device address: the address passed to the
// kernels comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[NOALLOC_SCRATCH_BYTES];

std::mutex g_mu;
void* g_scratch_dev[MAX_DEVICES] = {};

fwi_status err(fwi_status st, const std::string& msg) {
  set_last_error(msg);
  return st;
}

#define NA_CK(call)                                                                            \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return err(FWI_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// Device address of the scratch array on the current device. Resolved on every
// call outside stream capture, so that a module reloaded at another address
// (after the primary context was destroyed and created again) is followed;
// during capture (where resolving could load the module, which capture
// forbids) the address resolved by an earlier call on this device is used.
fwi_status scratch_address(cudaStream_t st, void** out) {
  int dev = 0;
  NA_CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= MAX_DEVICES) return err(FWI_EINVAL, "device index out of range");
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  NA_CK(cudaStreamIsCapturing(st, &cap));
  std::lock_guard<std::mutex> lock(g_mu);
  if (cap != cudaStreamCaptureStatusNone) {
    if (!g_scratch_dev[dev])
      return err(FWI_EINVAL, "the first fwi_forward_noalloc call on a device must come before any stream capture");
    *out = g_scratch_dev[dev];
    return FWI_OK;
  }
  void* p = nullptr;
  NA_CK(cudaGetSymbolAddress(&p, g_scratch));
  g_scratch_dev[dev] = p;
  *out = p;
  return FWI_OK;
}

// True for device memory on the current device, and for managed memory.
// Memory of another GPU is refused: the step kernels would read it directly,
// which faults without peer access.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

extern "C" fwi_status fwi_forward_noalloc(const fwi_model* M, const fwi_sources* Sv, const fwi_receivers* R,
                                          int32_t nt, float dt, float* seis, void* stream) {
  // arguments (the same contract as fwi_forward, device pointers only)
  if (!M || !Sv || !R) return err(FWI_EINVAL, "model, sources and receivers must not be NULL");
  if (M->physics != FWI_ACOUSTIC) return err(FWI_ENOTIMPL, "fwi_forward_noalloc supports FWI_ACOUSTIC only");
  if (M->nz < 1 || M->nx < 1 || !(M->dz > 0.f) || !(M->dx > 0.f) || M->npml < 0)
    return err(FWI_EINVAL, "bad grid");
  if (M->order != 4 && M->order != 8) return err(FWI_EINVAL, "order must be 4 or 8");
  if (M->npml > 0 && (!(M->pml_R > 0.f && M->pml_R < 1.f) || !(M->pml_vmax > 0.f) || !(M->pml_f0 >= 0.f)))
    return err(FWI_EINVAL, "CPML needs 0 < pml_R < 1, pml_vmax > 0, pml_f0 >= 0");
  if (Sv->nshots < 1 || (Sv->kind != FWI_SRC_POINT && Sv->kind != FWI_SRC_GAUSSIAN))
    return err(FWI_EINVAL, "bad sources");
  if (M->op != FWI_OP_DIVERGENCE) return err(FWI_ENOTIMPL, "only the divergence-form operator runs without allocation");
  if (nt < 1 || !(dt > 0.f)) return err(FWI_EINVAL, "nt must be >= 1 and dt > 0");
  if (R->nrec < 0) return err(FWI_EINVAL, "nrec must be >= 0");
  // the padded grid in 64-bit arithmetic, before any int field is formed from it
  // (the same bound as the context calls: each side <= 2^20, cells <= 2^31)
  const long long Nz_ll = (long long)M->nz + 2LL * M->npml, Nx_ll = (long long)M->nx + 2LL * M->npml;
  if (Nz_ll > (1 << 20) || Nx_ll > (1 << 20) || Nz_ll * Nx_ll > (1LL << 31)) return err(FWI_EINVAL, "grid too large");
  int dev = 0;
  NA_CK(cudaGetDevice(&dev));
  if (!on_device(M->vp, dev) || !on_device(Sv->stf, dev) || !on_device(Sv->x0, dev) ||
      (R->nrec > 0 && (!on_device(R->iz, dev) || !on_device(R->ix, dev) || !on_device(seis, dev))))
    return err(FWI_EINVAL,
               "fwi_forward_noalloc takes device pointers on the current device only (vp, stf, x0, iz, ix, seis)");
  cudaStream_t st = (cudaStream_t)stream;

  // grid and the layout of the scratch
  Grid g{};
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
  const int S = Sv->nshots, nrec = R->nrec, ntiles = g.ntx * g.ntz;
  const int tablen = std::max(g.ntx * TILE_X, g.rows - 2 * APRON) + 2 * APRON + 2 * TAB_OFF;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = (off + 255) & ~size_t(255);
    const size_t o = off;
    off += bytes;
    return o;
  };
  const size_t field = (size_t)S * (size_t)g.slice * 4;
  const size_t o_status = take(64), o_m = take((size_t)g.slice * 4), o_tab = take((size_t)8 * tablen * 4);
  const size_t o_box = take((size_t)S * 2 * 4), o_w = take((size_t)S * SRC_W * SRC_W * 4);
  const size_t o_rc = take(((size_t)nrec + 1) * 2 * 4), o_rk = take(((size_t)nrec + 1) * 4);
  const size_t o_ts = take(((size_t)ntiles * NTHREADS + 1) * 4), o_tc = take(((size_t)ntiles * NTHREADS + 1) * 4);
  const size_t o_tl = take(((size_t)nrec + 1) * 4);
  const size_t o_u = take(2 * field);  // wavefield pair, contiguous for its tensor map
  size_t o_f[6];
  for (int k = 0; k < 6; k++) o_f[k] = take(field);
  const size_t need = (off + 255) & ~size_t(255);
  if (need > NOALLOC_SCRATCH_BYTES)
    return err(FWI_EINVAL, "problem needs " + std::to_string(need) + " bytes of working memory; the fixed scratch of "
                               "fwi_forward_noalloc holds " + std::to_string(NOALLOC_SCRATCH_BYTES) +
                               " bytes (use fwi_forward)");

  void* base_v = nullptr;
  fwi_status s0 = scratch_address(st, &base_v);
  if (s0 != FWI_OK) return s0;
  char* base = (char*)base_v;
  // everything this call relies on being zero: aprons, initial state, status
  NA_CK(cudaMemsetAsync(base, 0, need, st));
  int* status = (int*)(base + o_status);
  float* T = (float*)(base + o_tab);

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
  NA_CK(launch_model_check(M->vp, (long long)g.nz * g.nx, coef, status, st));
  NA_CK(launch_pad_model(M->vp, g, (float*)(base + o_m), st));
  NA_CK(launch_cpml_tables(g.nx, g.npml, g.Nx, tablen, M->dx, dt, M->pml_R, M->pml_vmax, M->pml_f0, T, T + tablen,
                           T + 2 * tablen, T + 3 * tablen, st));
  NA_CK(launch_cpml_tables(g.nz, g.npml, g.Nz, tablen, M->dz, dt, M->pml_R, M->pml_vmax, M->pml_f0, T + 4 * tablen,
                           T + 5 * tablen, T + 6 * tablen, T + 7 * tablen, st));
  NA_CK(launch_src_prep(S, Sv->kind, Sv->x0, g, M->dx, M->dz, (int*)(base + o_box), (float*)(base + o_w), status,
                        st));
  NA_CK(launch_rec_csr(nrec, R->iz, R->ix, g, (int*)(base + o_rc), (int*)(base + o_rk), (int*)(base + o_ts),
                       (int*)(base + o_tc), (int*)(base + o_tl), status, st));

  AcuStep p;
  memset(&p, 0, sizeof p);
  p.g = g;
  p.S = S;
  p.S_pair = S;
  p.s0 = 0;
  p.N = M->order / 2;
  p.nt = nt;
  p.nrec = nrec;
  p.dt2 = dt * dt;
  for (int k = 0; k < 4; k++) {
    p.c1x[k] = a[k] / M->dx;
    p.c1z[k] = a[k] / M->dz;
    p.c2x[k] = a[k] * p.dt2 / M->dx;
    p.c2z[k] = a[k] * p.dt2 / M->dz;
  }
  p.ntiles = S * g.ntx * g.ntz;
  p.status = status;
  p.mh = (float*)(base + o_m);
  p.ax = T; p.bx = T + tablen; p.axh = T + 2 * tablen; p.bxh = T + 3 * tablen;
  p.az = T + 4 * tablen; p.bz = T + 5 * tablen; p.azh = T + 6 * tablen; p.bzh = T + 7 * tablen;
  p.u = (float*)(base + o_u);
  float* psix[2] = {(float*)(base + o_f[0]), (float*)(base + o_f[1])};
  float* psiz[2] = {(float*)(base + o_f[2]), (float*)(base + o_f[3])};
  p.zetx = (float*)(base + o_f[4]);
  p.zetz = (float*)(base + o_f[5]);
  p.src_box = (int*)(base + o_box);
  p.src_w = (float*)(base + o_w);
  p.src_n = Sv->kind == FWI_SRC_GAUSSIAN ? SRC_W : 1;
  p.stf = Sv->stf;
  p.thr_rec_start = (int*)(base + o_ts);
  p.thr_rec = (int*)(base + o_tl);
  p.rec_cell = (int*)(base + o_rc);
  p.seis = seis;
  p.x0 = Sv->x0;
  p.dx = M->dx;
  p.dz = M->dz;
  AcuMaps maps;
  NA_CK(acu_make_maps(&maps, g, S, p.u, p.mh));
  for (int n = 0; n < nt; n++) {
    p.n = n;
    p.cur = n & 1;
    p.psix_in = psix[n & 1];
    p.psix_out = psix[(n + 1) & 1];
    p.psiz_in = psiz[n & 1];
    p.psiz_out = psiz[(n + 1) & 1];
    NA_CK(launch_acu_fwd(p, maps, true, false, st));
  }
  const long long ns = (long long)S * nrec * nt;
  if (ns > 0) NA_CK(launch_finite_check(seis, ns, status, st));
  int h_status = 0;
  NA_CK(cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, st));
  NA_CK(cudaStreamSynchronize(st));
  // a timeout first: every later result of the call is invalid
  if (h_status & ST_TIMEOUT) return err(FWI_ETIMEOUT, "a step kernel gave up waiting for its tile fetch");
  if (h_status & ST_BADMODEL) return err(FWI_EINVAL, "velocity model must be finite and > 0");
  if (h_status & ST_BADREC) return err(FWI_EINVAL, "a receiver lies outside the physical grid");
  if (h_status & ST_BADSRC) return err(FWI_EINVAL, "a source (or its 7x7 Gaussian support) lies outside the grid");
  if (h_status & ST_CFL) return err(FWI_ECFL, "CFL condition violated: c_max dt sqrt(1/dx^2+1/dz^2) sum|a_k| > 1");
  if (h_status & ST_NONFINITE) return err(FWI_EUNSTABLE, "non-finite value in the seismograms");
  set_last_error("");
  return FWI_OK;
}
