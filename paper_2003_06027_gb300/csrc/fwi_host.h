// fwi_host.h - host-side context and helpers shared by the orchestration
// files of libfwi (not part of the public ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/fwi.h"

struct fwi_ctx {
  int device = 0;
  char* arena = nullptr;
  size_t arena_bytes = 0;
  std::string layout_key;   // layout of the arena's current contents
  int* h_status = nullptr;  // pinned
  cudaEvent_t ev[4] = {};
  std::vector<cudaEvent_t> seg_ev;
  float phase_ms[3] = {0, 0, 0};
  float kernel_ms[3] = {0, 0, 0};
  int64_t launches = 0;
  // shot groups run concurrently on these streams, forked from and joined to the call's stream
  cudaStream_t gstream[4] = {};
  cudaEvent_t fork_ev = nullptr;
  cudaEvent_t join_ev[4] = {};
  // bumped whenever the arena is reallocated or takes a new layout: a recorded
  // graph (fwi_misfit_grad_graph) is valid only for the epoch it was captured in
  unsigned long long arena_epoch = 0;
  int fwd_groups = 0, adj_groups = 0;  // shot groups of the acoustic step launches (0: the library's default)
  int fwd_tile_rows = 0;               // tile height of the acoustic forward steps: 32 or 64 (0: 32)
  cudaStream_t cap_stream = nullptr;  // stream the graphs are captured on
  // set for the duration of an fwi_forward_vjp call: the "observed" buffer holds
  // the cotangent, which seeds the adjoint sweep as it stands
  bool vjp = false;
};

namespace fwi {
fwi_status host_fail(fwi_status st, const std::string& msg);
fwi_status arena_acquire(fwi_ctx* ctx, size_t bytes, const std::string& key, size_t zero_lo, size_t zero_hi,
                         cudaStream_t st);
fwi_status finish_status_dev(fwi_ctx* ctx, const int* d_status, cudaStream_t st);
fwi_status decode_status(int status_word, const std::string& where);
void ensure_events(fwi_ctx* ctx, size_t nseg);
}  // namespace fwi

// elastic paths of fwi_forward / fwi_misfit_grad (fwi_elastic.cu)
fwi_status ela_forward(fwi_ctx* ctx, const fwi_model* M, const fwi_sources* Sv, const fwi_receivers* R, int32_t nt,
                       float dt, float* seis, void* stream);
fwi_status ela_workspace_bytes(const fwi_model* M, const fwi_sources* Sv, const fwi_receivers* R, int32_t nt,
                               int32_t K, uint64_t* bytes);
fwi_status ela_misfit_grad(fwi_ctx* ctx, const fwi_model* M, const fwi_sources* Sv, const fwi_receivers* R,
                           int32_t nt, float dt, const float* observed, int32_t K, double* misfit, float* grad,
                           float* grad_stf, float* grad_x0, float* seis_out, void* stream);
