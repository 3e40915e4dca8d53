/*
 * fwi.h - C ABI of the GB300 seismic-inversion library (libfwi.so).
 *
 * The library implements the hot path of the seismic-inversion method of
 * Zhu, Xu, Darve & Beroza, "A General Approach to Seismic Inversion with
 * Automatic Differentiation": explicit time stepping of the 2D acoustic wave
 * equation u_tt = div(c^2 grad u) + f (Implementation, Eq. acoustic) and of
 * the 2D elastic velocity-stress system (Implementation, Eq. elastic) on
 * staggered grids with convolutional PML, receiver sampling, the L2 misfit
 * J = 1/2 sum_k |U_k - U_k^obs|^2 (Method, after Eq. forward), and its exact
 * gradient by the adjoint recursion lambda_k = A^T lambda_{k+1} + (U_k - U_k^obs)
 * (Eq. adjoint-backward) with sum_k lambda_k^T (dA/dtheta) U_{k-1}
 * (Eq. adjoint-gradient), which the paper's Theorem shows to be identical to
 * reverse-mode automatic differentiation.
 *
 * Conventions shared by every call
 *   - Arrays are row-major, x (the horizontal index) fastest. The physical
 *     model is [nz][nx]; npml CPML cells are added OUTSIDE it on all four
 *     sides. Positions in metres are physical coordinates: x = ix*dx,
 *     z = iz*dz, with (0,0) the first physical cell.
 *   - Every array pointer may point to host memory (pageable or pinned) or to
 *     device memory of the context's device; the library detects which and
 *     copies host data through its own device workspace. The caller keeps
 *     ownership of all its arrays; the library never frees them.
 *   - Calls enqueue work on the given CUDA stream (NULL = legacy default
 *     stream) and return after the stream has finished the call's work (the
 *     status of the numerical checks is known only then). Outputs are
 *     overwritten, never accumulated.
 *   - FP32 storage and arithmetic for wavefields; FP64 for the misfit and for
 *     the reductions of the gradient over time segments and shots.
 *   - Results are deterministic run to run (no floating-point atomics).
 *   - No call throws; each returns a status, and fwi_last_error() gives a
 *     message for the calling thread.
 *   - A context is not thread-safe: use one context per host thread.
 */
#ifndef FWI_H
#define FWI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FWI_OK = 0,
  FWI_EINVAL = 1,     /* bad argument: sizes, NULL pointer, position outside the grid */
  FWI_ECFL = 2,       /* c_max dt sqrt(1/dx^2 + 1/dz^2) sum_k |a_k| > 1 (unstable) */
  FWI_ENOMEM = 3,     /* device workspace could not be allocated */
  FWI_ECUDA = 4,      /* a CUDA runtime call failed (message in fwi_last_error) */
  FWI_EUNSTABLE = 5,  /* non-finite value in the seismograms or the misfit */
  FWI_ETIMEOUT = 6,   /* a bounded device wait gave up (results invalid; context usable) */
  FWI_ENOTIMPL = 7    /* combination the library does not implement */
} fwi_status;

enum { FWI_ACOUSTIC = 0, FWI_ELASTIC = 1 };
/* Acoustic operator: the paper's divergence form div(c^2 grad u) (Eq.
 * acoustic; staggered, c^2 averaged to the half points), or the c^2 Laplacian
 * form c^2 (D-x D+x u + D-z D+z u) with c^2 at the cells (same derivatives and
 * CPML). They coincide in homogeneous media and differ at interfaces (normal
 * reflection (c1 - c2)/(c1 + c2) against (c2 - c1)/(c2 + c1)). The Laplacian
 * form runs on plain per-point kernels, not on the tiled kernels of the
 * divergence form. */
enum { FWI_OP_DIVERGENCE = 0, FWI_OP_LAPLACIAN = 1 };
enum { FWI_SRC_POINT = 0, FWI_SRC_GAUSSIAN = 1, FWI_SRC_MOMENT = 2, FWI_SRC_LINE = 3 };

typedef struct fwi_ctx fwi_ctx; /* opaque; owns only its device workspace */

/* Medium and discretisation.
 * physics  FWI_ACOUSTIC (uses vp = c only) or FWI_ELASTIC (vp, vs, rho).
 * nz, nx   physical grid, >= 1.   dz, dx  spacing in metres, > 0.
 * order    spatial order of the staggered first derivative: 4 or 8.
 * npml     CPML thickness in cells, >= 0 (0 = rigid u = 0 boundary).
 * pml_R, pml_vmax, pml_f0  CPML constants: target reflection, the velocity
 *          that sets the damping (a fixed input, not differentiated) and the
 *          frequency that sets alpha_max = pi f0.
 * vp, vs, rho  [nz][nx] FP32 fields (m/s, m/s, kg/m^3); acoustic needs vp. */
typedef struct {
  int32_t physics;
  int32_t nz, nx;
  float dz, dx;
  int32_t order;
  int32_t npml;
  float pml_R, pml_vmax, pml_f0;
  const float *vp, *vs, *rho;
  int32_t op;  /* acoustic operator: FWI_OP_DIVERGENCE (0) or FWI_OP_LAPLACIAN (1) */
} fwi_model;

/* Sources, one per shot.
 * kind  FWI_SRC_POINT: weight 1/(dx dz) on the cell nearest x0, which must be
 *       a physical cell. FWI_SRC_GAUSSIAN: the paper's re-parameterisation
 *       g(t)/(2 pi s^2) exp(-|x - x0|^2 / (2 s^2)), s = dx/2, over the 7 x 7
 *       cells around the nearest cell (Earthquake Location and Source Time
 *       Function Retrieval); the 7 x 7 support must lie in the padded grid.
 * x0    [nshots][2] (x, z) in metres.
 * stf   [nshots][nt] source time function g(t_n), t_n = n dt.
 * mt    [nshots][3] moment tensor (Mxx, Mzz, Mxz): required for FWI_ELASTIC,
 *       ignored for FWI_ACOUSTIC. Elastic sources inject sigma <- sigma -
 *       dt M g(t_n) w into the stresses at step n (g is the moment rate), with
 *       point or Gaussian weights w on the normal-stress grid and on the shear
 *       grid (offset by half a cell); FWI_SRC_MOMENT means Gaussian weights.
 *       FWI_SRC_LINE (acoustic): the paper's plane-wave sources, as a row of
 *       line_len physical cells starting at the cell nearest x0 (x of the
 *       first cell, z of the row), each cell with weight 1/(dx dz) and its own
 *       time function: stf is then [nshots][nt][line_len] and grad_stf of
 *       fwi_misfit_grad has that shape too (grad_x0 must be NULL). A plane
 *       wave is the same wavelet delayed linearly along the row.
 * line_len  cells of a FWI_SRC_LINE source (ignored otherwise). */
typedef struct {
  int32_t nshots;
  int32_t kind;
  const float *x0;
  const float *stf;
  const float *mt;
  int32_t line_len;
} fwi_sources;

/* Receivers, shared by all shots: physical cell indices iz[r], ix[r]. An
 * elastic receiver records vx at (iz, ix+1/2) and vz at (iz+1/2, ix), the
 * staggered velocity nodes of its cell. */
typedef struct {
  int32_t nrec;
  const int32_t *iz, *ix;
} fwi_receivers;

/* Create a context bound to CUDA device `device`. The workspace is allocated
 * on first use and grown when a larger problem arrives. */
fwi_status fwi_create(fwi_ctx **ctx, int device);

/* Free the context and its workspace (waits for its device work). */
fwi_status fwi_destroy(fwi_ctx *ctx);

/* Forward modelling (Eq. forward).
 * Acoustic: seis[s][r][n] = u^{n+1} at receiver r of shot s, n = 0..nt-1,
 *   u^0 = u^{-1} = 0, source term dt^2 g(t_n) w at step n; seis [nshots][nrec][nt].
 * Elastic: seis[s][c][r][n] = component c (0 vx, 1 vz) of v^{n+1/2} at receiver
 *   r; v^{-1/2} = 0, sigma^0 = 0; seis [nshots][2][nrec][nt].
 * FP32. */
fwi_status fwi_forward(fwi_ctx *ctx, const fwi_model *model, const fwi_sources *src,
                       const fwi_receivers *rec, int32_t nt, float dt, float *seis,
                       void *cuda_stream);

/* Misfit and exact gradient (Eqs. adjoint-backward and adjoint-gradient).
 * observed   FP32 observed seismograms, shaped like seis of fwi_forward.
 * ckpt_every wavefield checkpoint interval K (1..nt); the reverse sweep
 *            recomputes each K-step segment from its checkpoint. Acoustic
 *            calls keep the last segment's stored fields from the forward
 *            sweep itself, so only the first ceil(nt/K) - 1 segments are
 *            recomputed: K = nt recomputes nothing, at the cost of 2 nt
 *            stored fields (each nshots x the tile-aligned padded grid, FP32).
 * misfit     J = 1/2 sum_{s,r,n} (seis - observed)^2, one double (host or device).
 * grad       acoustic: [nz][nx] dJ/dc; elastic: [3][nz][nx] the partial
 *            derivatives dJ/dlambda, dJ/dmu, dJ/drho (lambda = rho (vp^2 - 2 vs^2),
 *            mu = rho vs^2, the paper's elastic inversion parameters); or NULL.
 * grad_stf   [nshots][nt] dJ/dg(t_n), or NULL.
 * grad_x0    [nshots][2] dJ/dx0 (Gaussian sources; zero for point sources), or NULL.
 * seis_out   the predicted seismograms (shaped like observed), or NULL. */
fwi_status fwi_misfit_grad(fwi_ctx *ctx, const fwi_model *model, const fwi_sources *src,
                           const fwi_receivers *rec, int32_t nt, float dt,
                           const float *observed, int32_t ckpt_every, double *misfit,
                           float *grad, float *grad_stf, float *grad_x0, float *seis_out,
                           void *cuda_stream);

/* Vector-Jacobian product of the forward map d = F(theta): for a cotangent
 * v = dL/dd of any scalar L of the seismograms, the adjoint sweep seeded with
 * v at the receivers gives (dF/dtheta)^T v. This is the reverse-mode rule of
 * the paper's AD section applied step by step (dU_k/dU_{k-1} = A^T, Eq.
 * ad-backward), with the misfit derivative d - d_obs of Eq. adjoint-backward
 * replaced by v; fwi_misfit_grad is the special case v = d - d_obs.
 * Arguments as fwi_misfit_grad, except:
 * cotangent  v, shaped like the seismograms ([S][nrec][nt] acoustic,
 *            [S][2][nrec][nt] elastic), host or device; NULL only if nrec = 0.
 * value      <d, v> = sum of seis * cotangent in FP64 (the linear functional
 *            whose gradient is returned), one double (host or device), or NULL.
 * grad, grad_stf, grad_x0  (dF/dtheta)^T v for the model (acoustic c;
 *            elastic lambda, mu, rho), the source time functions and the
 *            source positions, laid out as in fwi_misfit_grad; each may be NULL.
 * Same checkpointing, status codes (FWI_EUNSTABLE on a non-finite <d, v>) and
 * synchronisation as fwi_misfit_grad. */
fwi_status fwi_forward_vjp(fwi_ctx *ctx, const fwi_model *model, const fwi_sources *src,
                           const fwi_receivers *rec, int32_t nt, float dt,
                           const float *cotangent, int32_t ckpt_every, double *value,
                           float *grad, float *grad_stf, float *grad_x0, float *seis_out,
                           void *cuda_stream);

/* Misfit of sub-sources acting together (the rupture imaging of the paper's
 * source-inversion applications): the nshots sources of src are the
 * sub-sources of ONE event, each propagated in its own wavefield (the wave
 * equation is linear in the source), and the event's seismograms are their sum:
 *   J = 1/2 sum_{r,n} (sum_s d_s - observed)^2,
 * with the gradients of the sub-sources' time functions and positions (and the
 * model) from the adjoint sweep of every sub-source seeded with the common
 * residual sum_s d_s - observed. The sum, the residual and J (FP64) are formed on
 * the device. Acoustic models only (FWI_ENOTIMPL otherwise).
 * observed   [nrec][nt] FP32, host or device (one event, not per sub-source).
 * Other arguments, outputs and status codes as fwi_misfit_grad (grad_stf
 * [nshots][nt], grad_x0 [nshots][2], grad [nz][nx], each may be NULL). Runs a
 * forward call and a vector-Jacobian call on ctx; its scratch comes from the
 * stream-ordered allocator (FWI_ENOMEM if that fails). Synchronises. */
fwi_status fwi_superposed_misfit_grad(fwi_ctx *ctx, const fwi_model *model, const fwi_sources *src,
                                      const fwi_receivers *rec, int32_t nt, float dt, const float *observed,
                                      int32_t ckpt_every, double *misfit, float *grad, float *grad_stf,
                                      float *grad_x0, void *cuda_stream);

/* Device workspace (bytes) that a call allocates in its context: the forward
 * call (ckpt_every = 0) or fwi_misfit_grad with checkpoint interval
 * ckpt_every (1..nt), for the given model, sources, receivers and nt; sized
 * by the layout the call itself uses, so a context whose arena is at least
 * this large allocates nothing for that call. The dominant terms are fields
 * of nshots x R x P floats, R = ceil(Nz/64)*64 + 16 rows (acoustic; elastic
 * ceil(Nz/32)*32 + 16) and
 * P = ceil(Nx/64)*64 + 16 columns (the padded grid Nz x Nx, tile-aligned,
 * with an 8-cell apron): per gradient call 6 per checkpoint (ceil(nt/K) of
 * them, acoustic; 13 elastic) and 2 per step of a segment (K of them,
 * acoustic; 1 with FWI_OP_LAPLACIAN, whose storing step keeps one field; 5
 * elastic). Host arithmetic only: no device is touched; inputs are
 * validated as by the call (FWI_EINVAL, FWI_ENOTIMPL). */
fwi_status fwi_workspace_bytes(const fwi_model *model, const fwi_sources *src,
                               const fwi_receivers *rec, int32_t nt, int32_t ckpt_every,
                               uint64_t *bytes);

/* Checkpoint interval for fwi_misfit_grad that fits a memory budget: among
 * the K in [1, nt] whose workspace (fwi_workspace_bytes) is at most
 * budget_bytes, the one that recomputes the fewest forward steps
 * ((ceil(nt/K) - 1) K, acoustic and elastic, since the forward sweep keeps the
 * last segment), then the fewest segments, then the least memory. K = nt
 * (no recomputation) whenever it fits. budget_bytes = 0 means the device's
 * free memory plus ctx's current arena, less max(1 GiB, 2% of the device):
 * that needs ctx; an explicit budget needs no device (ctx may be NULL).
 * FWI_ENOMEM (with the smallest workspace in fwi_last_error) if no K fits. */
fwi_status fwi_choose_ckpt(fwi_ctx *ctx, const fwi_model *model, const fwi_sources *src,
                           const fwi_receivers *rec, int32_t nt, uint64_t budget_bytes,
                           int32_t *ckpt_every);

/* Tile shape of the acoustic forward steps of ctx's calls (forward sweep and
 * segment recompute): tiles of 64 columns x forward_tile_rows rows, 32 (256
 * threads per CTA) or 64 (512 threads; half the z-halo flux recompute per cell,
 * fewer and larger CTAs). 0 keeps the library's default (32). Results do not
 * depend on it (each cell's arithmetic is the same). Takes effect for later
 * calls and recordings; FWI_EINVAL for other values. The batched autotuner
 * picks it per workload. */
fwi_status fwi_set_tile_shape(fwi_ctx *ctx, int32_t forward_tile_rows);

/* Launch shape of the acoustic calls on ctx: the shots of a call are split
 * into forward_groups (forward and recompute steps) and adjoint_groups
 * (adjoint steps) contiguous groups, each step launched once per group on its
 * own stream, so that the groups' launches fill each other's idle SMs. 0 keeps
 * the library's default (4 and 2); at most 4; never more groups than shots.
 * Results do not depend on it (the per-shot arithmetic and the fixed-order
 * cross-shot sums are the same). Takes effect for later calls and recordings;
 * FWI_EINVAL outside [0, 4]. */
fwi_status fwi_set_shot_groups(fwi_ctx *ctx, int32_t forward_groups, int32_t adjoint_groups);

/* A recorded gradient: one acoustic fwi_misfit_grad call captured as a CUDA
 * graph, for loops that evaluate the same problem many times (an FWI iteration
 * per launch) or many small problems side by side, where launching the tens of
 * thousands of step kernels of a call one by one costs host time. The paper's
 * method is unchanged: each launch computes exactly what fwi_misfit_grad
 * computes (Eqs. adjoint-backward, adjoint-gradient) from the CURRENT contents
 * of the buffers named at recording time, so an inversion updates the model in
 * place and launches again.
 *
 * fwi_misfit_grad_graph: arguments as fwi_misfit_grad (no seis_out, no stream);
 *   every buffer must be device memory or page-locked host memory
 *   (cudaMallocHost / cudaHostRegister; FWI_EINVAL otherwise) and stays owned
 *   by the caller, who keeps it alive and at the same address while the graph
 *   exists. Host buffers are read and written by the graph's own copy nodes at
 *   every launch (inputs copied in at its start, results copied out at its
 *   end), as a direct call with host buffers does. Runs the call once on the context's own stream (its results are
 *   left in the outputs), then records it. FWI_ENOTIMPL for elastic models.
 *   The graph uses ctx's workspace: it is valid until a call on ctx needs a
 *   larger workspace or a different problem layout, after which
 *   fwi_graph_launch returns FWI_EINVAL. Use one context per recorded problem.
 * fwi_graph_launch: enqueue one evaluation on cuda_stream (asynchronous). Two
 *   launches of graphs of the SAME context must not overlap (they share the
 *   workspace); graphs of different contexts may run concurrently.
 * fwi_graph_status: wait for cuda_stream and decode the device status word of
 *   the last evaluation (the codes of fwi_misfit_grad). The recording keeps the
 *   call's phase marks as event-record nodes, so afterwards fwi_last_timing(ctx)
 *   reports that replay's phase and per-step kernel times and its launch count,
 *   as for a direct call.
 * fwi_graph_destroy: free the graph (not the context). */
typedef struct fwi_graph fwi_graph;
fwi_status fwi_misfit_grad_graph(fwi_ctx *ctx, const fwi_model *model, const fwi_sources *src,
                                 const fwi_receivers *rec, int32_t nt, float dt, const float *observed,
                                 int32_t ckpt_every, double *misfit, float *grad, float *grad_stf,
                                 float *grad_x0, fwi_graph **graph);
fwi_status fwi_graph_launch(fwi_graph *graph, void *cuda_stream);
fwi_status fwi_graph_status(fwi_graph *graph, void *cuda_stream);
fwi_status fwi_graph_destroy(fwi_graph *graph);

/* Batched gradients of many independent acoustic inversion instances of
 * uneven size (different grids, time lengths, shot and receiver counts): the
 * shot-parallel execution of the paper's Performance Benchmarking section,
 * carried across instances. Each instance's result is exactly what
 * fwi_misfit_grad(model_i, ..., nt_i, dt, observed_i, ckpt_every) computes
 * (J_i and dJ_i/dc_i, Eqs. adjoint-backward and adjoint-gradient), bit for bit.
 * Execution: every time step is ONE persistent launch whose CTAs walk a device
 * work table of (instance, shot, tile) items, each item carrying its
 * instance's grid and tensor maps; the whole sweep (inputs, preparation,
 * forward sweep with checkpoints, misfits, recompute and adjoint segments,
 * folds, outputs) is recorded once as a CUDA graph and replayed per launch.
 *
 * fwi_batch_create: n instances; models[i], srcs[i], recs[i], nt[i] as for
 *   fwi_misfit_grad (acoustic, divergence form, point or Gaussian sources);
 *   the instances share order, dx, dz and dt. observed[i] [S_i][nrec_i][nt_i],
 *   grads[i] [nz_i][nx_i] (dJ_i/dc_i), misfit [n] (J_i, double); every
 *   buffer is DEVICE memory owned by the caller, kept alive and in place while
 *   the batch exists, and read again at every launch (an FWI loop updates the
 *   models in place). ckpt_every (>= 1) is common to all instances; an
 *   instance with nt_i < ckpt_every keeps all its steps. Allocates one device
 *   workspace (the sum of the instances' fwi_workspace_bytes plus small
 *   tables) on `device`, runs the sweep once (its results are left in the
 *   outputs) and records it. FWI_EINVAL on a bad argument (the message names
 *   the instance), FWI_ENOTIMPL for other operators or source kinds,
 *   FWI_ENOMEM if the workspace does not fit.
 * fwi_batch_launch: enqueue one sweep on cuda_stream (asynchronous). Two
 *   launches of the same batch must not overlap.
 * fwi_batch_status: wait for cuda_stream and decode the instances' status
 *   words (the codes of fwi_misfit_grad); *instance (may be NULL) receives
 *   the first failing instance or -1.
 * fwi_batch_launches: kernels enqueued by one sweep.
 * fwi_batch_destroy: free the graph and the workspace. */
typedef struct fwi_batch fwi_batch;
fwi_status fwi_batch_create(int32_t device, int32_t n, const fwi_model *models,
                            const fwi_sources *srcs, const fwi_receivers *recs,
                            const int32_t *nt, float dt, const float *const *observed,
                            int32_t ckpt_every, double *misfit, float *const *grads,
                            fwi_batch **batch);
fwi_status fwi_batch_launch(fwi_batch *batch, void *cuda_stream);
fwi_status fwi_batch_status(fwi_batch *batch, void *cuda_stream, int32_t *instance);
int64_t fwi_batch_launches(const fwi_batch *batch);
fwi_status fwi_batch_destroy(fwi_batch *batch);

/* Forward modelling that allocates no device memory, for callers that cannot
 * let a library call cudaMalloc: applications that hand all device memory to
 * their own allocator and account for every byte, and latency-sensitive loops
 * that cannot afford the device-wide synchronisation cudaMalloc/cudaFree may
 * cause. The paper has no counterpart of this call; it computes exactly what
 * fwi_forward computes, with the same kernels.
 * Differences from fwi_forward: no context; vp, stf, x0, iz, ix and seis must
 * be DEVICE pointers on the current device; the working memory is one fixed
 * 32 MiB device array inside libfwi (held on every GPU where the library is
 * loaded, until the process exits), so a problem needing more is rejected with
 * FWI_EINVAL (the message gives the bytes needed). Every call shares that
 * array and clears the part it uses; calls that overlap on the GPU race and
 * must be serialised by the caller. The first call on a device resolves the
 * array's address: make it before any stream capture begins on that device
 * (a call made while capturing, with no earlier call on the device, gets
 * FWI_EINVAL). Calls outside capture resolve the address again, so a context
 * that was destroyed and created again is followed. Checked on the host before
 * any device work: the padded grid (each side <= 2^20 cells, at most 2^31
 * cells, else FWI_EINVAL "grid too large"), and that every pointer is device
 * memory of the current device or managed memory (else FWI_EINVAL). */
fwi_status fwi_forward_noalloc(const fwi_model *model, const fwi_sources *src,
                               const fwi_receivers *rec, int32_t nt, float dt, float *seis,
                               void *cuda_stream);

/* Timing of the last call, measured with CUDA events recorded on the call's
 * stream. phase_ms3: [0] forward sweep (with checkpoint saves), [1] reverse
 * sweep (recompute + adjoint + folds), [2] whole call. kernel_ms3: average
 * duration of one time step of [0] the recording forward step, [1] the storing
 * forward step of the recompute (with the checkpoint restores; per recomputed
 * step), [2] the adjoint step; 0 if none ran. Acoustic calls split the shots into up to 4
 * groups whose launches run concurrently on internal streams (forked from and
 * joined to the call's stream), so one step is one launch per group, and the
 * step time includes launch gaps. launches: number of kernels the call
 * launched. After fwi_graph_status, the values of the last graph replay on
 * ctx. Any pointer may be NULL. */
fwi_status fwi_last_timing(const fwi_ctx *ctx, float *phase_ms3, float *kernel_ms3,
                           int64_t *launches);

/* Elastic gradient in the velocity parametrisation: the chain rule through
 * lambda = rho (vp^2 - 2 vs^2) and mu = rho vs^2 (Implementation, elastic
 * wave equation) applied to the grad output of fwi_misfit_grad:
 *   dJ/dvp  = 2 rho vp dJ/dlambda
 *   dJ/dvs  = 2 rho vs (dJ/dmu - 2 dJ/dlambda)
 *   dJ/drho = (vp^2 - 2 vs^2) dJ/dlambda + vs^2 dJ/dmu + dJ/drho (lambda, mu fixed)
 * vp, vs, rho  [n] device arrays (the model of the fwi_misfit_grad call).
 * grad_lame    [3][n] device array (dJ/dlambda, dJ/dmu, dJ/drho).
 * grad_vel     [3][n] device array receiving (dJ/dvp, dJ/dvs, dJ/drho); may be grad_lame.
 * Asynchronous on cuda_stream; FWI_EINVAL on a NULL pointer or n < 0. */
fwi_status fwi_elastic_velocity_grad(const float *vp, const float *vs, const float *rho,
                                     const float *grad_lame, float *grad_vel, int64_t n,
                                     void *cuda_stream);

/* Self-test of the failure detection inside the step kernels. Every step
 * kernel waits for its tile copies on an mbarrier with a bound (2^24 polls or
 * 1 s, whichever comes first), after which it records a timeout that the call
 * returns as FWI_ETIMEOUT. This call runs that same wait, in one thread on the
 * context's device, on a barrier whose expected bytes no copy will deliver.
 * Returns FWI_ETIMEOUT when the wait gave up as designed (the expected result),
 * with the time it waited in *waited_ns (may be NULL); the device and the
 * context stay usable. Synchronous; allocates and frees 16 bytes. */
fwi_status fwi_selftest_wait_timeout(fwi_ctx *ctx, int64_t *waited_ns);

/* Message describing the last error of the calling thread ("" if none). */
const char *fwi_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
