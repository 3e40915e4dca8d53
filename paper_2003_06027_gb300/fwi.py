"""Thin Python binding of libfwi (include/fwi.h): argument marshalling only.

Every step of the computation runs in the library's CUDA kernels. PyTorch is
used for device memory and streams. Arrays may be CUDA tensors (device
pointers are passed as is), or CPU tensors / numpy arrays (host pointers; the
library copies them through its device workspace). There is no CPU fallback:
if the library cannot be loaded, the calls raise.
"""

from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

from . import build as _build

FWI_ACOUSTIC, FWI_ELASTIC = 0, 1
FWI_SRC_POINT, FWI_SRC_GAUSSIAN, FWI_SRC_MOMENT, FWI_SRC_LINE = 0, 1, 2, 3
FWI_OP_DIVERGENCE, FWI_OP_LAPLACIAN = 0, 1
STATUS = {0: "FWI_OK", 1: "FWI_EINVAL", 2: "FWI_ECFL", 3: "FWI_ENOMEM", 4: "FWI_ECUDA",
          5: "FWI_EUNSTABLE", 6: "FWI_ETIMEOUT", 7: "FWI_ENOTIMPL"}


class FwiError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _Model(ctypes.Structure):
    _fields_ = [("physics", ctypes.c_int32), ("nz", ctypes.c_int32), ("nx", ctypes.c_int32),
                ("dz", ctypes.c_float), ("dx", ctypes.c_float), ("order", ctypes.c_int32),
                ("npml", ctypes.c_int32), ("pml_R", ctypes.c_float), ("pml_vmax", ctypes.c_float),
                ("pml_f0", ctypes.c_float), ("vp", ctypes.c_void_p), ("vs", ctypes.c_void_p),
                ("rho", ctypes.c_void_p), ("op", ctypes.c_int32)]


class _Sources(ctypes.Structure):
    _fields_ = [("nshots", ctypes.c_int32), ("kind", ctypes.c_int32), ("x0", ctypes.c_void_p),
                ("stf", ctypes.c_void_p), ("mt", ctypes.c_void_p), ("line_len", ctypes.c_int32)]


class _Receivers(ctypes.Structure):
    _fields_ = [("nrec", ctypes.c_int32), ("iz", ctypes.c_void_p), ("ix", ctypes.c_void_p)]


_lib = None
_lib_lock = threading.Lock()
_ctx = threading.local()

EXPORTS = ["fwi_create", "fwi_destroy", "fwi_forward", "fwi_misfit_grad", "fwi_last_timing",
           "fwi_forward_noalloc", "fwi_elastic_velocity_grad", "fwi_selftest_wait_timeout",
           "fwi_misfit_grad_graph", "fwi_graph_launch", "fwi_graph_status", "fwi_graph_destroy",
           "fwi_set_shot_groups", "fwi_workspace_bytes", "fwi_choose_ckpt", "fwi_forward_vjp", "fwi_batch_create",
           "fwi_batch_launch", "fwi_batch_status", "fwi_batch_destroy", "fwi_set_tile_shape", "fwi_last_error"]


def library_path() -> str:
    return _build.LIB


def library(build_if_missing: bool = True):
    """Load libfwi.so (building it with nvcc if it is missing or stale)."""
    global _lib
    with _lib_lock:
        if _lib is None:
            path = _build.build() if build_if_missing else _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"libfwi.so not found at {path}; run __graft_entry__.build()")
            L = ctypes.CDLL(path)
            P = ctypes.c_void_p
            L.fwi_create.argtypes = [ctypes.POINTER(P), ctypes.c_int]
            L.fwi_destroy.argtypes = [P]
            L.fwi_forward.argtypes = [P, ctypes.POINTER(_Model), ctypes.POINTER(_Sources),
                                      ctypes.POINTER(_Receivers), ctypes.c_int32, ctypes.c_float, P, P]
            L.fwi_misfit_grad.argtypes = [P, ctypes.POINTER(_Model), ctypes.POINTER(_Sources),
                                          ctypes.POINTER(_Receivers), ctypes.c_int32, ctypes.c_float, P,
                                          ctypes.c_int32, P, P, P, P, P, P]
            L.fwi_forward_vjp.argtypes = L.fwi_misfit_grad.argtypes
            L.fwi_superposed_misfit_grad.argtypes = [P, ctypes.POINTER(_Model), ctypes.POINTER(_Sources),
                                                     ctypes.POINTER(_Receivers), ctypes.c_int32, ctypes.c_float, P,
                                                     ctypes.c_int32, P, P, P, P, P]
            L.fwi_batch_create.argtypes = [ctypes.c_int32, ctypes.c_int32, P, P, P, P, ctypes.c_float, P,
                                           ctypes.c_int32, P, P, ctypes.POINTER(P)]
            L.fwi_batch_launch.argtypes = [P, P]
            L.fwi_set_tile_shape.argtypes = [P, ctypes.c_int32]
            L.fwi_batch_status.argtypes = [P, P, ctypes.POINTER(ctypes.c_int32)]
            L.fwi_batch_launches.argtypes = [P]
            L.fwi_batch_launches.restype = ctypes.c_int64
            L.fwi_batch_destroy.argtypes = [P]
            L.fwi_last_timing.argtypes = [P, P, P, P]
            L.fwi_forward_noalloc.argtypes = [ctypes.POINTER(_Model), ctypes.POINTER(_Sources),
                                              ctypes.POINTER(_Receivers), ctypes.c_int32, ctypes.c_float, P,
                                              P]
            L.fwi_elastic_velocity_grad.argtypes = [P, P, P, P, P, ctypes.c_int64, P]
            L.fwi_selftest_wait_timeout.argtypes = [P, P]
            L.fwi_misfit_grad_graph.argtypes = [P, ctypes.POINTER(_Model), ctypes.POINTER(_Sources),
                                                ctypes.POINTER(_Receivers), ctypes.c_int32, ctypes.c_float, P,
                                                ctypes.c_int32, P, P, P, P, ctypes.POINTER(P)]
            L.fwi_graph_launch.argtypes = [P, P]
            L.fwi_graph_status.argtypes = [P, P]
            L.fwi_graph_destroy.argtypes = [P]
            L.fwi_set_shot_groups.argtypes = [P, ctypes.c_int32, ctypes.c_int32]
            L.fwi_workspace_bytes.argtypes = [ctypes.POINTER(_Model), ctypes.POINTER(_Sources),
                                              ctypes.POINTER(_Receivers), ctypes.c_int32, ctypes.c_int32,
                                              ctypes.POINTER(ctypes.c_uint64)]
            L.fwi_choose_ckpt.argtypes = [P, ctypes.POINTER(_Model), ctypes.POINTER(_Sources),
                                          ctypes.POINTER(_Receivers), ctypes.c_int32, ctypes.c_uint64,
                                          ctypes.POINTER(ctypes.c_int32)]
            L.fwi_last_error.restype = ctypes.c_char_p
            for f in EXPORTS[:-1]:
                getattr(L, f).restype = ctypes.c_int
            _lib = L
    return _lib


def _check(st: int):
    if st != 0:
        raise FwiError(st, library().fwi_last_error().decode())


def context(device: int = 0):
    """Per-thread, per-device library context."""
    ctxs = getattr(_ctx, "ctxs", None)
    if ctxs is None:
        ctxs = _ctx.ctxs = {}
    if device not in ctxs:
        h = ctypes.c_void_p()
        _check(library().fwi_create(ctypes.byref(h), int(device)))
        ctxs[device] = h
    return ctxs[device]


def release_context(device: int | None = None):
    """Destroy the calling thread's library context(s), freeing their device
    arenas (a thread that ends without this keeps its arena until exit)."""
    ctxs = getattr(_ctx, "ctxs", None) or {}
    for dev in list(ctxs):
        if device is None or dev == device:
            _check(library().fwi_destroy(ctxs.pop(dev)))


@dataclass
class Timing:
    forward_ms: float      # forward sweep (with checkpoint saves)
    reverse_ms: float      # recompute + adjoint + folds
    total_ms: float
    fwd_step_ms: float     # average launch of the recording forward step
    store_step_ms: float   # average launch of the storing forward step (recompute)
    adj_step_ms: float     # average launch of the adjoint step
    launches: int          # kernels launched by the call


def set_shot_groups(forward_groups: int = 0, adjoint_groups: int = 0, device: int = 0):
    """Launch shape of this thread's context for acoustic calls: shot groups of
    the forward/recompute steps and of the adjoint steps (0: the library's
    default; fwi_set_shot_groups)."""
    _check(library().fwi_set_shot_groups(context(device), int(forward_groups), int(adjoint_groups)))


def set_tile_shape(forward_tile_rows: int = 0, device: int = 0):
    """Tile height (32 or 64 rows; 0: the default) of the acoustic forward steps
    of this thread's context (fwi_set_tile_shape)."""
    _check(library().fwi_set_tile_shape(context(device), int(forward_tile_rows)))


def last_timing(device: int = 0) -> Timing:
    ph = (ctypes.c_float * 3)()
    km = (ctypes.c_float * 3)()
    n = ctypes.c_int64()
    _check(library().fwi_last_timing(context(device), ph, km, ctypes.byref(n)))
    return Timing(ph[0], ph[1], ph[2], km[0], km[1], km[2], int(n.value))


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _arr(x, dtype):
    """Contiguous array of the given numpy dtype; torch tensors stay torch."""
    if _is_torch(x):
        import torch

        tdt = {np.float32: torch.float32, np.int32: torch.int32}[dtype]
        return x.detach().to(tdt).contiguous()
    return np.ascontiguousarray(x, dtype=dtype)


def _ptr(x):
    if x is None:
        return None
    if _is_torch(x):
        return ctypes.c_void_p(x.data_ptr())
    return ctypes.c_void_p(x.ctypes.data)


def _empty_like_place(ref, shape, dtype=np.float32):
    if _is_torch(ref):
        import torch

        tdt = {np.float32: torch.float32, np.float64: torch.float64}[dtype]
        return torch.empty(shape, dtype=tdt, device=ref.device)
    return np.empty(shape, dtype=dtype)


def _stream(ref, stream):
    if stream is not None:
        return ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))
    if _is_torch(ref) and ref.is_cuda:
        import torch

        return ctypes.c_void_p(torch.cuda.current_stream(ref.device).cuda_stream)
    return ctypes.c_void_p(0)


def _device(ref, device):
    if device is not None:
        return int(device)
    if _is_torch(ref) and ref.is_cuda:
        return ref.device.index or 0
    return 0


class _Call:
    """Holds the marshalled arguments (and keeps their buffers alive)."""

    def __init__(self, c, stf, x0, rec_iz, rec_ix, dx, dz, order, npml, pml_R, pml_vmax, pml_f0,
                 src_kind, op=FWI_OP_DIVERGENCE):
        self.c = _arr(c, np.float32)
        self.stf = _arr(stf, np.float32)
        # a line source (plane wave) has one time function per cell: stf [S][nt][line_len]
        self.line_len = 0
        if src_kind == FWI_SRC_LINE:
            if self.stf.ndim == 2:
                self.stf = self.stf.reshape(1, *self.stf.shape)
            self.line_len = int(self.stf.shape[2])
        elif self.stf.ndim == 1:
            self.stf = self.stf.reshape(1, -1)
        self.x0 = _arr(x0, np.float32).reshape(-1, 2)
        self.iz = _arr(rec_iz, np.int32).reshape(-1)
        self.ix = _arr(rec_ix, np.int32).reshape(-1)
        nz, nx = self.c.shape
        self.S, self.nt = self.stf.shape[:2]
        self.nrec = self.iz.shape[0]
        self.model = _Model(FWI_ACOUSTIC, nz, nx, dz, dx, order, npml, pml_R, pml_vmax, pml_f0,
                            _ptr(self.c), None, None, int(op))
        self.src = _Sources(self.S, src_kind, _ptr(self.x0), _ptr(self.stf), None, self.line_len)
        self.rec = _Receivers(self.nrec, _ptr(self.iz), _ptr(self.ix))


def forward(c, stf, x0, rec_iz, rec_ix, *, dx, dz, dt, order=4, npml=20, pml_R=1e-3,
            pml_vmax=4500.0, pml_f0=10.0, src_kind=FWI_SRC_POINT, op=FWI_OP_DIVERGENCE, out=None, stream=None,
            device=None):
    """Seismograms [nshots][nrec][nt] (fwi_forward). nt = stf.shape[-1]."""
    a = _Call(c, stf, x0, rec_iz, rec_ix, dx, dz, order, npml, pml_R, pml_vmax, pml_f0, src_kind, op)
    if out is None:
        out = _empty_like_place(a.c, (a.S, a.nrec, a.nt))
    dev = _device(a.c, device)
    _check(library().fwi_forward(context(dev), ctypes.byref(a.model), ctypes.byref(a.src),
                                 ctypes.byref(a.rec), a.nt, float(dt), _ptr(out), _stream(a.c, stream)))
    return out


def forward_noalloc(c, stf, x0, rec_iz, rec_ix, *, dx, dz, dt, order=4, npml=20, pml_R=1e-3,
                    pml_vmax=4500.0, pml_f0=10.0, src_kind=FWI_SRC_POINT, op=FWI_OP_DIVERGENCE, out=None, stream=None):
    """fwi_forward_noalloc: the forward map without any device allocation by
    the library (for callers whose device memory is fully managed by their own
    allocator). All arrays must be CUDA tensors on the current device; ``out``
    (the seismograms) is allocated here by torch when not given."""
    a = _Call(c, stf, x0, rec_iz, rec_ix, dx, dz, order, npml, pml_R, pml_vmax, pml_f0, src_kind, op)
    if out is None:
        out = _empty_like_place(a.c, (a.S, a.nrec, a.nt))
    _check(library().fwi_forward_noalloc(ctypes.byref(a.model), ctypes.byref(a.src), ctypes.byref(a.rec),
                                         a.nt, float(dt), _ptr(out), _stream(a.c, stream)))
    return out


def misfit_grad(c, stf, x0, rec_iz, rec_ix, observed, *, dx, dz, dt, order=4, npml=20,
                pml_R=1e-3, pml_vmax=4500.0, pml_f0=10.0, src_kind=FWI_SRC_POINT, op=FWI_OP_DIVERGENCE, ckpt_every=100,
                want_grad=True, want_src=True, want_seis=False, out=None, stream=None, device=None, _vjp=False):
    """(J, dJ/dc, dJ/dstf, dJ/dx0, seis) of J = 1/2 sum (d - d_obs)^2 (fwi_misfit_grad).

    ``out`` may hold preallocated outputs {"misfit", "grad", "grad_stf", "grad_x0", "seis"}.
    With ``src_kind=FWI_SRC_LINE`` (plane-wave sources) stf and dJ/dstf are
    [S][nt][line_len] and dJ/dx0 is None.
    """
    a = _Call(c, stf, x0, rec_iz, rec_ix, dx, dz, order, npml, pml_R, pml_vmax, pml_f0, src_kind, op)
    obs = _arr(observed, np.float32)
    out = dict(out or {})
    ref = a.c
    if "misfit" not in out:
        out["misfit"] = _empty_like_place(ref, (1,), np.float64)
    if want_grad and "grad" not in out:
        out["grad"] = _empty_like_place(ref, tuple(a.c.shape))
    line = src_kind == FWI_SRC_LINE
    if want_src and "grad_stf" not in out:
        out["grad_stf"] = _empty_like_place(ref, (a.S, a.nt, a.line_len) if line else (a.S, a.nt))
    if want_src and not line and "grad_x0" not in out:  # a line source has no position gradient
        out["grad_x0"] = _empty_like_place(ref, (a.S, 2))
    if want_seis and "seis" not in out:
        out["seis"] = _empty_like_place(ref, (a.S, a.nrec, a.nt))
    dev = _device(ref, device)
    K = max(1, min(int(ckpt_every), a.nt))
    fn = library().fwi_forward_vjp if _vjp else library().fwi_misfit_grad
    _check(fn(
        context(dev), ctypes.byref(a.model), ctypes.byref(a.src), ctypes.byref(a.rec), a.nt,
        float(dt), _ptr(obs), K, _ptr(out["misfit"]), _ptr(out.get("grad")),
        _ptr(out.get("grad_stf")), _ptr(out.get("grad_x0")), _ptr(out.get("seis")),
        _stream(ref, stream)))
    return out["misfit"], out.get("grad"), out.get("grad_stf"), out.get("grad_x0"), out.get("seis")


def superposed_misfit_grad(c, stf, x0, rec_iz, rec_ix, observed, *, dx, dz, dt, order=4, npml=20, pml_R=1e-3,
                           pml_vmax=4500.0, pml_f0=10.0, src_kind=FWI_SRC_GAUSSIAN, op=FWI_OP_DIVERGENCE,
                           ckpt_every=100, want_grad=True, want_src=True, stream=None, device=None):
    """(J, dJ/dc, dJ/dstf, dJ/dx0) of J = 1/2 sum (sum_s d_s - d_obs)^2 for the
    sub-sources stf [k][nt] at x0 [k][2] of one event, observed [nrec][nt]
    (fwi_superposed_misfit_grad)."""
    a = _Call(c, stf, x0, rec_iz, rec_ix, dx, dz, order, npml, pml_R, pml_vmax, pml_f0, src_kind, op)
    obs = _arr(observed, np.float32)
    ref = a.c
    J = _empty_like_place(ref, (1,), np.float64)
    gc = _empty_like_place(ref, tuple(a.c.shape)) if want_grad else None
    gs = _empty_like_place(ref, (a.S, a.nt)) if want_src else None
    gx = _empty_like_place(ref, (a.S, 2)) if want_src else None
    K = max(1, min(int(ckpt_every), a.nt))
    _check(library().fwi_superposed_misfit_grad(
        context(_device(ref, device)), ctypes.byref(a.model), ctypes.byref(a.src), ctypes.byref(a.rec), a.nt,
        float(dt), _ptr(obs), K, _ptr(J), _ptr(gc), _ptr(gs), _ptr(gx), _stream(ref, stream)))
    return J, gc, gs, gx


def forward_vjp(c, stf, x0, rec_iz, rec_ix, cotangent, **kw):
    """(<d, v>, (dd/dc)^T v, (dd/dstf)^T v, (dd/dx0)^T v, seis) for the
    seismograms d = forward(c, stf, x0, ...) and a cotangent v shaped like d
    (fwi_forward_vjp: the adjoint sweep seeded with v). Keywords as misfit_grad."""
    return misfit_grad(c, stf, x0, rec_iz, rec_ix, cotangent, _vjp=True, **kw)


class GradGraph:
    """One acoustic misfit/gradient evaluation recorded as a CUDA graph
    (fwi_misfit_grad_graph) on a library context of its own.

    The arguments are either all CUDA tensors or all page-locked (pinned) host
    tensors of the call's own dtypes (float32; int32 receiver indices) on the
    CUDA device ``device`` (default: the current one). They are kept referenced
    and are read again at every launch, so an inversion updates ``c`` in place
    and launches again; with host tensors the graph's copy nodes move the inputs
    in and the results out at every launch. Outputs live in ``self.misfit``,
    ``self.grad`` (and ``grad_stf``, ``grad_x0`` when ``want_src``), in the
    inputs' memory kind. ``groups`` = (forward, adjoint) shot groups of the
    recorded launches (0: default). Recording runs the evaluation once."""

    def __init__(self, c, stf, x0, rec_iz, rec_ix, observed, *, dx, dz, dt, order=4, npml=20, pml_R=1e-3,
                 pml_vmax=4500.0, pml_f0=10.0, src_kind=FWI_SRC_POINT, op=FWI_OP_DIVERGENCE, ckpt_every=100,
                 want_src=False,
                 groups=(0, 0), tile_rows=0, device=None):
        import torch

        ts = (c, stf, x0, rec_iz, rec_ix, observed)
        if not all(_is_torch(t) for t in ts):
            raise ValueError("GradGraph takes torch tensors")
        host = not c.is_cuda
        if host:
            # a converted copy would not see the caller's in-place updates: the
            # host tensors must already be pinned, contiguous and of the call's dtypes
            want = (torch.float32, torch.float32, torch.float32, torch.int32, torch.int32, torch.float32)
            for t, dt_ in zip(ts, want):
                if t.is_cuda or not t.is_pinned() or t.dtype != dt_ or not t.is_contiguous():
                    raise ValueError("GradGraph host inputs must all be pinned, contiguous, float32 "
                                     "(int32 receiver indices)")
        elif not all(t.is_cuda for t in ts):
            raise ValueError("GradGraph takes CUDA tensors, or pinned host tensors, not a mix")
        self._a = _Call(c, stf, x0, rec_iz, rec_ix, dx, dz, order, npml, pml_R, pml_vmax, pml_f0, src_kind, op)
        a = self._a
        self._obs = _arr(observed, np.float32)
        if host:
            self.device = torch.cuda.current_device() if device is None else int(device)
            place = lambda shape, dtype=torch.float32: torch.empty(shape, dtype=dtype).pin_memory()
            self.misfit = place((1,), torch.float64)
            self.grad = place(tuple(a.c.shape))
            self.grad_stf = place((a.S, a.nt)) if want_src else None
            self.grad_x0 = place((a.S, 2)) if want_src else None
        else:
            self.device = a.c.device.index
            self.misfit = _empty_like_place(a.c, (1,), np.float64)
            self.grad = _empty_like_place(a.c, tuple(a.c.shape))
            self.grad_stf = _empty_like_place(a.c, (a.S, a.nt)) if want_src else None
            self.grad_x0 = _empty_like_place(a.c, (a.S, 2)) if want_src else None
        L = library()
        self._L = L
        self.ctx = ctypes.c_void_p()
        _check(L.fwi_create(ctypes.byref(self.ctx), int(self.device)))
        self.groups = tuple(groups)
        st = L.fwi_set_shot_groups(self.ctx, int(groups[0]), int(groups[1]))
        if st == 0:
            st = L.fwi_set_tile_shape(self.ctx, int(tile_rows))
        if st != 0:
            L.fwi_destroy(self.ctx)
            self.ctx = None
            _check(st)
        self.graph = ctypes.c_void_p()
        K = max(1, min(int(ckpt_every), a.nt))
        st = L.fwi_misfit_grad_graph(self.ctx, ctypes.byref(a.model), ctypes.byref(a.src), ctypes.byref(a.rec), a.nt,
                                     float(dt), _ptr(self._obs), K, _ptr(self.misfit), _ptr(self.grad),
                                     _ptr(self.grad_stf), _ptr(self.grad_x0), ctypes.byref(self.graph))
        if st != 0:
            L.fwi_destroy(self.ctx)
            self.ctx = None
            _check(st)

    def launch(self, stream=None):
        """Enqueue one evaluation on ``stream`` (default: the current stream)."""
        _check(self._L.fwi_graph_launch(self.graph, _stream(self._a.c, stream)))

    def check(self, stream=None):
        """Wait for ``stream`` and raise if the last evaluation reported an error."""
        _check(self._L.fwi_graph_status(self.graph, _stream(self._a.c, stream)))

    def timing(self) -> Timing:
        """Phase and per-step kernel times of the replay that the last ``check``
        waited for (the recording keeps the library's phase marks)."""
        ph = (ctypes.c_float * 3)()
        km = (ctypes.c_float * 3)()
        n = ctypes.c_int64()
        _check(self._L.fwi_last_timing(self.ctx, ph, km, ctypes.byref(n)))
        return Timing(ph[0], ph[1], ph[2], km[0], km[1], km[2], int(n.value))

    def close(self):
        if getattr(self, "graph", None):
            self._L.fwi_graph_destroy(self.graph)
            self.graph = None
        if getattr(self, "ctx", None):
            self._L.fwi_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """fwi_batch_*: J_i and dJ_i/dc_i of several acoustic instances of uneven
    size in one recorded sweep, each time step one persistent launch over the
    tiles of all instances (shared order, dx, dz, dt).

    ``instances``: sequence of (c, stf, x0, rec_iz, rec_ix, observed, kw) with
    CUDA tensors (kept referenced, read again at every launch: update ``c`` in
    place and launch again) and kw the geometry keywords of misfit_grad.
    Results: ``self.misfit`` [n] float64, ``self.grads`` (one [nz][nx] tensor
    per instance). Creation runs the sweep once and records it."""

    def __init__(self, instances, *, ckpt_every=100, device=None):
        import torch

        if not instances:
            raise ValueError("a batch needs at least one instance")
        self._calls, self._obs = [], []
        dts = set()
        for c, stf, x0, iz, ix, obs, kw in instances:
            for t in (c, stf, x0, iz, ix, obs):
                if not (_is_torch(t) and t.is_cuda):
                    raise ValueError("Batch takes CUDA tensors only")
            a = _Call(c, stf, x0, iz, ix, kw["dx"], kw["dz"], kw.get("order", 4), kw.get("npml", 20),
                      kw.get("pml_R", 1e-3), kw.get("pml_vmax", 4500.0), kw.get("pml_f0", 10.0),
                      kw.get("src_kind", FWI_SRC_POINT), kw.get("op", FWI_OP_DIVERGENCE))
            self._calls.append(a)
            self._obs.append(_arr(obs, np.float32))
            dts.add(float(kw["dt"]))
        if len(dts) != 1:
            raise ValueError("the instances of a batch share dt")
        n = len(self._calls)
        ref = self._calls[0].c
        self.device = _device(ref, device)
        self.misfit = torch.zeros(n, dtype=torch.float64, device=ref.device)
        self.grads = [torch.empty_like(a.c) for a in self._calls]
        M = (_Model * n)(*[a.model for a in self._calls])
        S = (_Sources * n)(*[a.src for a in self._calls])
        R = (_Receivers * n)(*[a.rec for a in self._calls])
        nts = (ctypes.c_int32 * n)(*[a.nt for a in self._calls])
        obs = (ctypes.c_void_p * n)(*[o.data_ptr() for o in self._obs])
        grads = (ctypes.c_void_p * n)(*[g.data_ptr() for g in self.grads])
        self._keep = (M, S, R, nts, obs, grads)
        self._L = library()
        self.handle = ctypes.c_void_p()
        _check(self._L.fwi_batch_create(self.device, n, M, S, R, nts, dts.pop(), obs, int(ckpt_every),
                                        ctypes.c_void_p(self.misfit.data_ptr()), grads, ctypes.byref(self.handle)))
        self.launches = int(self._L.fwi_batch_launches(self.handle))

    def launch(self, stream=None):
        """Enqueue one sweep on ``stream`` (default: the current stream)."""
        _check(self._L.fwi_batch_launch(self.handle, _stream(self._calls[0].c, stream)))

    def check(self, stream=None):
        """Wait for ``stream`` and raise if an instance reported an error."""
        bad = ctypes.c_int32(-1)
        _check(self._L.fwi_batch_status(self.handle, _stream(self._calls[0].c, stream), ctypes.byref(bad)))

    def close(self):
        if getattr(self, "handle", None):
            self._L.fwi_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _ECall:
    """Marshalled arguments of an elastic call."""

    def __init__(self, vp, vs, rho, stf, x0, mt, rec_iz, rec_ix, dx, dz, order, npml, pml_R, pml_vmax,
                 pml_f0, src_kind):
        self.vp, self.vs, self.rho = (_arr(a, np.float32) for a in (vp, vs, rho))
        self.stf = _arr(stf, np.float32)
        if self.stf.ndim == 1:
            self.stf = self.stf.reshape(1, -1)
        self.x0 = _arr(x0, np.float32).reshape(-1, 2)
        self.mt = _arr(mt, np.float32).reshape(-1, 3)
        self.iz = _arr(rec_iz, np.int32).reshape(-1)
        self.ix = _arr(rec_ix, np.int32).reshape(-1)
        nz, nx = self.vp.shape
        self.S, self.nt = self.stf.shape
        self.nrec = self.iz.shape[0]
        self.model = _Model(FWI_ELASTIC, nz, nx, dz, dx, order, npml, pml_R, pml_vmax, pml_f0,
                            _ptr(self.vp), _ptr(self.vs), _ptr(self.rho))
        self.src = _Sources(self.S, src_kind, _ptr(self.x0), _ptr(self.stf), _ptr(self.mt))
        self.rec = _Receivers(self.nrec, _ptr(self.iz), _ptr(self.ix))


def _workspace(a, ckpt_every):
    b = ctypes.c_uint64()
    _check(library().fwi_workspace_bytes(ctypes.byref(a.model), ctypes.byref(a.src), ctypes.byref(a.rec), a.nt,
                                         int(ckpt_every), ctypes.byref(b)))
    return int(b.value)


def _choose(a, budget_bytes, device):
    k = ctypes.c_int32()
    ctx = context(device) if not budget_bytes else None  # 0: the device's free memory
    _check(library().fwi_choose_ckpt(ctx, ctypes.byref(a.model), ctypes.byref(a.src), ctypes.byref(a.rec), a.nt,
                                     int(budget_bytes), ctypes.byref(k)))
    return int(k.value)


def workspace_bytes(c, stf, x0, rec_iz, rec_ix, *, ckpt_every=0, dx, dz, dt=None, order=4, npml=20, pml_R=1e-3,
                    pml_vmax=4500.0, pml_f0=10.0, src_kind=FWI_SRC_POINT, op=FWI_OP_DIVERGENCE):
    """Device workspace in bytes of the acoustic forward call (ckpt_every=0)
    or of misfit_grad with that checkpoint interval (fwi_workspace_bytes).
    Host arithmetic only; the arrays may live anywhere."""
    a = _Call(c, stf, x0, rec_iz, rec_ix, dx, dz, order, npml, pml_R, pml_vmax, pml_f0, src_kind, op)
    return _workspace(a, ckpt_every)


def choose_ckpt(c, stf, x0, rec_iz, rec_ix, *, budget_bytes=0, device=0, dx, dz, dt=None, order=4, npml=20,
                pml_R=1e-3, pml_vmax=4500.0, pml_f0=10.0, src_kind=FWI_SRC_POINT, op=FWI_OP_DIVERGENCE):
    """Checkpoint interval of an acoustic misfit_grad that fits budget_bytes of
    device memory with the fewest recomputed steps (fwi_choose_ckpt);
    budget_bytes=0: the free memory of ``device``."""
    a = _Call(c, stf, x0, rec_iz, rec_ix, dx, dz, order, npml, pml_R, pml_vmax, pml_f0, src_kind, op)
    return _choose(a, budget_bytes, device)


def workspace_bytes_elastic(vp, vs, rho, stf, x0, mt, rec_iz, rec_ix, *, ckpt_every=0, dx, dz, dt=None, order=4,
                            npml=20, pml_R=1e-3, pml_vmax=4500.0, pml_f0=10.0, src_kind=FWI_SRC_GAUSSIAN):
    """workspace_bytes for the elastic calls."""
    a = _ECall(vp, vs, rho, stf, x0, mt, rec_iz, rec_ix, dx, dz, order, npml, pml_R, pml_vmax, pml_f0, src_kind)
    return _workspace(a, ckpt_every)


def choose_ckpt_elastic(vp, vs, rho, stf, x0, mt, rec_iz, rec_ix, *, budget_bytes=0, device=0, dx, dz, dt=None,
                        order=4, npml=20, pml_R=1e-3, pml_vmax=4500.0, pml_f0=10.0, src_kind=FWI_SRC_GAUSSIAN):
    """choose_ckpt for the elastic gradient."""
    a = _ECall(vp, vs, rho, stf, x0, mt, rec_iz, rec_ix, dx, dz, order, npml, pml_R, pml_vmax, pml_f0, src_kind)
    return _choose(a, budget_bytes, device)


def forward_elastic(vp, vs, rho, stf, x0, mt, rec_iz, rec_ix, *, dx, dz, dt, order=4, npml=20,
                    pml_R=1e-3, pml_vmax=4500.0, pml_f0=10.0, src_kind=FWI_SRC_GAUSSIAN, out=None,
                    stream=None, device=None):
    """Elastic seismograms [nshots][2][nrec][nt] (vx, vz) (fwi_forward, FWI_ELASTIC)."""
    a = _ECall(vp, vs, rho, stf, x0, mt, rec_iz, rec_ix, dx, dz, order, npml, pml_R, pml_vmax, pml_f0,
               src_kind)
    if out is None:
        out = _empty_like_place(a.vp, (a.S, 2, a.nrec, a.nt))
    dev = _device(a.vp, device)
    _check(library().fwi_forward(context(dev), ctypes.byref(a.model), ctypes.byref(a.src),
                                 ctypes.byref(a.rec), a.nt, float(dt), _ptr(out), _stream(a.vp, stream)))
    return out


def misfit_grad_elastic(vp, vs, rho, stf, x0, mt, rec_iz, rec_ix, observed, *, dx, dz, dt, order=4,
                        npml=20, pml_R=1e-3, pml_vmax=4500.0, pml_f0=10.0, src_kind=FWI_SRC_GAUSSIAN,
                        ckpt_every=100, want_grad=True, want_src=True, want_seis=False, out=None, stream=None,
                        device=None, _vjp=False):
    """(J, [dJ/dlambda, dJ/dmu, dJ/drho] [3][nz][nx], dJ/dstf, dJ/dx0, seis) (fwi_misfit_grad, FWI_ELASTIC).
    With want_grad=False no model gradient is formed (its entry is None)."""
    a = _ECall(vp, vs, rho, stf, x0, mt, rec_iz, rec_ix, dx, dz, order, npml, pml_R, pml_vmax, pml_f0,
               src_kind)
    obs = _arr(observed, np.float32)
    out = dict(out or {})
    ref = a.vp
    nz, nx = a.vp.shape
    out.setdefault("misfit", _empty_like_place(ref, (1,), np.float64))
    if want_grad:
        out.setdefault("grad", _empty_like_place(ref, (3, nz, nx)))
    if want_src:
        out.setdefault("grad_stf", _empty_like_place(ref, (a.S, a.nt)))
        out.setdefault("grad_x0", _empty_like_place(ref, (a.S, 2)))
    if want_seis:
        out.setdefault("seis", _empty_like_place(ref, (a.S, 2, a.nrec, a.nt)))
    dev = _device(ref, device)
    K = max(1, min(int(ckpt_every), a.nt))
    fn = library().fwi_forward_vjp if _vjp else library().fwi_misfit_grad
    _check(fn(
        context(dev), ctypes.byref(a.model), ctypes.byref(a.src), ctypes.byref(a.rec), a.nt,
        float(dt), _ptr(obs), K, _ptr(out["misfit"]), _ptr(out.get("grad")), _ptr(out.get("grad_stf")),
        _ptr(out.get("grad_x0")), _ptr(out.get("seis")), _stream(ref, stream)))
    return out["misfit"], out.get("grad"), out.get("grad_stf"), out.get("grad_x0"), out.get("seis")


def forward_vjp_elastic(vp, vs, rho, stf, x0, mt, rec_iz, rec_ix, cotangent, **kw):
    """(<d, v>, (dd/d(lambda, mu, rho))^T v [3][nz][nx], (dd/dstf)^T v, (dd/dx0)^T v, seis)
    for the elastic seismograms d [S][2][nrec][nt] and a cotangent v shaped
    like d (fwi_forward_vjp). Keywords as misfit_grad_elastic."""
    return misfit_grad_elastic(vp, vs, rho, stf, x0, mt, rec_iz, rec_ix, cotangent, _vjp=True, **kw)


def elastic_velocity_grad(vp, vs, rho, grad_lame, out=None, stream=None):
    """(dJ/dvp, dJ/dvs, dJ/drho) [3][nz][nx] from the (dJ/dlambda, dJ/dmu, dJ/drho)
    output of misfit_grad_elastic (fwi_elastic_velocity_grad). CUDA tensors on
    one device; ``out`` may be ``grad_lame`` itself."""
    vp, vs, rho = (_arr(a, np.float32) for a in (vp, vs, rho))
    gl = _arr(grad_lame, np.float32)
    if not (_is_torch(vp) and vp.is_cuda):
        raise ValueError("elastic_velocity_grad takes CUDA tensors")
    n = vp.numel()
    if gl.numel() != 3 * n or vs.numel() != n or rho.numel() != n:
        raise ValueError("grad_lame must hold 3 fields shaped like vp")
    if out is None:
        out = _empty_like_place(vp, (3,) + tuple(vp.shape))
    _check(library().fwi_elastic_velocity_grad(_ptr(vp), _ptr(vs), _ptr(rho), _ptr(gl), _ptr(out), n,
                                               _stream(vp, stream)))
    return out


def selftest_wait_timeout(device: int = 0):
    """(status, waited_ns) of fwi_selftest_wait_timeout: FWI_ETIMEOUT is the
    expected status (the bounded device wait gave up as designed)."""
    ns = ctypes.c_int64()
    st = library().fwi_selftest_wait_timeout(context(device), ctypes.byref(ns))
    return int(st), int(ns.value)


def problem_kwargs(d: dict) -> dict:
    """Keyword arguments of forward()/misfit_grad() from a synth problem dict."""
    kw = dict(dx=d["dx"], dz=d["dz"], dt=d["dt"], order=d["order"], npml=d["npml"],
              pml_R=d["pml_R"], pml_vmax=d["pml_vmax"], pml_f0=d["pml_f0"], src_kind=d["src_kind"])
    if d.get("op", 0):
        kw["op"] = d["op"]
    return kw
