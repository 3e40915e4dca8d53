"""Plain FP64 CPU oracle of the seismic-inversion hot path.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers. The product library never
imports this package, and the two share no code.

The numerical work is in ``acoustic.c`` / ``elastic.c`` (plain scalar C loops in
FP64); this module compiles them with gcc on first use and marshals numpy
arrays through ctypes.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SOURCES = ["acoustic.c", "elastic.c"]
_HEADERS = ["oracle.h", "acoustic_fwd_body.h", "elastic_body.h"]
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    srcs = [os.path.join(_HERE, s) for s in _SOURCES if os.path.exists(os.path.join(_HERE, s))]
    deps = srcs + [os.path.join(_HERE, h) for h in _HEADERS if os.path.exists(os.path.join(_HERE, h))]
    if not force and os.path.exists(_LIB_PATH):
        t = os.path.getmtime(_LIB_PATH)
        if all(os.path.getmtime(d) <= t for d in deps):
            return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-std=gnu11", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
    return _lib


class AcousticCfg(ctypes.Structure):
    _fields_ = [
        ("nz", ctypes.c_int), ("nx", ctypes.c_int), ("npml", ctypes.c_int),
        ("order", ctypes.c_int), ("nt", ctypes.c_int), ("nshots", ctypes.c_int),
        ("src_kind", ctypes.c_int), ("nrec", ctypes.c_int),
        ("dz", ctypes.c_double), ("dx", ctypes.c_double), ("dt", ctypes.c_double),
        ("pml_R", ctypes.c_double), ("pml_vmax", ctypes.c_double), ("pml_f0", ctypes.c_double),
        ("rec_iz", ctypes.POINTER(ctypes.c_int)), ("rec_ix", ctypes.POINTER(ctypes.c_int)),
        ("line_len", ctypes.c_int), ("op", ctypes.c_int),
    ]


def _declare(L):
    P = ctypes.c_void_p
    L.or_fd_coeffs.argtypes = [ctypes.c_int, P]
    L.or_fd_coeffs.restype = ctypes.c_int
    L.or_cpml_profile.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_int, ctypes.c_int, P, P]
    L.or_cpml_profile.restype = None
    for name in ("or_acoustic_forward", "or_acoustic_forward_cplx"):
        f = getattr(L, name)
        f.argtypes = [ctypes.POINTER(AcousticCfg), P, P, P, P]
        f.restype = ctypes.c_int
    L.or_acoustic_adjoint.argtypes = [ctypes.POINTER(AcousticCfg), P, P, P, P, P, P, P]
    L.or_acoustic_adjoint.restype = ctypes.c_int
    L.or_num_threads.argtypes = []
    L.or_num_threads.restype = ctypes.c_int
    for name in ("or_elastic_forward", "or_elastic_forward_cplx"):
        f = getattr(L, name)
        f.argtypes = [ctypes.POINTER(AcousticCfg), P, P, P, P, P, P, P]
        f.restype = ctypes.c_int
    L.or_elastic_snapshot.argtypes = [ctypes.POINTER(AcousticCfg), P, P, P, P, P, P, ctypes.c_int, P]
    L.or_elastic_snapshot.restype = ctypes.c_int
    L.or_elastic_adjoint.argtypes = [ctypes.POINTER(AcousticCfg)] + [P] * 12
    L.or_elastic_adjoint.restype = ctypes.c_int


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def num_threads() -> int:
    return int(lib().or_num_threads())


def fd_coeffs(order: int) -> np.ndarray:
    a = np.zeros(4, dtype=np.float64)
    if lib().or_fd_coeffs(int(order), _ptr(a)) != 0:
        raise ValueError(f"unsupported order {order}")
    return a[: order // 2].copy()


def cpml_profile(n_phys, npml, h, dt, R, vmax, f0, half, n_out):
    a = np.zeros(n_out, dtype=np.float64)
    b = np.zeros(n_out, dtype=np.float64)
    lib().or_cpml_profile(int(n_phys), int(npml), float(h), float(dt), float(R), float(vmax),
                          float(f0), int(half), int(n_out), _ptr(a), _ptr(b))
    return a, b


class _Geom:
    """Keeps the receiver index arrays alive while the cfg struct points at them."""

    def __init__(self, cls, g, nshots):
        self.iz = np.ascontiguousarray(g["rec_iz"], dtype=np.int32)
        self.ix = np.ascontiguousarray(g["rec_ix"], dtype=np.int32)
        self.cfg = cls(
            nz=g["nz"], nx=g["nx"], npml=g["npml"], order=g["order"], nt=g["nt"],
            nshots=nshots, src_kind=g.get("src_kind", 0), nrec=len(self.iz),
            dz=g["dz"], dx=g["dx"], dt=g["dt"], pml_R=g.get("pml_R", 1e-3),
            pml_vmax=g.get("pml_vmax", 4500.0), pml_f0=g.get("pml_f0", 10.0),
            rec_iz=self.iz.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
            rec_ix=self.ix.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
            line_len=g.get("line_len", 0), op=g.get("op", 0),
        )


def _stf_array(g, stf, dt_):
    """[S][nt] time functions, or [S][nt][line_len] per-cell ones of a line source."""
    if g.get("src_kind", 0) == 3:
        stf = np.ascontiguousarray(stf, dtype=dt_)
        if stf.ndim == 2:
            stf = stf[None]
        assert stf.ndim == 3 and stf.shape[2] == g["line_len"]
        return stf
    return np.ascontiguousarray(np.atleast_2d(stf), dtype=dt_)


def acoustic_forward(g: dict, c, stf, x0, complex_step: bool = False) -> np.ndarray:
    """Seismograms [nshots][nrec][nt] of the acoustic recursion.

    ``g`` holds the geometry (nz, nx, npml, order, nt, dz, dx, dt, src_kind,
    pml_R, pml_vmax, pml_f0, rec_iz, rec_ix, line_len for a line source, op: 0
    the divergence form div(c^2 grad u), 1 the c^2 Laplacian form);
    c is [nz][nx], stf [S][nt] ([S][nt][line_len] for a line source, src_kind
    3), x0 [S][2] = (x, z) in metres. With ``complex_step`` every input may be
    complex and the map is evaluated in complex arithmetic.
    """
    dt_ = np.complex128 if complex_step else np.float64
    c = np.ascontiguousarray(c, dtype=dt_)
    stf = _stf_array(g, stf, dt_)
    x0 = np.ascontiguousarray(np.reshape(x0, (-1, 2)), dtype=dt_)
    S = stf.shape[0]
    assert x0.shape[0] == S and c.shape == (g["nz"], g["nx"]) and stf.shape[1] == g["nt"]
    geo = _Geom(AcousticCfg, g, S)
    seis = np.zeros((S, geo.cfg.nrec, g["nt"]), dtype=dt_)
    f = lib().or_acoustic_forward_cplx if complex_step else lib().or_acoustic_forward
    if f(ctypes.byref(geo.cfg), _ptr(c), _ptr(stf), _ptr(x0), _ptr(seis)) != 0:
        raise ValueError("oracle forward: invalid configuration or source outside the grid")
    return seis


def acoustic_adjoint(g: dict, c, stf, x0, res):
    """Gradients (dJ/dc [nz][nx], dJ/dstf [S][nt] (line source: [S][nt][line_len]),
    dJ/dx0 [S][2]) of any misfit whose derivative with respect to the
    seismograms is ``res``."""
    c = np.ascontiguousarray(c, dtype=np.float64)
    stf = _stf_array(g, stf, np.float64)
    x0 = np.ascontiguousarray(np.reshape(x0, (-1, 2)), dtype=np.float64)
    res = np.ascontiguousarray(res, dtype=np.float64)
    S = stf.shape[0]
    geo = _Geom(AcousticCfg, g, S)
    assert res.shape == (S, geo.cfg.nrec, g["nt"])
    gc = np.zeros((g["nz"], g["nx"]), dtype=np.float64)
    gs = np.zeros(stf.shape, dtype=np.float64)
    gx = np.zeros((S, 2), dtype=np.float64)
    if lib().or_acoustic_adjoint(ctypes.byref(geo.cfg), _ptr(c), _ptr(stf), _ptr(x0), _ptr(res),
                                 _ptr(gc), _ptr(gs), _ptr(gx)) != 0:
        raise ValueError("oracle adjoint: invalid configuration or out of memory")
    return gc, gs, gx


def acoustic_misfit_grad(g: dict, c, stf, x0, observed):
    """J = 1/2 sum (d - d_obs)^2 over shots, receivers and samples, and its
    gradients with respect to c, stf and x0."""
    d = acoustic_forward(g, c, stf, x0)
    res = d - np.asarray(observed, dtype=np.float64)
    J = 0.5 * float(np.sum(res * res))
    gc, gs, gx = acoustic_adjoint(g, c, stf, x0, res)
    return J, gc, gs, gx


# ---------------------------------------------------------------- elastic
def _el_inputs(vp, vs, rho, stf, x0, mt, dt_):
    vp, vs, rho = (np.ascontiguousarray(a, dtype=dt_) for a in (vp, vs, rho))
    stf = np.ascontiguousarray(np.atleast_2d(stf), dtype=dt_)
    x0 = np.ascontiguousarray(np.reshape(x0, (-1, 2)), dtype=dt_)
    mt = np.ascontiguousarray(np.reshape(mt, (-1, 3)), dtype=dt_)
    assert x0.shape[0] == stf.shape[0] == mt.shape[0]
    return vp, vs, rho, stf, x0, mt


def elastic_forward(g: dict, vp, vs, rho, stf, x0, mt, complex_step: bool = False) -> np.ndarray:
    """Seismograms [nshots][2][nrec][nt] (vx, vz of v^{n+1/2}) of the elastic
    velocity-stress recursion with a moment-tensor source mt [nshots][3]."""
    dt_ = np.complex128 if complex_step else np.float64
    vp, vs, rho, stf, x0, mt = _el_inputs(vp, vs, rho, stf, x0, mt, dt_)
    S = stf.shape[0]
    geo = _Geom(AcousticCfg, g, S)
    seis = np.zeros((S, 2, geo.cfg.nrec, g["nt"]), dtype=dt_)
    f = lib().or_elastic_forward_cplx if complex_step else lib().or_elastic_forward
    if f(ctypes.byref(geo.cfg), _ptr(vp), _ptr(vs), _ptr(rho), _ptr(stf), _ptr(x0), _ptr(mt), _ptr(seis)) != 0:
        raise ValueError("oracle elastic forward: invalid configuration or source outside the grid")
    return seis


def elastic_snapshot(g: dict, vp, vs, rho, stf, x0, mt, step: int) -> np.ndarray:
    """(vx, vz, sxx, szz, sxz) of shot 0 after `step` steps, [5][Nz][Nx]."""
    vp, vs, rho, stf, x0, mt = _el_inputs(vp, vs, rho, stf, x0, mt, np.float64)
    geo = _Geom(AcousticCfg, g, stf.shape[0])
    Nz, Nx = g["nz"] + 2 * g["npml"], g["nx"] + 2 * g["npml"]
    out = np.zeros((5, Nz, Nx))
    if lib().or_elastic_snapshot(ctypes.byref(geo.cfg), _ptr(vp), _ptr(vs), _ptr(rho), _ptr(stf), _ptr(x0),
                                 _ptr(mt), int(step), _ptr(out)) != 0:
        raise ValueError("oracle elastic snapshot failed")
    return out


def elastic_adjoint(g: dict, vp, vs, rho, stf, x0, mt, res):
    """(dJ/dlambda, dJ/dmu, dJ/drho, dJ/dstf, dJ/dx0) for residual res [S][2][nrec][nt]."""
    vp, vs, rho, stf, x0, mt = _el_inputs(vp, vs, rho, stf, x0, mt, np.float64)
    res = np.ascontiguousarray(res, dtype=np.float64)
    S = stf.shape[0]
    geo = _Geom(AcousticCfg, g, S)
    assert res.shape == (S, 2, geo.cfg.nrec, g["nt"])
    gl, gm, gr = (np.zeros((g["nz"], g["nx"])) for _ in range(3))
    gs = np.zeros((S, g["nt"]))
    gx = np.zeros((S, 2))
    if lib().or_elastic_adjoint(ctypes.byref(geo.cfg), _ptr(vp), _ptr(vs), _ptr(rho), _ptr(stf), _ptr(x0),
                                _ptr(mt), _ptr(res), _ptr(gl), _ptr(gm), _ptr(gr), _ptr(gs), _ptr(gx)) != 0:
        raise ValueError("oracle elastic adjoint failed")
    return gl, gm, gr, gs, gx


def elastic_misfit_grad(g: dict, vp, vs, rho, stf, x0, mt, observed):
    d = elastic_forward(g, vp, vs, rho, stf, x0, mt)
    res = d - np.asarray(observed, dtype=np.float64)
    J = 0.5 * float(np.sum(res * res))
    return (J,) + elastic_adjoint(g, vp, vs, rho, stf, x0, mt, res)


def elastic_velocity_grad(vp, vs, rho, g_lam, g_mu, g_rho):
    """(dJ/dvp, dJ/dvs, dJ/drho) from the Lame-parameter gradient, by the chain
    rule through lambda = rho (vp^2 - 2 vs^2), mu = rho vs^2 (Implementation,
    elastic wave equation: the inversion parameters are lambda, mu, rho)."""
    vp, vs, rho = (np.asarray(a, np.float64) for a in (vp, vs, rho))
    dl_dvp, dl_dvs, dl_drho = 2 * rho * vp, -4 * rho * vs, vp ** 2 - 2 * vs ** 2
    dm_dvs, dm_drho = 2 * rho * vs, vs ** 2
    return (g_lam * dl_dvp,
            g_lam * dl_dvs + g_mu * dm_dvs,
            g_lam * dl_drho + g_mu * dm_drho + g_rho)
