"""Seeded synthetic inputs for the seismic-inversion workloads.

This module only builds INPUTS (velocity models, acquisition geometry, source
wavelets). It holds none of the method's arithmetic: the wave propagation,
misfit and gradients live in the CUDA library (and, independently, in the CPU
oracle used by the tests). Both sides receive the same arrays from here.

The paper's own models (Marmousi; a layered crust with elliptical inclusions,
Full-waveform Inversion section) are not available, so seeded layered models
with dipping interfaces and faults stand in for them.
"""

from __future__ import annotations

import math

import numpy as np


def ricker(f0: float, dt: float, nt: int, t0: float | None = None, dtype=np.float32) -> np.ndarray:
    """Ricker wavelet (1 - 2 pi^2 f0^2 tau^2) exp(-pi^2 f0^2 tau^2), tau = t - t0,
    sampled at t_n = n dt; t0 defaults to 1.2 / f0, peak value 1 (the paper
    uses a Ricker source time function, Full-waveform Inversion section)."""
    if t0 is None:
        t0 = 1.2 / f0
    t = np.arange(nt, dtype=np.float64) * dt - t0
    a = (math.pi * f0 * t) ** 2
    return ((1.0 - 2.0 * a) * np.exp(-a)).astype(dtype)


def gardner_density(vp: np.ndarray) -> np.ndarray:
    """Gardner's relation rho = 310 vp^0.25 (kg/m^3, vp in m/s)."""
    return (310.0 * np.power(vp.astype(np.float64), 0.25)).astype(np.float32)


def layered_model(seed: int, nz: int, nx: int, dx: float, vmin: float = 1500.0,
                  vmax: float = 4500.0, n_layers=(8, 15), n_faults: int = 2) -> np.ndarray:
    """Dipping-layer velocity model [nz][nx] (m/s), seeded.

    K ~ U{n_layers} interfaces z_k(x) = zbar_k + tan(theta_k)(x - xbar),
    theta_k ~ U(-15, 15) degrees; the velocity of a point is that of the number
    of interfaces above it, increasing from vmin to vmax with +-10% jitter.
    ``n_faults`` normal faults (dip 60-80 degrees, throw 20-100 m) shift the
    hanging wall down.
    """
    rng = np.random.default_rng(seed)
    K = int(rng.integers(n_layers[0], n_layers[1] + 1))
    depth = nz * dx
    width = nx * dx
    zbar = np.sort(rng.uniform(0.05 * depth, 0.95 * depth, K))
    theta = np.deg2rad(rng.uniform(-15.0, 15.0, K))
    base = np.linspace(vmin, vmax, K + 1)
    jitter = 1.0 + rng.uniform(-0.1, 0.1, K + 1)
    vel = np.clip(base * jitter, vmin, vmax)
    vel = np.maximum.accumulate(vel)
    faults = []
    for _ in range(n_faults):
        xf = rng.uniform(0.2 * width, 0.8 * width)
        dip = np.deg2rad(rng.uniform(60.0, 80.0))
        throw = rng.uniform(20.0, 100.0)
        side = 1.0 if rng.uniform() < 0.5 else -1.0
        faults.append((xf, dip, throw, side))
    z = (np.arange(nz, dtype=np.float64) * dx)[:, None]
    x = (np.arange(nx, dtype=np.float64) * dx)[None, :]
    z_eff = np.broadcast_to(z, (nz, nx)).copy()
    for xf, dip, throw, side in faults:
        trace = xf + z / math.tan(dip) * side
        hanging = (x - trace) * side > 0
        z_eff = np.where(hanging, z_eff - throw, z_eff)
    xbar = 0.5 * width
    count = np.zeros((nz, nx), dtype=np.int64)
    for k in range(K):
        zk = zbar[k] + math.tan(theta[k]) * (x - xbar)
        count += (z_eff >= zk).astype(np.int64)
    return vel[count].astype(np.float32)


def smooth(model: np.ndarray, sigma_cells: float) -> np.ndarray:
    """Gaussian-smoothed starting model (edge values extended)."""
    from scipy.ndimage import gaussian_filter

    return gaussian_filter(model.astype(np.float64), sigma_cells, mode="nearest").astype(np.float32)


def acoustic_small(perturbed: bool = False) -> dict:
    """100 x 100 two-layer acoustic problem: dx = dz = 10 m, dt = 1 ms, 500
    steps, 4th order, 20 CPML cells; 2000 m/s above 500 m, 3000 m/s below;
    one 10 Hz Ricker point source at (x, z) = (500, 50) m; 50 receivers at
    iz = 5, ix = 1, 3, ..., 99. ``perturbed`` moves the interface to 520 m
    (the model that produces the observed data)."""
    nz = nx = 100
    c = np.full((nz, nx), 2000.0, dtype=np.float32)
    c[(52 if perturbed else 50):, :] = 3000.0
    nt, dt, f0 = 500, 1e-3, 10.0
    return dict(
        name="acoustic-100x100-o4-nt500", nz=nz, nx=nx, dz=10.0, dx=10.0, dt=dt, nt=nt, order=4,
        npml=20, pml_R=1e-3, pml_vmax=4500.0, pml_f0=f0, src_kind=0, c=c,
        stf=ricker(f0, dt, nt)[None, :].copy(), x0=np.array([[500.0, 50.0]], dtype=np.float32),
        rec_iz=np.full(50, 5, dtype=np.int32), rec_ix=np.arange(1, 100, 2, dtype=np.int32),
        ckpt_every=100,
    )


def acoustic_fwi(nshots: int = 16, nt: int = 3000, seed: int = 2003) -> dict:
    """201 x 601 acoustic FWI gradient problem: dx = 10 m, dt = 0.8 ms, 3000
    steps, 8th order, 32 CPML cells (R = 1e-5); seeded dipping-layer model
    1500-4500 m/s with 2 faults (true model) and its Gaussian smoothing
    (sigma = 15 cells, starting model); ``nshots`` 8 Hz Ricker point sources
    at iz = 2 evenly spread over ix = 0..600; 301 receivers at iz = 2,
    ix = 0, 2, ..., 600; checkpoint every 100 steps."""
    nz, nx, dx, dt, f0 = 201, 601, 10.0, 0.8e-3, 8.0
    true = layered_model(seed, nz, nx, dx)
    start = smooth(true, 15.0)
    ix_src = np.linspace(0, nx - 1, nshots)
    x0 = np.stack([ix_src * dx, np.full(nshots, 2 * dx)], axis=1).astype(np.float32)
    stf = np.tile(ricker(f0, dt, nt), (nshots, 1))
    return dict(
        name=f"acoustic-201x601-o8-nt{nt}-{nshots}shots", nz=nz, nx=nx, dz=dx, dx=dx, dt=dt,
        nt=nt, order=8, npml=32, pml_R=1e-5, pml_vmax=4500.0, pml_f0=f0, src_kind=0,
        c=start, c_true=true, stf=stf, x0=x0,
        rec_iz=np.full(301, 2, dtype=np.int32), rec_ix=np.arange(0, 601, 2, dtype=np.int32),
        ckpt_every=100,
    )


def acoustic_xl(nshots: int = 256, nt: int = 3000) -> dict:
    """The 201 x 601 FWI discretisation with many shots, so that the per-step
    working set is several times the L2 cache."""
    d = acoustic_fwi(nshots=nshots, nt=nt)
    d["name"] = f"acoustic-201x601-o8-nt{nt}-{nshots}shots"
    return d


def uneven_instance(seed: int, i: int) -> dict:
    """Instance i of the batched uneven workload (seed ``seed``): nz ~ U{128..512}
    and nx ~ U{128..1024} in steps of 32, nt ~ U{1000..4000} in steps of 100,
    shots ~ U{4..16}; the 201 x 601 discretisation (order 8, 32 CPML cells,
    dx = 10 m, dt = 0.8 ms, 8 Hz Ricker); a layered model without faults (true)
    and its sigma = 10 cell smoothing (start); sources and receivers (every 4th
    cell) at iz = 2."""
    rng = np.random.default_rng([seed, i])
    nz = int(rng.integers(4, 17)) * 32
    nx = int(rng.integers(4, 33)) * 32
    nt = int(rng.integers(10, 41)) * 100
    S = int(rng.integers(4, 17))
    dx, dt, f0 = 10.0, 0.8e-3, 8.0
    true = layered_model(int(rng.integers(1 << 30)), nz, nx, dx, n_faults=0)
    start = smooth(true, 10.0)
    x0 = np.stack([np.linspace(0, nx - 1, S) * dx, np.full(S, 2 * dx)], axis=1).astype(np.float32)
    rec_ix = np.arange(0, nx, 4, dtype=np.int32)
    return dict(
        name=f"uneven-{seed}-{i}-{nz}x{nx}-nt{nt}-{S}shots", nz=nz, nx=nx, dz=dx, dx=dx, dt=dt, nt=nt,
        order=8, npml=32, pml_R=1e-5, pml_vmax=4500.0, pml_f0=f0, src_kind=0, c=start, c_true=true,
        stf=np.tile(ricker(f0, dt, nt), (S, 1)), x0=x0, rec_iz=np.full(rec_ix.shape, 2, dtype=np.int32),
        rec_ix=rec_ix, ckpt_every=100,
    )


def random_acoustic(seed: int, nz: int, nx: int, nt: int, nshots: int, order: int, npml: int,
                    src_kind: int = 0, nrec: int = 7, dx: float = 10.0, dt: float = 1e-3,
                    f0: float = 15.0) -> dict:
    """Small seeded heterogeneous problem for parity and adjoint tests: smooth
    random velocity 1800-2600 m/s, sources and receivers at random interior
    cells (Gaussian sources kept 3 cells away from the padded edge)."""
    rng = np.random.default_rng(seed)
    c = 2200.0 + 400.0 * np.tanh(rng.standard_normal((nz, nx)))
    c = smooth(c.astype(np.float32), 1.5)
    stf = np.stack([ricker(f0 * (1.0 + 0.2 * s), dt, nt) for s in range(nshots)])
    margin = 0 if src_kind == 0 else max(0, 3 - npml)
    xs = rng.uniform(margin, nx - 1 - margin, nshots) * dx
    zs = rng.uniform(margin, nz - 1 - margin, nshots) * dx
    return dict(
        name=f"acoustic-rand-{nz}x{nx}-o{order}-nt{nt}", nz=nz, nx=nx, dz=dx, dx=dx, dt=dt,
        nt=nt, order=order, npml=npml, pml_R=1e-3, pml_vmax=4500.0, pml_f0=f0,
        src_kind=src_kind, c=c, stf=stf.astype(np.float32),
        x0=np.stack([xs, zs], axis=1).astype(np.float32),
        rec_iz=rng.integers(0, nz, nrec).astype(np.int32),
        rec_ix=rng.integers(0, nx, nrec).astype(np.int32), ckpt_every=max(1, nt // 4),
    )


def plane_wave(wavelet: np.ndarray, dt: float, theta_deg: float, c_ref: float, line_len: int,
               dx: float) -> np.ndarray:
    """Per-cell time functions [nt][line_len] of a plane wave launched from a
    line of cells (the paper's plane-wave sources: a line of sources fired
    with delays): cell q fires the sampled ``wavelet`` delayed by
    tau_q = q dx sin(theta) / c_ref, shifted so that the earliest cell fires
    at delay 0, by linear interpolation between samples (zero before t = 0)."""
    nt = wavelet.shape[0]
    tau = np.arange(line_len) * dx * np.sin(np.radians(theta_deg)) / c_ref
    tau -= tau.min()
    t = np.arange(nt)[:, None] * dt - tau[None, :]
    k = np.floor(t / dt).astype(np.int64)
    f = t / dt - k
    w = np.concatenate([wavelet.astype(np.float64), [0.0]])
    k0 = np.clip(k, -1, nt - 1)
    k1 = np.clip(k + 1, -1, nt - 1)
    v0 = np.where(k0 >= 0, w[np.maximum(k0, 0)], 0.0)
    v1 = np.where((k1 >= 0) & (k + 1 < nt), w[np.maximum(k1, 0)], 0.0)
    return ((1.0 - f) * v0 + f * v1).astype(np.float32)


def line_source_problem(seed: int, nz: int, nx: int, nt: int, nshots: int, order: int, npml: int,
                        line_len: int, nrec: int = 7, dx: float = 10.0, dt: float = 1e-3,
                        f0: float = 15.0, rec_on_line: bool = True) -> dict:
    """Small seeded heterogeneous problem with plane-wave (line) sources: shot s
    fires a line of ``line_len`` cells along one row with a Ricker plane wave
    at angle -30 + 20 s degrees (as the paper's bottom plane waves); some
    receivers lie on the source row when ``rec_on_line``."""
    d = random_acoustic(seed, nz, nx, nt, nshots, order, npml, src_kind=0, nrec=nrec, dx=dx, dt=dt, f0=f0)
    rng = np.random.default_rng(seed + 1)
    rows = rng.integers(0, nz, nshots)
    cols = rng.integers(0, nx - line_len + 1, nshots)
    wav = ricker(f0, dt, nt)
    stf = np.stack([plane_wave(wav, dt, -30.0 + 20.0 * s, 2200.0, line_len, dx) for s in range(nshots)])
    x0 = np.stack([cols * dx, rows * dx], axis=1).astype(np.float32)
    if rec_on_line and nrec >= 2:
        d["rec_iz"][:2] = rows[0]
        d["rec_ix"][:2] = [cols[0], cols[0] + line_len - 1]
    d.update(name=f"acoustic-line-{nz}x{nx}-o{order}-nt{nt}", src_kind=3, line_len=line_len, stf=stf, x0=x0)
    return d


def plane_wave_survey(nz: int = 60, nx: int = 100, nt: int = 700, dx: float = 10.0, dt: float = 1e-3,
                      f0: float = 12.0, angles=(-30.0, -10.0, 10.0, 30.0), order: int = 8, npml: int = 20,
                      seed: int = 31) -> dict:
    """A small instance of the paper's plane-wave FWI setting (a layered crust
    with an elliptical anomaly, plane waves from the bottom at -30, -10, 10, 30
    degrees, receivers along the surface; the paper gives no sizes, so these
    are this generator's): true model with a slow ellipse in two layers, start
    model = the layers without the ellipse; one shot per angle, each a line
    source along the deepest physical row firing a Ricker plane wave."""
    rng = np.random.default_rng(seed)
    z = np.arange(nz)[:, None] * dx
    x = np.arange(nx)[None, :] * dx
    layers = np.where(z < nz * dx * 0.5, 2200.0, 2800.0) + 0.0 * x
    ex, ez = nx * dx * (0.45 + 0.1 * rng.random()), nz * dx * 0.45
    ell = ((x - ex) / (0.18 * nx * dx)) ** 2 + ((z - ez) / (0.12 * nz * dx)) ** 2 < 1.0
    true = np.where(ell, layers - 300.0, layers).astype(np.float32)
    wav = ricker(f0, dt, nt)
    stf = np.stack([plane_wave(wav, dt, a, 2800.0, nx, dx) for a in angles])
    x0 = np.stack([np.zeros(len(angles)), np.full(len(angles), (nz - 1) * dx)], axis=1).astype(np.float32)
    return dict(name=f"acoustic-planewave-{nz}x{nx}-nt{nt}", nz=nz, nx=nx, dz=dx, dx=dx, dt=dt, nt=nt, order=order,
                npml=npml, pml_R=1e-3, pml_vmax=4500.0, pml_f0=f0, src_kind=3, line_len=nx, c=layers.astype(np.float32),
                c_true=true, stf=stf, x0=x0, rec_iz=np.full(nx // 2, 1, np.int32),
                rec_ix=np.arange(0, nx, 2, dtype=np.int32), ckpt_every=100)


def double_couple(phi: np.ndarray) -> np.ndarray:
    """2D double-couple moment tensors (Mxx, Mzz, Mxz) = (-sin 2phi, sin 2phi, cos 2phi)."""
    return np.stack([-np.sin(2 * phi), np.sin(2 * phi), np.cos(2 * phi)], axis=1)


MOMENT_SCALE = 1e12  # N m per unit moment-tensor entry: keeps seismograms O(0.1-1) m/s in FP32


def elastic_layered(nshots: int = 32, nt: int = 4000, seed: int = 3) -> dict:
    """300 x 800 elastic problem: dx = 5 m, dt = 0.5 ms, 4000 steps, 4th order,
    32 CPML cells; seeded dipping layers (no faults) with vp 1800-4500 m/s,
    vs = vp / 1.73, Gardner density; ``nshots`` Gaussian (sigma = dx/2)
    moment-tensor sources at depths 400-1200 m with random double-couple
    mechanisms and a 10 Hz Ricker moment rate; 200 receivers at iz = 2 every 4
    cells recording vx and vz."""
    nz, nx, dx, dt, f0 = 300, 800, 5.0, 0.5e-3, 10.0
    vp = layered_model(seed, nz, nx, dx, vmin=1800.0, vmax=4500.0, n_faults=0)
    vs = (vp / 1.73).astype(np.float32)
    rho = gardner_density(vp)
    rng = np.random.default_rng(seed + 100)
    xs = rng.uniform(40, nx - 40, nshots) * dx
    zs = rng.uniform(400.0, 1200.0, nshots)
    mt = (double_couple(rng.uniform(0, np.pi, nshots)) * MOMENT_SCALE).astype(np.float32)
    stf = np.tile(ricker(f0, dt, nt), (nshots, 1))
    return dict(
        name=f"elastic-300x800-o4-nt{nt}-{nshots}shots", nz=nz, nx=nx, dz=dx, dx=dx, dt=dt, nt=nt, order=4,
        npml=32, pml_R=1e-5, pml_vmax=4500.0, pml_f0=f0, src_kind=1, vp=vp, vs=vs, rho=rho, stf=stf,
        x0=np.stack([xs, zs], axis=1).astype(np.float32), mt=mt,
        rec_iz=np.full(200, 2, dtype=np.int32), rec_ix=np.arange(0, 800, 4, dtype=np.int32), ckpt_every=100,
    )


def random_elastic(seed: int, nz: int, nx: int, nt: int, nshots: int, order: int, npml: int,
                   src_kind: int = 1, nrec: int = 7, dx: float = 10.0, dt: float = 1e-3,
                   f0: float = 15.0) -> dict:
    """Small seeded heterogeneous elastic problem for parity tests."""
    rng = np.random.default_rng(seed)
    vp = smooth((2600.0 + 600.0 * rng.random((nz, nx))).astype(np.float32), 1.5)
    vs = (vp / (1.6 + 0.3 * rng.random((nz, nx)))).astype(np.float32)
    rho = (310.0 * vp.astype(np.float64) ** 0.25 * (1 + 0.1 * rng.random((nz, nx)))).astype(np.float32)
    stf = np.stack([ricker(f0 * (1.0 + 0.2 * s), dt, nt) for s in range(nshots)])
    margin = 0 if src_kind == 0 else max(0, 4 - npml)
    xs = rng.uniform(margin, nx - 1 - margin, nshots) * dx
    zs = rng.uniform(margin, nz - 1 - margin, nshots) * dx
    mt = (rng.standard_normal((nshots, 3)) * MOMENT_SCALE).astype(np.float32)
    return dict(
        name=f"elastic-rand-{nz}x{nx}-o{order}-nt{nt}", nz=nz, nx=nx, dz=dx, dx=dx, dt=dt, nt=nt, order=order,
        npml=npml, pml_R=1e-3, pml_vmax=4500.0, pml_f0=f0, src_kind=src_kind, vp=vp, vs=vs, rho=rho,
        stf=stf.astype(np.float32), x0=np.stack([xs, zs], axis=1).astype(np.float32), mt=mt,
        rec_iz=rng.integers(0, nz, nrec).astype(np.int32), rec_ix=rng.integers(0, nx, nrec).astype(np.int32),
        ckpt_every=max(1, nt // 4),
    )
