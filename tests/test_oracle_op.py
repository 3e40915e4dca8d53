"""Pins of the oracle's second acoustic operator, u_tt = c^2 (Laplacian u) + f
(op 1; the paper's Eq. acoustic is the divergence form div(c^2 grad u), op 0).

* In a homogeneous medium the two forms are the same operator, CPML included:
  identical seismograms (against the op 0 path, pinned by the analytic Green's
  function).
* At a 2000 -> 3000 m/s interface the c^2 Laplacian form reflects with
  R = (c2 - c1)/(c2 + c1) = +0.2 (continuity of u and du/dz), the opposite sign
  of the divergence form's -0.2.
* Its exact adjoint: complex-step derivatives of the misfit in c (single cells
  incl. CPML-adjacent, source and receiver cells, and a random direction) and in
  the source time function."""

import math

import numpy as np
import pytest

import oracle
from paper_2003_06027_gb300 import synth

from test_oracle_acoustic import _geom, _green_ricker, _misfit


def test_homogeneous_medium_both_forms_agree():
    for order, npml in ((4, 8), (8, 10)):
        g0 = _geom(30, 40, 160, order=order, npml=npml, rec=([0, 5, 29], [3, 20, 39]))
        g1 = dict(g0, op=1)
        c = np.full((30, 40), 2300.0)
        s = synth.ricker(18.0, 1e-3, 160, dtype=np.float64)[None]
        x0 = [[150.0, 120.0]]
        d0 = oracle.acoustic_forward(g0, c, s, x0)
        d1 = oracle.acoustic_forward(g1, c, s, x0)
        assert np.linalg.norm(d1 - d0) <= 1e-12 * np.linalg.norm(d0)
    # and they differ once the medium varies
    c[15:, :] = 3000.0
    assert np.linalg.norm(oracle.acoustic_forward(g1, c, s, x0) - oracle.acoustic_forward(g0, c, s, x0)) > 0


def test_interface_reflection_positive():
    dx, dt, f0 = 5.0, 0.5e-3, 10.0
    nz, nx, nt = 140, 240, 1000
    zs, zi = 10, 70
    c = np.full((nz, nx), 2000.0)
    c[zi:, :] = 3000.0
    g = dict(_geom(nz, nx, nt, order=8, npml=30, dx=dx, dt=dt, f0=f0, rec=([zs], [nx // 2 + 4])), op=1)
    stf = synth.ricker(f0, dt, nt, dtype=np.float64)[None]
    d = oracle.acoustic_forward(g, c, stf, [[nx // 2 * dx, zs * dx]])[0, 0]
    zint = (zi - 0.5) * dx
    r_img = math.hypot(4 * dx, 2 * (zint - zs * dx))
    t = (np.arange(nt) + 1) * dt
    ref = _green_ricker(r_img, 2000.0, f0, t)
    win = t > 0.2
    pk = np.argmax(np.abs(ref[win]))
    ratio = d[win][pk] / ref[win][pk]
    assert 0.17 < ratio < 0.23, ratio


def test_gradient_vs_complex_step():
    g = dict(_geom(24, 32, 150, order=4, npml=8, rec=([0, 3, 20, 23], [0, 16, 30, 5])), op=1)
    rng = np.random.default_rng(7)
    c_true = 2000 + 500 * rng.random((24, 32))
    c = synth.smooth(c_true.astype(np.float32), 2.0).astype(np.float64)
    x0 = np.array([[80.0, 50.0], [250.0, 30.0]])
    s = np.stack([synth.ricker(f, 1e-3, 150, dtype=np.float64) for f in (18.0, 22.0)])
    obs = oracle.acoustic_forward(g, c_true, s, x0)
    J, gc, gs, _ = oracle.acoustic_misfit_grad(g, c, s, x0, obs)
    assert J > 0
    h = 1e-30
    for (i, j) in [(0, 0), (23, 31), (5, 8), (0, 16), (12, 17)]:
        e = np.zeros_like(c)
        e[i, j] = 1.0
        cs = _misfit(g, c + 1j * h * e, s, x0, obs, cs=True).imag / h
        assert gc[i, j] == pytest.approx(cs, rel=1e-10, abs=1e-10 * np.abs(gc).max())
    dirn = rng.standard_normal(c.shape)
    cs = _misfit(g, c + 1j * h * dirn, s, x0, obs, cs=True).imag / h
    assert np.sum(gc * dirn) == pytest.approx(cs, rel=1e-10)
    ds = rng.standard_normal(s.shape)
    cs = _misfit(g, c, s + 1j * h * ds, x0, obs, cs=True).imag / h
    assert np.sum(gs * ds) == pytest.approx(cs, rel=1e-10)


def test_line_source_superposition_and_dot_product():
    """With op 1 a line source is still the sum of its cells' point sources
    (the operator is linear in u whatever multiplies it), and the map from the
    per-cell time functions to the seismograms passes the dot-product test
    against the oracle's op-1 source gradient."""
    d = synth.line_source_problem(14, 18, 24, 80, 2, 4, 5, line_len=6)
    g = {k: d[k] for k in ("nz", "nx", "npml", "order", "nt", "dz", "dx", "dt", "src_kind", "pml_R", "pml_vmax",
                           "pml_f0", "rec_iz", "rec_ix", "line_len")}
    g["op"] = 1
    c = np.float64(d["c"])
    seis = oracle.acoustic_forward(g, c, np.float64(d["stf"]), np.float64(d["x0"]))
    gp = dict(g, src_kind=0)
    for s in range(2):
        want = np.zeros_like(seis[s])
        for q in range(d["line_len"]):
            xq = np.array([[d["x0"][s, 0] + q * d["dx"], d["x0"][s, 1]]])
            want += oracle.acoustic_forward(gp, c, np.float64(d["stf"][s, :, q])[None], xq)[0]
        assert np.linalg.norm(seis[s] - want) <= 1e-12 * np.linalg.norm(want)
    rng = np.random.default_rng(15)
    a = rng.standard_normal(d["stf"].shape)
    Fa = oracle.acoustic_forward(g, c, a, np.float64(d["x0"]))
    r = rng.standard_normal(Fa.shape)
    _, FTr, _ = oracle.acoustic_adjoint(g, c, a, np.float64(d["x0"]), r)
    lhs, rhs = float(np.sum(Fa * r)), float(np.sum(a * FTr))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs))
