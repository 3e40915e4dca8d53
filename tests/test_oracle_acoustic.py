"""Pins of the FP64 acoustic oracle against facts fixed outside it: closed
forms, the analytic 2D Green's function, reciprocity, linearity, dot-product
adjoint tests, complex-step and finite-difference gradients. CPU only."""

import math

import numpy as np
import pytest

import oracle
from paper_2003_06027_gb300 import synth


def _geom(nz, nx, nt, order=4, npml=10, dx=10.0, dt=1e-3, src_kind=0, rec=None, f0=15.0, R=1e-3):
    rec = rec if rec is not None else ([nz // 3, nz - 2], [nx // 4, nx - 3])
    return dict(nz=nz, nx=nx, npml=npml, order=order, nt=nt, dz=dx, dx=dx, dt=dt,
                src_kind=src_kind, pml_R=R, pml_vmax=4500.0, pml_f0=f0,
                rec_iz=np.asarray(rec[0], np.int32), rec_ix=np.asarray(rec[1], np.int32))


# ---------------------------------------------------------------- coefficients
def test_fd_coefficients_closed_form():
    # Staggered-grid weights from the Taylor moment conditions (Fornberg 1988;
    # the 4th-order pair is Levander's 9/8, -1/24).
    np.testing.assert_allclose(oracle.fd_coeffs(4), [9 / 8, -1 / 24], rtol=0, atol=1e-15)
    np.testing.assert_allclose(oracle.fd_coeffs(8), [1225 / 1024, -245 / 3072, 49 / 5120, -5 / 7168],
                               rtol=0, atol=1e-15)


@pytest.mark.parametrize("order", [4, 8])
def test_fd_exact_on_polynomials(order):
    # D+ at x = 1/2 must return the exact derivative of every polynomial of
    # degree <= order - 1, and must fail for degree = order + 1.
    a = oracle.fd_coeffs(order)
    N = order // 2
    for deg in range(order):
        d = sum(a[k - 1] * ((k) ** deg - (-k + 1) ** deg) for k in range(1, N + 1))
        exact = deg * 0.5 ** (deg - 1) if deg >= 1 else 0.0
        assert abs(d - exact) < 1e-9 * max(1.0, abs(exact)), (deg, d, exact)
    deg = order + 1
    d = sum(a[k - 1] * ((k) ** deg - (-k + 1) ** deg) for k in range(1, N + 1))
    assert abs(d - deg * 0.5 ** (deg - 1)) > 1e-6


def test_cpml_profile_closed_form():
    n, npml, h, dt, R, vmax, f0 = 50, 10, 10.0, 1e-3, 1e-3, 4500.0, 10.0
    N = n + 2 * npml
    a, b = oracle.cpml_profile(n, npml, h, dt, R, vmax, f0, 0, N)
    ah, bh = oracle.cpml_profile(n, npml, h, dt, R, vmax, f0, 1, N)
    # interior (and the first/last physical node) is untouched
    assert np.all(a[npml:npml + n] == 0) and np.all(b[npml:npml + n] == 1)
    # outermost node: l = L so d = d0, alpha = 0 -> b = exp(-d0 dt), a = b - 1
    L = npml * h
    d0 = -3 * vmax * math.log(R) / (2 * L)
    assert b[0] == pytest.approx(math.exp(-d0 * dt), rel=1e-14)
    assert a[0] == pytest.approx(math.exp(-d0 * dt) - 1, rel=1e-14)
    assert b[-1] == pytest.approx(b[0], rel=1e-14)
    # symmetric about the centre, damping grows outward, a in (-1, 0]
    np.testing.assert_allclose(a, a[::-1], atol=1e-15)
    np.testing.assert_allclose(ah[:N - 1], ah[:N - 1][::-1], atol=1e-15)
    assert np.all(np.diff(b[:npml + 1]) > 0)
    assert np.all(a <= 0) and np.all(a > -1) and np.all(ah[:N - 1] <= 0)
    # a half point 4.5 cells deep: l = 4.5 h
    l = 4.5 * h
    d = d0 * (l / L) ** 2
    al = math.pi * f0 * (1 - l / L)
    bb = math.exp(-(d + al) * dt)
    assert bh[npml - 5] == pytest.approx(bb, rel=1e-14)
    assert ah[npml - 5] == pytest.approx(d * (bb - 1) / (d + al), rel=1e-13)


# ---------------------------------------------------------------- forward map
def test_zero_source_zero_output_and_linearity():
    g = _geom(20, 24, 80)
    rng = np.random.default_rng(0)
    c = 2000 + 300 * rng.random((20, 24))
    x0 = np.array([[100.0, 80.0], [130.0, 90.0]])
    s1, s2 = rng.standard_normal((2, 80)), rng.standard_normal((2, 80))
    assert np.all(oracle.acoustic_forward(g, c, np.zeros((2, 80)), x0) == 0)
    d1 = oracle.acoustic_forward(g, c, s1, x0)
    d2 = oracle.acoustic_forward(g, c, s2, x0)
    d12 = oracle.acoustic_forward(g, c, 2.5 * s1 - 0.75 * s2, x0)
    np.testing.assert_allclose(d12, 2.5 * d1 - 0.75 * d2, rtol=0, atol=1e-13 * np.abs(d12).max())


def _swap_traces(g, c, pa, pb, stf):
    """Trace at b for a point source at a, and at a for a source at b."""
    ga = dict(g, rec_iz=np.array([pb[0]], np.int32), rec_ix=np.array([pb[1]], np.int32))
    gb = dict(g, rec_iz=np.array([pa[0]], np.int32), rec_ix=np.array([pa[1]], np.int32))
    da = oracle.acoustic_forward(ga, c, stf, [[pa[1] * g["dx"], pa[0] * g["dz"]]])
    db = oracle.acoustic_forward(gb, c, stf, [[pb[1] * g["dx"], pb[0] * g["dz"]]])
    return da[0, 0], db[0, 0]


@pytest.mark.parametrize("order", [4, 8])
def test_reciprocity_dirichlet_exact(order):
    # With no absorbing layer the discrete operator div(c^2 grad) = -D+^T M D+
    # is symmetric, so swapping source and receiver gives the same trace.
    g = _geom(30, 36, 300, order=order, npml=0)
    rng = np.random.default_rng(1)
    c = synth.smooth((1800 + 900 * rng.random((30, 36))).astype(np.float32), 1.0).astype(np.float64)
    stf = synth.ricker(20.0, 1e-3, 300, dtype=np.float64)[None]
    ta, tb = _swap_traces(g, c, (7, 5), (22, 29), stf)
    assert np.abs(ta).max() > 0
    np.testing.assert_allclose(ta, tb, rtol=0, atol=1e-12 * np.abs(ta).max())


def test_reciprocity_with_cpml():
    g = _geom(30, 36, 300, order=4, npml=12, f0=20.0)
    rng = np.random.default_rng(2)
    c = synth.smooth((1800 + 900 * rng.random((30, 36))).astype(np.float32), 1.0).astype(np.float64)
    stf = synth.ricker(20.0, 1e-3, 300, dtype=np.float64)[None]
    ta, tb = _swap_traces(g, c, (4, 3), (25, 31), stf)
    assert np.linalg.norm(ta - tb) <= 1e-3 * np.linalg.norm(ta)


def _green_ricker(r, c, f0, t):
    """Analytic 2D Green's function of u_tt - c^2 lap u = delta(x) delta(t),
    H(t - r/c) / (2 pi c sqrt(c^2 t^2 - r^2)), convolved with a Ricker source
    starting at t = 0: with tau = (r/c) cosh(eta) the integral is
    (1 / (2 pi c^2)) int_0^{acosh(ct/r)} s(t - (r/c) cosh eta) d eta."""
    xg, wg = np.polynomial.legendre.leggauss(400)
    t0 = 1.2 / f0
    out = np.zeros_like(t)
    for i, ti in enumerate(t):
        if ti <= r / c:
            continue
        emax = math.acosh(c * ti / r)
        eta = 0.5 * emax * (xg + 1)
        tau = ti - (r / c) * np.cosh(eta)
        a = (math.pi * f0 * (tau - t0)) ** 2
        s = (1 - 2 * a) * np.exp(-a)
        out[i] = 0.5 * emax * np.sum(wg * s) / (2 * math.pi * c * c)
    return out


def _green_case(dx, dt, order):
    c0, f0 = 2000.0, 10.0
    L = 1200.0
    n = int(round(L / dx)) + 1
    nt = int(round(0.42 / dt))
    src = (n // 2, n // 2)
    off = int(round(300.0 / dx))
    g = _geom(n, n, nt, order=order, npml=20, dx=dx, dt=dt, f0=f0,
              rec=([src[0], src[0] + off], [src[1] + off, src[1]]))
    c = np.full((n, n), c0)
    stf = synth.ricker(f0, dt, nt, dtype=np.float64)[None]
    d = oracle.acoustic_forward(g, c, stf, [[src[1] * dx, src[0] * dx]])[0]
    t = (np.arange(nt) + 1) * dt  # sample n holds u^{n+1}
    ref = _green_ricker(off * dx, c0, f0, t)
    return max(np.linalg.norm(d[k] - ref) / np.linalg.norm(ref) for k in range(2))


@pytest.mark.slow
def test_homogeneous_green_function_and_convergence():
    # 300 m offset, window ends before any boundary echo. The scheme is second
    # order in time, so with 8th order in space halving dx and dt must cut the
    # error about 4x. (At 4th order and dx = 10 m the spatial and temporal
    # dispersion errors have opposite signs and partly cancel, so there the
    # ratio is not a clean test of the order.)
    e4 = _green_case(10.0, 1e-3, 4)
    e8 = _green_case(10.0, 1e-3, 8)
    e8h = _green_case(5.0, 0.5e-3, 8)
    assert e4 < 2e-2, e4
    assert e8 < 5e-3, e8
    assert 3.5 < e8 / e8h < 4.5, (e8, e8h)


def test_interface_reflection_sign_and_size():
    # Divergence form: continuity of u and c^2 du/dz gives the normal-incidence
    # reflection coefficient R = (c1 - c2)/(c1 + c2) = -0.2 for 2000 -> 3000 m/s.
    dx, dt, f0 = 5.0, 0.5e-3, 10.0
    nz, nx, nt = 140, 240, 1000
    zs, zi = 10, 70  # source depth and interface (cells)
    c = np.full((nz, nx), 2000.0)
    c[zi:, :] = 3000.0
    g = _geom(nz, nx, nt, order=8, npml=30, dx=dx, dt=dt, f0=f0, rec=([zs], [nx // 2 + 4]))
    stf = synth.ricker(f0, dt, nt, dtype=np.float64)[None]
    d = oracle.acoustic_forward(g, c, stf, [[nx // 2 * dx, zs * dx]])[0, 0]
    # the interface sits half-way between the last 2000 m/s node and the first
    # 3000 m/s node of the arithmetic-mean half-point coefficient
    zint = (zi - 0.5) * dx
    r_img = math.hypot(4 * dx, 2 * (zint - zs * dx))
    t = (np.arange(nt) + 1) * dt
    ref = _green_ricker(r_img, 2000.0, f0, t)
    win = t > 0.2  # direct wave (4 cells offset) has passed by then
    refl = d[win]
    pk = np.argmax(np.abs(ref[win]))
    ratio = refl[pk] / ref[win][pk]
    assert -0.23 < ratio < -0.17, ratio


def test_cpml_absorbs():
    # Trace in a small domain with CPML versus the same source/receiver in a
    # domain so large that its edges are never reached within the window.
    dx, dt, f0, nt = 10.0, 1e-3, 10.0, 600
    small = 60
    big = 300
    stf = synth.ricker(f0, dt, nt, dtype=np.float64)[None]
    out = []
    for n, npml in ((small, 20), (big, 0)):
        o = (n - small) // 2
        g = _geom(n, n, nt, order=4, npml=npml, dx=dx, dt=dt, f0=f0, R=1e-3,
                  rec=([o + 10], [o + 45]))
        out.append(oracle.acoustic_forward(g, np.full((n, n), 2000.0), stf,
                                           [[(o + 15) * dx, (o + 12) * dx]])[0, 0])
    diff = np.abs(out[0] - out[1]).max()
    assert diff <= 1e-2 * np.abs(out[1]).max(), diff / np.abs(out[1]).max()


# ---------------------------------------------------------------- adjoint
@pytest.mark.parametrize("order,npml,kind", [(4, 6, 0), (8, 5, 1)])
def test_dot_product_source_map(order, npml, kind):
    # seismograms are linear in the source time function: <F s, r> = <s, F^T r>
    g = _geom(16, 20, 90, order=order, npml=npml, src_kind=kind, rec=([2, 9, 13], [3, 17, 8]))
    rng = np.random.default_rng(3)
    c = 2000 + 400 * rng.random((16, 20))
    x0 = np.array([[93.0, 71.0], [52.0, 104.0]])
    s = rng.standard_normal((2, 90))
    r = rng.standard_normal((2, 3, 90))
    Fs = oracle.acoustic_forward(g, c, s, x0)
    _, FTr, _ = oracle.acoustic_adjoint(g, c, s, x0, r)
    lhs, rhs = np.sum(Fs * r), np.sum(s * FTr)
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs)), (lhs, rhs)


@pytest.mark.parametrize("order,npml", [(4, 6), (8, 8)])
def test_dot_product_model_tangent(order, npml):
    # J = d seis / d c from the complex step, J^T from the adjoint:
    # <J dc, r> = <dc, J^T r> to rounding.
    g = _geom(14, 18, 80, order=order, npml=npml, rec=([1, 7, 12], [2, 15, 9]))
    rng = np.random.default_rng(4)
    c = 2000 + 400 * rng.random((14, 18))
    x0 = np.array([[85.0, 64.0]])
    s = synth.ricker(20.0, 1e-3, 80, dtype=np.float64)[None]
    dc = rng.standard_normal((14, 18))
    r = rng.standard_normal((1, 3, 80))
    h = 1e-30
    Jdc = oracle.acoustic_forward(g, c + 1j * h * dc, s, x0, complex_step=True).imag / h
    JTr, _, _ = oracle.acoustic_adjoint(g, c, s, x0, r)
    lhs, rhs = np.sum(Jdc * r), np.sum(dc * JTr)
    assert abs(lhs - rhs) <= 1e-11 * max(abs(lhs), abs(rhs)), (lhs, rhs)


def _misfit(g, c, s, x0, obs, cs=False):
    d = oracle.acoustic_forward(g, c, s, x0, complex_step=cs)
    r = d - obs
    return 0.5 * np.sum(r * r)


def test_gradient_vs_complex_step_and_fd():
    # tiny grid 24 x 32 + 8 CPML, 150 steps, 2 shots; cells include a CPML-edge
    # cell, a source cell and a receiver cell.
    g = _geom(24, 32, 150, order=4, npml=8, rec=([0, 3, 20, 23], [0, 16, 30, 5]))
    rng = np.random.default_rng(5)
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
    eps = 1e-3
    fd = (_misfit(g, c + eps * dirn, s, x0, obs) - _misfit(g, c - eps * dirn, s, x0, obs)) / (2 * eps)
    assert np.sum(gc * dirn) == pytest.approx(fd, rel=1e-6)
    # source time function
    ds = rng.standard_normal(s.shape)
    cs = _misfit(g, c, s + 1j * h * ds, x0, obs, cs=True).imag / h
    assert np.sum(gs * ds) == pytest.approx(cs, rel=1e-10)


def test_zero_residual_zero_gradient():
    g = _geom(12, 14, 60, npml=4)
    c = np.full((12, 14), 2100.0)
    x0 = np.array([[60.0, 50.0]])
    s = synth.ricker(20.0, 1e-3, 60, dtype=np.float64)[None]
    obs = oracle.acoustic_forward(g, c, s, x0)
    J, gc, gs, gx = oracle.acoustic_misfit_grad(g, c, s, x0, obs)
    assert J == 0 and np.all(gc == 0) and np.all(gs == 0) and np.all(gx == 0)


def test_gaussian_source_location_gradient():
    # Gaussian re-parameterisation of the point source makes x0 differentiable.
    g = _geom(20, 22, 120, order=8, npml=6, src_kind=1, rec=([0, 10, 19], [0, 21, 11]))
    rng = np.random.default_rng(6)
    c = 2000 + 300 * rng.random((20, 22))
    s = synth.ricker(18.0, 1e-3, 120, dtype=np.float64)[None]
    x_true = np.array([[101.3, 87.7]])
    x0 = np.array([[107.9, 82.2]])
    obs = oracle.acoustic_forward(g, c, s, x_true)
    J, _, gs, gx = oracle.acoustic_misfit_grad(g, c, s, x0, obs)
    h = 1e-30
    for k in range(2):
        e = np.zeros((1, 2))
        e[0, k] = 1.0
        cs = _misfit(g, c, s, x0 + 1j * h * e, obs, cs=True).imag / h
        assert gx[0, k] == pytest.approx(cs, rel=1e-9)
    # the Gaussian weights sum to about 1 / (dx dz) (sigma = dx / 2)
    assert J > 0
