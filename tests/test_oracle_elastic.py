"""Pins of the FP64 elastic oracle against facts fixed outside it:
  * with mu = 0 in a homogeneous medium the velocity-stress scheme is
    algebraically the acoustic divergence scheme (CPML included) with the
    source time function differenced: exact agreement with the (separately
    pinned) acoustic oracle;
  * with a rigid boundary and no source the staggered leapfrog conserves
    1/2 <sigma, C^-1 sigma> + 1/2 <rho v^{n-1/2}, v^{n+1/2}> exactly (this
    tests the stress-velocity coupling, the buoyancy average and the shear
    modulus average);
  * x <-> z transposition symmetry;
  * dot-product adjoint tests and complex-step gradients for lambda, mu, rho,
    the source time function and the Gaussian source position.
CPU only."""

import numpy as np
import pytest

import oracle
from paper_2003_06027_gb300 import synth


def _geom(nz, nx, nt, order=4, npml=8, dx=10.0, dt=1e-3, src_kind=0, rec=None, f0=15.0):
    rec = rec if rec is not None else ([nz // 3, nz - 2], [nx // 4, nx - 3])
    return dict(nz=nz, nx=nx, npml=npml, order=order, nt=nt, dz=dx, dx=dx, dt=dt, src_kind=src_kind,
                pml_R=1e-3, pml_vmax=4500.0, pml_f0=f0,
                rec_iz=np.asarray(rec[0], np.int32), rec_ix=np.asarray(rec[1], np.int32))


def _medium(seed, nz, nx):
    rng = np.random.default_rng(seed)
    vp = synth.smooth((2600 + 600 * rng.random((nz, nx))).astype(np.float32), 1.5).astype(np.float64)
    vs = vp / (1.6 + 0.3 * rng.random((nz, nx)))
    rho = 310.0 * vp ** 0.25 * (1 + 0.1 * rng.random((nz, nx)))
    return vp, vs, rho


@pytest.mark.parametrize("order,npml", [(4, 10), (8, 6)])
def test_fluid_limit_equals_acoustic_scheme(order, npml):
    # mu = 0, homogeneous: sxx = szz = P obeys P^{n+1} - 2P^n + P^{n-1} =
    # dt^2 lambda D-(b D+ P^n) (+ CPML) - dt w (g_n - g_{n-1}), i.e. the
    # acoustic recursion with c^2 = lambda/rho and f_n = -(g_n - g_{n-1})/dt.
    nz, nx, nt = 26, 30, 90
    g = _geom(nz, nx, nt, order=order, npml=npml, src_kind=1)
    vp = np.full((nz, nx), 2400.0)
    vs = np.zeros((nz, nx))
    rho = np.full((nz, nx), 1900.0)
    stf = synth.ricker(25.0, 1e-3, nt, dtype=np.float64)[None]
    x0 = np.array([[143.0, 121.0]])
    mt = np.array([[1.0, 1.0, 0.0]])
    cells = [(3, 4), (12, 15), (20, 27), (0, 0), (25, 29)]
    ga = dict(g, rec_iz=np.array([c[0] for c in cells], np.int32), rec_ix=np.array([c[1] for c in cells], np.int32))
    f = -np.diff(np.concatenate([[0.0], stf[0]])) / g["dt"]
    ua = oracle.acoustic_forward(ga, vp, f[None], x0)[0]  # sample n-1 holds u^n
    scale = np.abs(ua).max()
    assert scale > 0
    for step in (25, 60, 89):
        F = oracle.elastic_snapshot(g, vp, vs, rho, stf, x0, mt, step)
        sxx, szz, sxz = F[2], F[3], F[4]
        np.testing.assert_allclose(sxx, szz, rtol=0, atol=1e-13 * scale)
        assert np.all(sxz == 0)
        for k, (i, j) in enumerate(cells):
            assert abs(sxx[i + npml, j + npml] - ua[k, step - 1]) <= 1e-11 * scale


def _energy(F_lo, F_hi, vp, vs, rho):
    """Discrete energy at step n from the state after n steps (F_lo) and after
    n+1 steps (F_hi, for v^{n+1/2}); rigid boundary, no padding."""
    vx0, vz0, sxx, szz, sxz = F_lo
    vx1, vz1 = F_hi[0], F_hi[1]
    mu = rho * vs * vs
    lam = rho * vp * vp - 2 * mu
    rx = 0.5 * (rho[:, :-1] + rho[:, 1:])
    rz = 0.5 * (rho[:-1, :] + rho[1:, :])
    E = 0.5 * np.sum(rx * vx0[:, :-1] * vx1[:, :-1]) + 0.5 * np.sum(rz * vz0[:-1, :] * vz1[:-1, :])
    det = 4 * mu * (lam + mu)
    E += 0.5 * np.sum(((lam + 2 * mu) * (sxx * sxx + szz * szz) - 2 * lam * sxx * szz) / det)
    mxz = 4.0 / (1 / mu[:-1, :-1] + 1 / mu[1:, :-1] + 1 / mu[:-1, 1:] + 1 / mu[1:, 1:])
    E += 0.5 * np.sum(sxz[:-1, :-1] ** 2 / mxz)
    return E


@pytest.mark.parametrize("order", [4, 8])
def test_energy_conservation_rigid_boundary(order):
    nz, nx, nt = 24, 28, 160
    g = _geom(nz, nx, nt, order=order, npml=0, src_kind=1, dt=5e-4)
    vp, vs, rho = _medium(3, nz, nx)
    stf = np.zeros((1, nt))
    stf[0, :20] = np.sin(np.pi * np.arange(20) / 20.0) ** 2  # source off after 20 steps
    x0 = np.array([[131.0, 117.0]])
    mt = np.array([[0.7, -0.4, 0.9]])
    Es = []
    for n in (40, 90, 150):
        Es.append(_energy(oracle.elastic_snapshot(g, vp, vs, rho, stf, x0, mt, n),
                          oracle.elastic_snapshot(g, vp, vs, rho, stf, x0, mt, n + 1), vp, vs, rho))
    assert Es[0] > 0
    np.testing.assert_allclose(Es, Es[0], rtol=1e-11)


def test_energy_is_not_conserved_by_a_wrong_average():
    # the energy test has teeth: with an arithmetic instead of harmonic shear
    # modulus average in the energy, conservation fails
    nz, nx, nt = 20, 20, 120
    g = _geom(nz, nx, nt, npml=0, src_kind=1, dt=5e-4)
    vp, vs, rho = _medium(4, nz, nx)
    stf = np.zeros((1, nt))
    stf[0, :20] = np.sin(np.pi * np.arange(20) / 20.0) ** 2
    x0, mt = np.array([[95.0, 97.0]]), np.array([[0.3, 0.2, 1.0]])

    def E(n, vs_e):
        return _energy(oracle.elastic_snapshot(g, vp, vs, rho, stf, x0, mt, n),
                       oracle.elastic_snapshot(g, vp, vs, rho, stf, x0, mt, n + 1), vp, vs_e, rho)

    vs_bad = vs * (1 + 0.05 * np.random.default_rng(0).standard_normal(vs.shape))
    assert abs(E(60, vs_bad) - E(110, vs_bad)) > 1e-6 * abs(E(60, vs_bad))


def test_transposition_symmetry():
    n, nt = 24, 120
    rng = np.random.default_rng(5)
    base = synth.smooth((2600 + 500 * rng.random((n, n))).astype(np.float32), 1.0).astype(np.float64)
    vp = 0.5 * (base + base.T)
    vs = vp / 1.7
    rho = 310 * vp ** 0.25
    rec = ([3, 17, 9, 9], [17, 3, 20, 20])
    g = _geom(n, n, nt, order=8, npml=7, src_kind=1, rec=rec)
    stf = synth.ricker(25.0, 1e-3, nt, dtype=np.float64)[None]
    x0 = np.array([[113.0, 113.0]])
    mt = np.array([[0.8, 0.8, 0.45]])
    d = oracle.elastic_forward(g, vp, vs, rho, stf, x0, mt)[0]
    scale = np.abs(d).max()
    # vx at receiver (3, 17) equals vz at receiver (17, 3) and vice versa
    np.testing.assert_allclose(d[0, 0], d[1, 1], rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(d[1, 0], d[0, 1], rtol=0, atol=1e-12 * scale)


def test_dot_product_source_map():
    g = _geom(18, 22, 80, order=4, npml=6, src_kind=1, rec=([2, 9, 15], [3, 18, 10]))
    vp, vs, rho = _medium(6, 18, 22)
    rng = np.random.default_rng(6)
    x0 = np.array([[103.0, 87.0], [121.0, 66.0]])
    mt = np.array([[1.0, 0.3, -0.5], [0.2, 0.9, 0.4]])
    s = rng.standard_normal((2, 80))
    r = rng.standard_normal((2, 2, 3, 80))
    Fs = oracle.elastic_forward(g, vp, vs, rho, s, x0, mt)
    FTr = oracle.elastic_adjoint(g, vp, vs, rho, s, x0, mt, r)[3]
    lhs, rhs = np.sum(Fs * r), np.sum(s * FTr)
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs)), (lhs, rhs)


def _to_vel(lam, mu, rho):
    return np.sqrt((lam + 2 * mu) / rho), np.sqrt(mu / rho), rho


def _J(g, lam, mu, rho, stf, x0, mt, obs, cs=False):
    vp, vs, rh = _to_vel(lam, mu, rho)
    d = oracle.elastic_forward(g, vp, vs, rh, stf, x0, mt, complex_step=cs)
    r = d - obs
    return 0.5 * np.sum(r * r)


@pytest.mark.parametrize("order,npml,kind", [(4, 6, 0), (8, 5, 1)])
def test_gradients_vs_complex_step(order, npml, kind):
    nz, nx, nt = 16, 20, 110
    g = _geom(nz, nx, nt, order=order, npml=npml, src_kind=kind, rec=([0, 4, 15, 9], [0, 17, 5, 19]))
    vp, vs, rho = _medium(7, nz, nx)
    lam, mu = rho * (vp ** 2 - 2 * vs ** 2), rho * vs ** 2
    x0 = np.array([[93.7, 78.2]])
    mt = np.array([[0.6, -0.8, 0.5]])
    stf = synth.ricker(22.0, 1e-3, nt, dtype=np.float64)[None]
    vp_t, vs_t, rho_t = _medium(8, nz, nx)
    obs = oracle.elastic_forward(g, vp_t, vs_t, rho_t, stf, x0, mt)
    J, gl, gm, gr, gs, gx = oracle.elastic_misfit_grad(g, vp, vs, rho, stf, x0, mt, obs)
    assert J > 0
    h = 1e-30
    rng = np.random.default_rng(9)
    cells = [(0, 0), (15, 19), (7, 9), (0, 10), (4, 17)]
    for name, grad, base in (("lam", gl, lam), ("mu", gm, mu), ("rho", gr, rho)):
        for (i, j) in cells:
            e = np.zeros((nz, nx))
            e[i, j] = base[i, j]
            args = [lam, mu, rho]
            k = ("lam", "mu", "rho").index(name)
            args = [a + 1j * h * e if q == k else a.astype(np.complex128) for q, a in enumerate(args)]
            cs = _J(g, *args, stf, x0, mt, obs, cs=True).imag / h
            assert grad[i, j] * base[i, j] == pytest.approx(cs, rel=1e-9, abs=1e-9 * np.abs(grad * base).max()), (name, i, j)
        dirn = rng.standard_normal((nz, nx)) * base
        k = ("lam", "mu", "rho").index(name)
        args = [a + 1j * h * dirn if q == k else a.astype(np.complex128) for q, a in enumerate([lam, mu, rho])]
        cs = _J(g, *args, stf, x0, mt, obs, cs=True).imag / h
        assert np.sum(grad * dirn) == pytest.approx(cs, rel=1e-9), name
    ds = rng.standard_normal(stf.shape)
    cs = _J(g, lam + 0j, mu + 0j, rho + 0j, stf + 1j * h * ds, x0, mt, obs, cs=True).imag / h
    assert np.sum(gs * ds) == pytest.approx(cs, rel=1e-9)
    if kind == 1:
        for q in range(2):
            e = np.zeros((1, 2))
            e[0, q] = 1.0
            cs = _J(g, lam + 0j, mu + 0j, rho + 0j, stf, x0 + 1j * h * e, mt, obs, cs=True).imag / h
            assert gx[0, q] == pytest.approx(cs, rel=1e-8)
    else:
        assert np.all(gx == 0)


def test_zero_residual_zero_gradient():
    g = _geom(12, 14, 50, npml=4)
    vp, vs, rho = _medium(10, 12, 14)
    x0, mt = np.array([[60.0, 50.0]]), np.array([[1.0, 1.0, 0.0]])
    stf = synth.ricker(25.0, 1e-3, 50, dtype=np.float64)[None]
    obs = oracle.elastic_forward(g, vp, vs, rho, stf, x0, mt)
    J, gl, gm, gr, gs, gx = oracle.elastic_misfit_grad(g, vp, vs, rho, stf, x0, mt, obs)
    assert J == 0 and not np.any(gl) and not np.any(gm) and not np.any(gr) and not np.any(gs)


def test_velocity_gradient_vs_complex_step():
    """The chain rule to (vp, vs, rho) against complex-step derivatives taken in
    the velocity parametrisation itself (the oracle forward is evaluated with a
    complex vp, vs or rho, so lambda and mu carry the perturbation through the
    medium set-up of the scheme)."""
    nz, nx, nt = 14, 18, 100
    g = _geom(nz, nx, nt, order=4, npml=5, src_kind=1, rec=([0, 6, 13], [2, 17, 9]))
    vp, vs, rho = _medium(21, nz, nx)
    x0 = np.array([[81.3, 64.9]])
    mt = np.array([[0.3, -0.9, 0.7]])
    stf = synth.ricker(24.0, 1e-3, nt, dtype=np.float64)[None]
    obs = oracle.elastic_forward(g, *_medium(22, nz, nx), stf, x0, mt)
    J, gl, gm, gr, _, _ = oracle.elastic_misfit_grad(g, vp, vs, rho, stf, x0, mt, obs)
    gvp, gvs, grho = oracle.elastic_velocity_grad(vp, vs, rho, gl, gm, gr)
    h = 1e-30
    rng = np.random.default_rng(23)
    for k, grad in enumerate((gvp, gvs, grho)):
        dirn = rng.standard_normal((nz, nx)) * (vp, vs, rho)[k] * 1e-2
        args = [a.astype(np.complex128) for a in (vp, vs, rho)]
        args[k] = args[k] + 1j * h * dirn
        d = oracle.elastic_forward(g, *args, stf, x0, mt, complex_step=True)
        r = d - obs
        cs = (0.5 * np.sum(r * r)).imag / h
        assert np.sum(grad * dirn) == pytest.approx(cs, rel=1e-9), k
