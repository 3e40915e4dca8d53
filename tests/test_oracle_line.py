"""Pins of the oracle's line source (the paper's plane-wave sources: a line of
cells along one row, each firing its own time function): the response is the
sum of the point-source responses of its cells (superposition, against the
oracle's point-source path, itself pinned by the analytic Green's function);
its adjoint passes the dot-product test; the model gradient with a line source
matches complex-step derivatives; the plane-wave time functions are delayed
copies of the wavelet."""

import numpy as np

import oracle
from paper_2003_06027_gb300 import synth


def _g(d):
    return {k: d[k] for k in ("nz", "nx", "npml", "order", "nt", "dz", "dx", "dt", "src_kind", "pml_R",
                              "pml_vmax", "pml_f0", "rec_iz", "rec_ix", "line_len")}


def test_line_source_is_the_sum_of_its_point_sources():
    d = synth.line_source_problem(11, 20, 26, 90, 2, 4, 6, line_len=9)
    g = _g(d)
    seis = oracle.acoustic_forward(g, np.float64(d["c"]), np.float64(d["stf"]), np.float64(d["x0"]))
    gp = dict(g, src_kind=0)
    for s in range(2):
        want = np.zeros_like(seis[s])
        for q in range(d["line_len"]):
            xq = np.array([[d["x0"][s, 0] + q * d["dx"], d["x0"][s, 1]]])
            want += oracle.acoustic_forward(gp, np.float64(d["c"]), np.float64(d["stf"][s, :, q])[None], xq)[0]
        assert np.linalg.norm(seis[s] - want) <= 1e-12 * np.linalg.norm(want)
    assert np.abs(seis).max() > 0


def test_line_source_dot_product():
    """<F a, r> = <a, F^T r> for the map from the per-cell time functions a to
    the seismograms (F^T r is the oracle's source gradient for residual r)."""
    d = synth.line_source_problem(12, 18, 24, 80, 2, 8, 5, line_len=7)
    g = _g(d)
    rng = np.random.default_rng(5)
    a = rng.standard_normal(d["stf"].shape)
    Fa = oracle.acoustic_forward(g, np.float64(d["c"]), a, np.float64(d["x0"]))
    r = rng.standard_normal(Fa.shape)
    _, FTr, _ = oracle.acoustic_adjoint(g, np.float64(d["c"]), a, np.float64(d["x0"]), r)
    lhs, rhs = float(np.sum(Fa * r)), float(np.sum(a * FTr))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs))


def test_line_source_model_gradient_vs_complex_step():
    d = synth.line_source_problem(13, 16, 22, 70, 2, 4, 5, line_len=6)
    g = _g(d)
    c = np.float64(d["c"])
    obs = oracle.acoustic_forward(g, c * 1.02, np.float64(d["stf"]), np.float64(d["x0"]))
    J, gc, gs, _ = oracle.acoustic_misfit_grad(g, c, np.float64(d["stf"]), np.float64(d["x0"]), obs)
    assert gs.shape == d["stf"].shape
    rng = np.random.default_rng(9)
    dirn = rng.standard_normal(c.shape)
    h = 1e-20
    sc = oracle.acoustic_forward(g, c + 1j * h * dirn, np.complex128(d["stf"]), np.complex128(d["x0"]),
                                 complex_step=True)
    dJ = float(np.sum((sc.real - obs) * sc.imag / h))
    gd = float(np.sum(gc * dirn))
    assert abs(gd - dJ) <= 1e-10 * abs(dJ), (gd, dJ)


def test_plane_wave_delays():
    dt, dx = 1e-3, 10.0
    wav = synth.ricker(15.0, dt, 200)
    flat = synth.plane_wave(wav, dt, 0.0, 2000.0, 5, dx)
    assert all(np.array_equal(flat[:, q], wav) for q in range(5))
    # sin(theta) dx / c = 1 ms per cell: cell q is the wavelet q samples later
    th = np.degrees(np.arcsin(2000.0 * dt / dx))
    pw = synth.plane_wave(wav, dt, th, 2000.0, 5, dx)
    for q in range(5):
        np.testing.assert_allclose(pw[q:, q], wav[: 200 - q], atol=1e-6)
        assert np.all(pw[:q, q] == 0)
    neg = synth.plane_wave(wav, dt, -th, 2000.0, 5, dx)  # the far end fires first
    np.testing.assert_allclose(neg[:, 4], wav, atol=1e-6)
