"""The seeded synthetic inputs against the workloads they stand in for (CPU):
sizes, discretisation, value ranges and structure of each generator, its
seeding, and the stability (CFL) of the explicit schemes on it."""

import numpy as np
import pytest

from paper_2003_06027_gb300 import synth

# staggered-grid weights (Taylor moment conditions): sum |a_k| bounds the
# spatial operator in the CFL condition c dt sqrt(1/dx^2 + 1/dz^2) sum|a_k| <= 1
SUM_ABS = {4: 9 / 8 + 1 / 24, 8: 1225 / 1024 + 245 / 3072 + 49 / 5120 + 5 / 7168}


def _cfl(vmax, d):
    return vmax * d["dt"] * np.sqrt(1 / d["dx"] ** 2 + 1 / d["dz"] ** 2) * SUM_ABS[d["order"]]


def test_ricker():
    f0, dt, nt = 10.0, 1e-3, 500
    r = synth.ricker(f0, dt, nt)
    assert r.dtype == np.float32 and r.shape == (nt,)
    assert np.argmax(r) == round(1.2 / f0 / dt) and r.max() == pytest.approx(1.0)
    assert abs(float(r.astype(np.float64).sum()) * dt) < 1e-6  # zero mean: the second derivative of a Gaussian


def test_two_layer_problem():
    d, dp = synth.acoustic_small(), synth.acoustic_small(perturbed=True)
    assert d["c"].shape == (100, 100) and d["nt"] == 500 and d["order"] == 4 and d["npml"] == 20
    assert (d["c"][:50] == 2000).all() and (d["c"][50:] == 3000).all()  # interface at 500 m
    assert (dp["c"][:52] == 2000).all() and (dp["c"][52:] == 3000).all()  # observed: at 520 m
    assert list(d["rec_ix"]) == list(range(1, 100, 2)) and (d["rec_iz"] == 5).all()
    assert _cfl(3000.0, d) < 1


def test_fwi_workload():
    d = synth.acoustic_fwi()
    assert d["c"].shape == (201, 601) and d["stf"].shape == (16, 3000)
    assert (d["dx"], d["dt"], d["order"], d["npml"], d["ckpt_every"]) == (10.0, 0.8e-3, 8, 32, 100)
    assert len(d["rec_ix"]) == 301 and list(d["rec_ix"][:3]) == [0, 2, 4] and (d["rec_iz"] == 2).all()
    t = d["c_true"]
    assert t.min() >= 1500 and t.max() <= 4500
    # velocity increases with depth on average, and the start model is a smoothing of the true one
    rows = t.mean(axis=1)
    assert rows[-1] > rows[0] + 1500
    assert np.abs(np.diff(d["c"], axis=0)).max() < np.abs(np.diff(t, axis=0)).max() / 5
    assert abs(float(d["c"].mean()) - float(t.mean())) < 20
    assert np.allclose(d["x0"][:, 1], 20.0) and d["x0"][0, 0] == 0 and d["x0"][-1, 0] == pytest.approx(6000.0)
    assert _cfl(4500.0, d) < 1
    again = synth.acoustic_fwi()
    assert np.array_equal(again["c_true"], t) and np.array_equal(again["c"], d["c"])
    other = synth.acoustic_fwi(seed=2004)
    assert not np.array_equal(other["c_true"], t)


def test_elastic_workload():
    d = synth.elastic_layered()
    assert d["vp"].shape == (300, 800) and d["stf"].shape == (32, 4000)
    assert (d["dx"], d["dt"], d["order"], d["npml"]) == (5.0, 0.5e-3, 4, 32)
    assert d["vp"].min() >= 1800 and d["vp"].max() <= 4500
    np.testing.assert_allclose(d["vs"], d["vp"] / 1.73, rtol=1e-6)
    np.testing.assert_allclose(d["rho"], 310.0 * d["vp"].astype(np.float64) ** 0.25, rtol=1e-5)  # Gardner
    z = d["x0"][:, 1]
    assert z.min() >= 400 and z.max() <= 1200
    mt = d["mt"].astype(np.float64) / synth.MOMENT_SCALE  # double couple (Mxx, Mzz, Mxz) = (-sin 2p, sin 2p, cos 2p)
    np.testing.assert_allclose(mt[:, 0], -mt[:, 1], rtol=1e-6)
    np.testing.assert_allclose(mt[:, 0] ** 2 + mt[:, 2] ** 2, 1.0, rtol=1e-5)
    assert len(d["rec_ix"]) == 200 and list(d["rec_ix"][:2]) == [0, 4]
    assert _cfl(4500.0, d) < 1


def test_uneven_instances():
    seen = []
    for i in range(16):
        d = synth.uneven_instance(4, i)
        nz, nx, nt, S = d["nz"], d["nx"], d["nt"], d["stf"].shape[0]
        assert 128 <= nz <= 512 and nz % 32 == 0
        assert 128 <= nx <= 1024 and nx % 32 == 0
        assert 1000 <= nt <= 4000 and nt % 100 == 0
        assert 4 <= S <= 16
        assert (d["order"], d["npml"], d["dx"], d["dt"]) == (8, 32, 10.0, 0.8e-3)
        assert _cfl(float(d["c_true"].max()), d) < 1
        seen.append((nz, nx, nt, S))
    assert len(set(seen)) == len(seen)  # distinct instances
    assert synth.uneven_instance(4, 3)["c"].tobytes() == synth.uneven_instance(4, 3)["c"].tobytes()


def test_plane_wave_delays():
    dt, nt, dx, c = 1e-3, 400, 10.0, 2000.0
    w = synth.ricker(12.0, dt, nt)
    flat = synth.plane_wave(w, dt, 0.0, c, 9, dx)
    assert flat.shape == (nt, 9)
    for q in range(9):
        np.testing.assert_allclose(flat[:, q], w, atol=1e-7)  # vertical incidence: all cells fire together
    # one sample of delay per cell when dx sin(theta) / c = dt (theta = 11.5 degrees here)
    th = np.degrees(np.arcsin(dt * c / dx))
    st = synth.plane_wave(w, dt, th, c, 5, dx)
    for q in range(5):
        np.testing.assert_allclose(st[q:, q], w[: nt - q], atol=1e-6)
        assert np.all(st[:q, q] == 0)
    back = synth.plane_wave(w, dt, -th, c, 5, dx)  # the other side fires first
    np.testing.assert_allclose(back[:, 4], w, atol=1e-6)
