"""Source inversions (earthquake location and time function; rupture imaging)
on the GPU path, against the FP64 oracle.

The superposed-source misfit of a rupture is checked against the oracle's own
forward map (sum of the sub-source seismograms) and its adjoint applied to the
common residual; the Gaussian-slip parametrisation against the chain rule of
the oracle's time-function gradient; the location inversion by recovering a
known source from its synthetic waveforms."""

import numpy as np
import pytest

import oracle
from paper_2003_06027_gb300 import synth

pytestmark = pytest.mark.gpu

SEIS_TOL = 1e-4
GRAD_TOL = 1e-3


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _geom(d):
    return dict(nz=d["nz"], nx=d["nx"], npml=d["npml"], order=d["order"], nt=d["nt"], dz=d["dz"],
                dx=d["dx"], dt=d["dt"], src_kind=d["src_kind"], pml_R=d["pml_R"], pml_vmax=d["pml_vmax"],
                pml_f0=d["pml_f0"], rec_iz=d["rec_iz"], rec_ix=d["rec_ix"])


def _cuda(x, grad=False):
    import torch

    t = torch.as_tensor(np.ascontiguousarray(x)).cuda()
    return t.requires_grad_(True) if grad else t


def _rupture(seed=61, k=4, nz=40, nx=64, nt=180):
    """k Gaussian sub-sources along a horizontal fault at depth, switched on
    from left to right with different delays and amplitudes."""
    d = synth.random_acoustic(seed, nz, nx, nt, k, 8, 8, src_kind=1, nrec=12)
    d["x0"] = np.stack([np.linspace(150.0, 480.0, k), np.full(k, 300.0)], 1).astype(np.float32)
    d["rec_iz"] = np.zeros(12, np.int32) + 2
    d["rec_ix"] = np.linspace(2, nx - 3, 12).astype(np.int32)
    return d


def test_superposed_misfit_matches_oracle(fwi_lib):
    from paper_2003_06027_gb300 import fwi
    from paper_2003_06027_gb300.apps import superposed_misfit

    d = _rupture()
    g = _geom(d)
    c64, stf64, x064 = np.float64(d["c"]), np.float64(d["stf"]), np.float64(d["x0"])
    each = oracle.acoustic_forward(g, c64, stf64, x064)
    rng = np.random.default_rng(3)
    obs = (each.sum(0) * 0.7 + rng.standard_normal(each.shape[1:]) * np.abs(each).max() * 0.05).astype(np.float32)
    r = each.sum(0) - obs
    Jo = 0.5 * float(np.sum(r * r))
    _, gso, gxo = oracle.acoustic_adjoint(g, c64, stf64, x064, np.broadcast_to(r, each.shape))
    stf, x0 = _cuda(d["stf"], True), _cuda(d["x0"], True)
    J = superposed_misfit(stf, x0, _cuda(d["c"]), _cuda(obs), _cuda(d["rec_iz"]), _cuda(d["rec_ix"]),
                          ckpt_every=50, **fwi.problem_kwargs(d))
    J.backward()
    assert abs(float(J.detach()) - Jo) <= SEIS_TOL * Jo
    assert rel(stf.grad.cpu().numpy(), gso) <= GRAD_TOL, rel(stf.grad.cpu().numpy(), gso)
    assert rel(x0.grad.cpu().numpy(), gxo) <= GRAD_TOL, rel(x0.grad.cpu().numpy(), gxo)


def test_gaussian_slip_gradient(fwi_lib):
    """dJ/dA_k and dJ/dt0_k through the Gaussian slip g_k(t) = A_k exp(-(t - t0_k)^2 / 2s^2)."""
    import torch

    from paper_2003_06027_gb300 import fwi
    from paper_2003_06027_gb300.apps import gaussian_slip, superposed_misfit

    d = _rupture(seed=62)
    k, nt, dt = 4, d["nt"], d["dt"]
    sig = 8 * dt
    A_t, t_t = np.array([1.0, 0.6, 1.3, 0.8]), np.array([0.03, 0.045, 0.06, 0.075])
    tt = np.arange(nt) * dt
    slip = lambda A, t0: A[:, None] * np.exp(-((tt[None] - t0[:, None]) ** 2) / (2 * sig * sig))
    g = _geom(d)
    c64, x064 = np.float64(d["c"]), np.float64(d["x0"])
    obs = oracle.acoustic_forward(g, c64, slip(A_t, t_t), x064).sum(0).astype(np.float32)
    A0, t00 = np.full(k, 0.9), np.full(k, 0.05)
    each = oracle.acoustic_forward(g, c64, slip(A0, t00), x064)
    r = each.sum(0) - obs
    _, gso, _ = oracle.acoustic_adjoint(g, c64, slip(A0, t00), x064, np.broadcast_to(r, each.shape))
    e = np.exp(-((tt[None] - t00[:, None]) ** 2) / (2 * sig * sig))
    want_A = np.sum(gso * e, 1)
    want_t = np.sum(gso * A0[:, None] * e * (tt[None] - t00[:, None]) / (sig * sig), 1)
    A = torch.tensor(A0, dtype=torch.float32, device="cuda", requires_grad=True)
    t0 = torch.tensor(t00, dtype=torch.float32, device="cuda", requires_grad=True)
    J = superposed_misfit(gaussian_slip(A, t0, sig, nt, dt), _cuda(d["x0"]), _cuda(d["c"]), _cuda(obs),
                          _cuda(d["rec_iz"]), _cuda(d["rec_ix"]), **fwi.problem_kwargs(d))
    J.backward()
    assert rel(A.grad.cpu().numpy(), want_A) <= GRAD_TOL
    assert rel(t0.grad.cpu().numpy(), want_t) <= GRAD_TOL


def test_locate_source_recovers_location_and_time_function(fwi_lib):
    """Joint location / time-function inversion from a displaced start and a
    zero time function recovers the true source."""
    from paper_2003_06027_gb300 import fwi
    from paper_2003_06027_gb300.apps import locate_source

    nz, nx, nt, dx, dt = 50, 70, 300, 10.0, 1e-3
    d = synth.random_acoustic(71, nz, nx, nt, 1, 8, 10, src_kind=1, nrec=1)
    d["rec_iz"] = np.array([2] * 10 + [nz - 3] * 10 + list(range(5, nz - 5, 8)), np.int32)
    d["rec_ix"] = np.array(list(np.linspace(3, nx - 4, 10, dtype=int)) * 2 + [nx - 3] * len(range(5, nz - 5, 8)),
                           np.int32)
    x_true = np.array([[352.0, 241.0]], np.float32)
    obs = fwi.forward(_cuda(d["c"]), _cuda(d["stf"]), _cuda(x_true), _cuda(d["rec_iz"]), _cuda(d["rec_ix"]),
                      **fwi.problem_kwargs(d))
    start = x_true + np.array([[32.0, -27.0]], np.float32)
    out = locate_source(_cuda(d["c"]), obs, _cuda(d["rec_iz"]), _cuda(d["rec_ix"]), start, nt=nt, dx=dx, dz=dx,
                        dt=dt, iters=300, lr_stf=0.01, order=8, npml=10, pml_R=d["pml_R"],
                        pml_vmax=d["pml_vmax"], pml_f0=d["pml_f0"])
    err = np.linalg.norm(out.x0.cpu().numpy() - x_true)
    assert err < 0.25 * dx, (err, out.path[-1])
    assert out.misfit[-1] < 1e-3 * out.misfit[0]
    # the time function is fixed by the data only inside their frequency band
    assert rel(out.stf.cpu().numpy(), d["stf"]) < 0.15


def test_plane_wave_fwi_with_lbfgs(fwi_lib):
    """The paper's plane-wave FWI setting in miniature: four plane waves from the
    bottom (line sources), surface receivers, L-BFGS on the exact gradient from
    the layered model without its anomaly. The misfit falls at least fourfold
    and the model moves towards the anomaly."""
    import torch

    from paper_2003_06027_gb300 import fwi
    from paper_2003_06027_gb300.optim import lbfgs

    d = synth.plane_wave_survey()
    kw = fwi.problem_kwargs(d)
    stf, x0, iz, ix = _cuda(d["stf"]), _cuda(d["x0"]), _cuda(d["rec_iz"]), _cuda(d["rec_ix"])
    obs = fwi.forward(_cuda(d["c_true"]), stf, x0, iz, ix, **kw)

    def fun_grad(c):
        J, g, _, _, _ = fwi.misfit_grad(c, stf, x0, iz, ix, obs, ckpt_every=100, want_src=False, **kw)
        return float(J[0]), g

    c0 = _cuda(d["c"])
    c, log = lbfgs(fun_grad, c0, 12, step0=30.0, lower=1500.0, upper=4500.0)
    assert log.f[-1] < 0.25 * log.f[0], log.f
    err0 = float(torch.linalg.vector_norm(c0 - _cuda(d["c_true"])))
    err1 = float(torch.linalg.vector_norm(c - _cuda(d["c_true"])))
    assert err1 < err0, (err0, err1)
