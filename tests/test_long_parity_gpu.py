"""Parity at the configured time lengths: the 201 x 601 acoustic FWI gradient
at nt = 3000 (element by element, one shot) and the 300 x 800 elastic problem
at nt = 4000 (seismograms element by element for two moment-tensor shots; the
lambda, mu and rho gradients through directional derivatives against central
differences of the oracle's misfit). These runs show the FP32 accumulation over
thousands of steps on the device against the FP64 oracle.

The oracle runs take minutes; they are started together on host threads when
the module's first test asks for them (the oracle's C calls release the GIL),
so the whole file costs about as long as its slowest oracle run.
"""

from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from paper_2003_06027_gb300 import synth

pytestmark = pytest.mark.gpu

SEIS_TOL = 1e-4
GRAD_TOL = 1e-3
FD_REL = 1e-4  # central-difference step, relative to each parameter


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _geom(d):
    return dict(nz=d["nz"], nx=d["nx"], npml=d["npml"], order=d["order"], nt=d["nt"], dz=d["dz"],
                dx=d["dx"], dt=d["dt"], src_kind=d["src_kind"], pml_R=d["pml_R"], pml_vmax=d["pml_vmax"],
                pml_f0=d["pml_f0"], rec_iz=d["rec_iz"], rec_ix=d["rec_ix"])


def _cuda(x):
    import torch

    return torch.as_tensor(np.ascontiguousarray(x)).cuda()


def _acoustic():
    """One shot of the 201 x 601 FWI problem (the middle source), nt = 3000."""
    d = synth.acoustic_fwi(nshots=3, nt=3000)
    for k in ("stf", "x0"):
        d[k] = np.ascontiguousarray(d[k][1:2])
    return d


def _elastic():
    return synth.elastic_layered(nshots=2, nt=4000)


def _lame(vp, vs, rho):
    mu = rho * vs * vs
    return rho * vp * vp - 2.0 * mu, mu, rho


def _vel(lam, mu, rho):
    return np.sqrt((lam + 2.0 * mu) / rho), np.sqrt(mu / rho), rho


def _directions(d):
    """Smooth seeded perturbations of lambda, mu and rho (one per parameter),
    each relative to the parameter's own values."""
    rng = np.random.default_rng(4000)
    lam, mu, rho = _lame(*(np.float64(d[k]) for k in ("vp", "vs", "rho")))
    out = []
    for p in (lam, mu, rho):
        r = synth.smooth(rng.standard_normal(p.shape).astype(np.float32), 6.0).astype(np.float64)
        out.append(p * r / np.abs(r).max())
    return out


def _elastic_J(d, shot, lam, mu, rho):
    vp, vs, rh = _vel(lam, mu, rho)
    s = slice(shot, shot + 1)
    seis = oracle.elastic_forward(_geom(d), vp, vs, rh, np.float64(d["stf"][s]), np.float64(d["x0"][s]),
                                  np.float64(d["mt"][s]))
    return 0.5 * float(np.sum(seis * seis))  # observed data = 0: J = 1/2 |d|^2


@pytest.fixture(scope="module")
def oracle_runs():
    ex = ThreadPoolExecutor(max_workers=8)
    runs = {}
    da = _acoustic()
    ga = _geom(da)

    def acoustic_grad():
        obs = oracle.acoustic_forward(ga, np.float64(da["c_true"]), np.float64(da["stf"]), np.float64(da["x0"]))
        return obs, oracle.acoustic_misfit_grad(ga, np.float64(da["c"]), np.float64(da["stf"]),
                                                np.float64(da["x0"]), obs)

    runs["acoustic"] = ex.submit(acoustic_grad)
    de = _elastic()
    ins = [np.float64(de[k]) for k in ("vp", "vs", "rho", "stf", "x0", "mt")]
    runs["elastic_seis"] = ex.submit(oracle.elastic_forward, _geom(de), *ins)
    lam, mu, rho = _lame(*ins[:3])
    for k, dp in enumerate(_directions(de)):
        for sgn in (1, -1):
            p = [lam, mu, rho]
            p[k] = p[k] + sgn * FD_REL * dp
            runs[("elastic_J", k, sgn)] = ex.submit(_elastic_J, de, 0, *p)
    yield runs
    ex.shutdown(wait=True, cancel_futures=True)


def test_acoustic_fwi_gradient_elementwise_nt3000(fwi_lib, oracle_runs):
    from paper_2003_06027_gb300 import fwi

    d = _acoustic()
    kw = fwi.problem_kwargs(d)
    args = [_cuda(d[k]) for k in ("c", "stf", "x0", "rec_iz", "rec_ix")]
    obs_g = fwi.forward(_cuda(d["c_true"]), *args[1:], **kw)
    Jg, gg, gsg, _, _ = fwi.misfit_grad(*args, obs_g, ckpt_every=d["ckpt_every"], **kw)
    obs_o, (Jo, go, gso, _) = oracle_runs["acoustic"].result()
    e_obs = rel(obs_g.cpu().numpy(), obs_o)
    e_J = abs(float(Jg.cpu()[0]) - Jo) / Jo
    e_g = rel(gg.cpu().numpy(), go)
    e_s = rel(gsg.cpu().numpy(), gso)
    print(f"\nacoustic 201x601 nt=3000: observed {e_obs:.2e}, J {e_J:.2e}, grad {e_g:.2e}, grad_stf {e_s:.2e}")
    assert e_obs <= SEIS_TOL, e_obs
    assert e_J <= GRAD_TOL, e_J
    assert e_g <= GRAD_TOL, e_g
    assert e_s <= GRAD_TOL, e_s


def test_elastic_seismograms_elementwise_nt4000(fwi_lib, oracle_runs):
    from paper_2003_06027_gb300 import fwi

    d = _elastic()
    kw = fwi.problem_kwargs(d)
    dg = fwi.forward_elastic(*[_cuda(d[k]) for k in ("vp", "vs", "rho", "stf", "x0", "mt", "rec_iz", "rec_ix")],
                             **kw).cpu().numpy()
    do = oracle_runs["elastic_seis"].result()
    e = rel(dg, do)
    # the drift over time: error of the first and second halves of the record
    h = d["nt"] // 2
    e1, e2 = rel(dg[..., :h], do[..., :h]), rel(dg[..., h:], do[..., h:])
    print(f"\nelastic 300x800 nt=4000 seismograms: {e:.2e} (first half {e1:.2e}, second half {e2:.2e})")
    assert np.abs(do).max() > 0
    assert e <= SEIS_TOL, e


@pytest.mark.parametrize("k,name", [(0, "lambda"), (1, "mu"), (2, "rho")])
def test_elastic_gradient_directional_nt4000(fwi_lib, oracle_runs, k, name):
    from paper_2003_06027_gb300 import fwi

    d = _elastic()
    kw = fwi.problem_kwargs(d)
    s = slice(0, 1)
    args = [_cuda(d[n]) for n in ("vp", "vs", "rho")] + [_cuda(d[n][s]) for n in ("stf", "x0", "mt")] + \
           [_cuda(d["rec_iz"]), _cuda(d["rec_ix"])]
    obs = _cuda(np.zeros((1, 2, len(d["rec_iz"]), d["nt"]), np.float32))
    _, g, _, _, _ = fwi.misfit_grad_elastic(*args, obs, ckpt_every=d["ckpt_every"], want_src=False, **kw)
    dp = _directions(d)[k]
    got = float(np.sum(np.float64(g[k].cpu().numpy()) * dp))
    Jp = oracle_runs[("elastic_J", k, 1)].result()
    Jm = oracle_runs[("elastic_J", k, -1)].result()
    want = (Jp - Jm) / (2.0 * FD_REL)
    e = abs(got - want) / abs(want)
    print(f"\nelastic 300x800 nt=4000 dJ/d{name} . delta: device {got:.6e}, oracle FD {want:.6e}, rel {e:.2e}")
    assert e <= GRAD_TOL, e
