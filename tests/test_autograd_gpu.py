"""torch.autograd over the library's exact gradient, against the FP64 oracle.

The Functions run fwi_misfit_grad (and, for the elastic model, the chain rule
to vp, vs, rho in fwi_elastic_velocity_grad); backward must hand torch exactly
those gradients scaled by the upstream gradient. Bar: misfit within 1e-4 and
gradients within relative L2 1e-3 of the oracle on the same seeded inputs."""

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


def _kw(d, K):
    from paper_2003_06027_gb300 import fwi

    return dict(fwi.problem_kwargs(d), ckpt_every=K)


def test_acoustic_autograd_matches_oracle(fwi_lib):
    from paper_2003_06027_gb300.autograd import acoustic_misfit

    d = synth.random_acoustic(41, 33, 47, 130, 2, 8, 7, src_kind=1, nrec=8)
    do = oracle.acoustic_forward(_geom(d), np.float64(d["c"]), np.float64(d["stf"]), np.float64(d["x0"]))
    obs = (np.random.default_rng(41).standard_normal(do.shape) * np.abs(do).max() * 0.3).astype(np.float32)
    c, stf, x0 = _cuda(d["c"], True), _cuda(d["stf"], True), _cuda(d["x0"], True)
    J = acoustic_misfit(c, stf, x0, _cuda(obs), _cuda(d["rec_iz"]), _cuda(d["rec_ix"]), **_kw(d, 45))
    assert J.dim() == 0 and J.requires_grad
    (2.5 * J).backward()
    Jo, go, gso, gxo = oracle.acoustic_misfit_grad(_geom(d), np.float64(d["c"]), np.float64(d["stf"]),
                                                   np.float64(d["x0"]), np.float64(obs))
    assert abs(float(J.detach()) - Jo) <= SEIS_TOL * Jo
    assert rel(c.grad.cpu().numpy(), 2.5 * go) <= GRAD_TOL
    assert rel(stf.grad.cpu().numpy(), 2.5 * gso) <= GRAD_TOL
    assert rel(x0.grad.cpu().numpy(), 2.5 * gxo) <= GRAD_TOL


def test_acoustic_autograd_model_only(fwi_lib):
    """Only the model requires a gradient: the source gradients are not asked
    of the library and torch receives None for them."""
    from paper_2003_06027_gb300.autograd import acoustic_misfit
    from paper_2003_06027_gb300 import fwi

    d = synth.random_acoustic(42, 25, 30, 90, 1, 4, 5, nrec=6)
    obs = np.zeros((1, 6, 90), np.float32)
    c = _cuda(d["c"], True)
    stf, x0 = _cuda(d["stf"], True), _cuda(d["x0"])
    stf.requires_grad_(False)
    J = acoustic_misfit(c, stf, x0, _cuda(obs), _cuda(d["rec_iz"]), _cuda(d["rec_ix"]), **_kw(d, 30))
    J.backward()
    Jd, gd, _, _, _ = fwi.misfit_grad(c.detach(), stf, x0, _cuda(d["rec_iz"]), _cuda(d["rec_ix"]), _cuda(obs),
                                      **_kw(d, 30))
    assert float(J.detach()) == float(Jd[0])
    assert np.array_equal(c.grad.cpu().numpy(), gd.cpu().numpy())
    assert stf.grad is None


def test_acoustic_autograd_descent_step(fwi_lib):
    """A plain torch optimiser step along the library's gradient lowers J."""
    import torch

    from paper_2003_06027_gb300.autograd import acoustic_misfit
    from paper_2003_06027_gb300 import fwi

    d = synth.acoustic_small()
    dt_ = synth.acoustic_small(perturbed=True)
    kw = _kw(d, 100)
    iz, ix = _cuda(d["rec_iz"]), _cuda(d["rec_ix"])
    obs = fwi.forward(_cuda(dt_["c"]), _cuda(d["stf"]), _cuda(d["x0"]), iz, ix, **fwi.problem_kwargs(d))
    c = torch.nn.Parameter(_cuda(d["c"]))
    stf, x0 = _cuda(d["stf"]), _cuda(d["x0"])
    J0 = acoustic_misfit(c, stf, x0, obs, iz, ix, **kw)
    J0.backward()
    with torch.no_grad():
        g = c.grad
        c -= 1.0 * g / g.abs().max()  # at most 1 m/s per cell
    J1 = acoustic_misfit(c, stf, x0, obs, iz, ix, **kw)
    assert float(J1.detach()) < float(J0.detach())


def test_elastic_autograd_matches_oracle(fwi_lib):
    from paper_2003_06027_gb300.autograd import elastic_misfit

    d = synth.random_elastic(51, 29, 38, 110, 2, 4, 6, src_kind=1, nrec=7)
    ins = [np.float64(d[k]) for k in ("vp", "vs", "rho", "stf", "x0", "mt")]
    do = oracle.elastic_forward(_geom(d), *ins)
    obs = (np.random.default_rng(51).standard_normal(do.shape) * np.abs(do).max() * 0.3).astype(np.float32)
    vp, vs, rho = (_cuda(d[k], True) for k in ("vp", "vs", "rho"))
    stf, x0 = _cuda(d["stf"], True), _cuda(d["x0"], True)
    J = elastic_misfit(vp, vs, rho, stf, x0, _cuda(d["mt"]), _cuda(obs), _cuda(d["rec_iz"]), _cuda(d["rec_ix"]),
                       **_kw(d, 40))
    J.backward()
    Jo, gl, gm, gr, gso, gxo = oracle.elastic_misfit_grad(_geom(d), *ins, np.float64(obs))
    gvp, gvs, grho = oracle.elastic_velocity_grad(ins[0], ins[1], ins[2], gl, gm, gr)
    assert abs(float(J.detach()) - Jo) <= SEIS_TOL * Jo
    assert rel(vp.grad.cpu().numpy(), gvp) <= GRAD_TOL, rel(vp.grad.cpu().numpy(), gvp)
    assert rel(vs.grad.cpu().numpy(), gvs) <= GRAD_TOL, rel(vs.grad.cpu().numpy(), gvs)
    assert rel(rho.grad.cpu().numpy(), grho) <= GRAD_TOL, rel(rho.grad.cpu().numpy(), grho)
    assert rel(stf.grad.cpu().numpy(), gso) <= GRAD_TOL
    assert rel(x0.grad.cpu().numpy(), gxo) <= GRAD_TOL


def test_elastic_velocity_grad_elementwise(fwi_lib):
    """fwi_elastic_velocity_grad against the oracle's chain rule, cell by cell,
    out of place and in place."""
    from paper_2003_06027_gb300 import fwi

    rng = np.random.default_rng(5)
    nz, nx = 37, 129
    vp = (2500 + 1000 * rng.random((nz, nx))).astype(np.float32)
    vs = (vp / 1.8).astype(np.float32)
    rho = (2000 + 300 * rng.random((nz, nx))).astype(np.float32)
    gl3 = rng.standard_normal((3, nz, nx)).astype(np.float32)
    want = oracle.elastic_velocity_grad(vp, vs, rho, *np.float64(gl3))
    out = fwi.elastic_velocity_grad(_cuda(vp), _cuda(vs), _cuda(rho), _cuda(gl3)).cpu().numpy()
    g = _cuda(gl3)
    fwi.elastic_velocity_grad(_cuda(vp), _cuda(vs), _cuda(rho), g, out=g)
    for k in range(3):
        np.testing.assert_allclose(out[k], want[k], rtol=2e-6, atol=2e-6 * np.abs(want[k]).max())
    assert np.array_equal(g.cpu().numpy(), out)


# ------------------------------------------------------ seismogram operators (VJP)
def test_acoustic_seismogram_vjp_matches_oracle(fwi_lib):
    """d = F(c, stf, x0) as a differentiable op: backward with a random
    upstream gradient v is the adjoint sweep seeded with v, (dF/dtheta)^T v,
    which the oracle computes with the same v as its residual."""
    import torch

    from paper_2003_06027_gb300.autograd import acoustic_seismograms

    d = synth.random_acoustic(43, 31, 53, 140, 3, 8, 7, src_kind=1, nrec=9)
    c, stf, x0 = _cuda(d["c"], True), _cuda(d["stf"], True), _cuda(d["x0"], True)
    seis = acoustic_seismograms(c, stf, x0, _cuda(d["rec_iz"]), _cuda(d["rec_ix"]), **_kw(d, 35))
    do = oracle.acoustic_forward(_geom(d), np.float64(d["c"]), np.float64(d["stf"]), np.float64(d["x0"]))
    assert rel(seis.detach().cpu().numpy(), do) <= SEIS_TOL
    v = np.random.default_rng(43).standard_normal(do.shape).astype(np.float32)
    seis.backward(_cuda(v))
    go, gso, gxo = oracle.acoustic_adjoint(_geom(d), np.float64(d["c"]), np.float64(d["stf"]), np.float64(d["x0"]),
                                           np.float64(v))
    assert rel(c.grad.cpu().numpy(), go) <= GRAD_TOL, rel(c.grad.cpu().numpy(), go)
    assert rel(stf.grad.cpu().numpy(), gso) <= GRAD_TOL, rel(stf.grad.cpu().numpy(), gso)
    assert rel(x0.grad.cpu().numpy(), gxo) <= GRAD_TOL, rel(x0.grad.cpu().numpy(), gxo)
    # a torch loss composed with the operator: L = sum(w * d^2) has dL/dd = 2 w d
    c.grad = None
    w = _cuda(np.random.default_rng(44).random(do.shape).astype(np.float32))
    seis = acoustic_seismograms(c, stf.detach(), x0.detach(), _cuda(d["rec_iz"]), _cuda(d["rec_ix"]), **_kw(d, 35))
    torch.sum(w * seis * seis).backward()
    go2, _, _ = oracle.acoustic_adjoint(_geom(d), np.float64(d["c"]), np.float64(d["stf"]), np.float64(d["x0"]),
                                        2.0 * np.float64(w.cpu().numpy()) * do)
    assert rel(c.grad.cpu().numpy(), go2) <= GRAD_TOL, rel(c.grad.cpu().numpy(), go2)


def test_laplacian_seismogram_vjp_matches_oracle(fwi_lib):
    """The same seismogram operator with the c^2 Laplacian operator (op 1):
    backward with a random upstream gradient against the oracle's op-1 adjoint
    seeded with it, on a grid of several tiles with an interior one."""
    from paper_2003_06027_gb300.autograd import acoustic_seismograms

    d = dict(synth.random_acoustic(47, 70, 150, 110, 2, 8, 10, src_kind=1, nrec=9), op=1)
    g = dict(_geom(d), op=1)
    c, stf, x0 = _cuda(d["c"], True), _cuda(d["stf"], True), _cuda(d["x0"], True)
    seis = acoustic_seismograms(c, stf, x0, _cuda(d["rec_iz"]), _cuda(d["rec_ix"]), **_kw(d, 40))
    do = oracle.acoustic_forward(g, np.float64(d["c"]), np.float64(d["stf"]), np.float64(d["x0"]))
    assert rel(seis.detach().cpu().numpy(), do) <= SEIS_TOL
    v = np.random.default_rng(47).standard_normal(do.shape).astype(np.float32)
    seis.backward(_cuda(v))
    go, gso, gxo = oracle.acoustic_adjoint(g, np.float64(d["c"]), np.float64(d["stf"]), np.float64(d["x0"]),
                                           np.float64(v))
    assert rel(c.grad.cpu().numpy(), go) <= GRAD_TOL, rel(c.grad.cpu().numpy(), go)
    assert rel(stf.grad.cpu().numpy(), gso) <= GRAD_TOL, rel(stf.grad.cpu().numpy(), gso)
    assert rel(x0.grad.cpu().numpy(), gxo) <= GRAD_TOL, rel(x0.grad.cpu().numpy(), gxo)


def test_forward_vjp_value_is_the_inner_product(fwi_lib):
    """fwi_forward_vjp's scalar is <d, v> in FP64, and v = d - d_obs reproduces
    fwi_misfit_grad's gradient bit for bit (the same sweep, the same seed)."""
    from paper_2003_06027_gb300 import fwi

    d = synth.random_acoustic(45, 29, 41, 120, 2, 4, 6, src_kind=0, nrec=6)
    args = [_cuda(d[k]) for k in ("c", "stf", "x0", "rec_iz", "rec_ix")]
    kw = _kw(d, 30)
    seis = fwi.forward(*args, **fwi.problem_kwargs(d))
    v = np.random.default_rng(45).standard_normal(tuple(seis.shape)).astype(np.float32)
    val, _, _, _, _ = fwi.forward_vjp(*args, _cuda(v), **kw)
    want = float(np.sum(np.float64(seis.cpu().numpy()) * np.float64(v)))
    assert abs(float(val.cpu()[0]) - want) <= 1e-12 * max(1.0, abs(want)) + 1e-9 * np.abs(v).sum() * float(
        seis.abs().max())
    obs = np.float32(seis.cpu().numpy() * 0.5)
    _, g1, s1, _, _ = fwi.misfit_grad(*args, _cuda(obs), **kw)
    res = seis.cpu().numpy() - obs  # the residual k_misfit forms, in FP32
    _, g2, s2, _, _ = fwi.forward_vjp(*args, _cuda(res), **kw)
    assert np.array_equal(g1.cpu().numpy(), g2.cpu().numpy())
    assert np.array_equal(s1.cpu().numpy(), s2.cpu().numpy())


def test_elastic_seismogram_vjp_matches_oracle(fwi_lib):
    from paper_2003_06027_gb300.autograd import elastic_seismograms

    d = synth.random_elastic(53, 27, 36, 100, 2, 4, 6, src_kind=1, nrec=6)
    ins = [np.float64(d[k]) for k in ("vp", "vs", "rho", "stf", "x0", "mt")]
    vp, vs, rho = (_cuda(d[k], True) for k in ("vp", "vs", "rho"))
    stf, x0 = _cuda(d["stf"], True), _cuda(d["x0"], True)
    seis = elastic_seismograms(vp, vs, rho, stf, x0, _cuda(d["mt"]), _cuda(d["rec_iz"]), _cuda(d["rec_ix"]),
                               **_kw(d, 30))
    do = oracle.elastic_forward(_geom(d), *ins)
    assert rel(seis.detach().cpu().numpy(), do) <= SEIS_TOL
    v = np.random.default_rng(53).standard_normal(do.shape).astype(np.float32)
    seis.backward(_cuda(v))
    gl, gm, gr, gso, gxo = oracle.elastic_adjoint(_geom(d), *ins, np.float64(v))
    gvp, gvs, grho = oracle.elastic_velocity_grad(ins[0], ins[1], ins[2], gl, gm, gr)
    for got, want in ((vp, gvp), (vs, gvs), (rho, grho), (stf, gso), (x0, gxo)):
        assert rel(got.grad.cpu().numpy(), want) <= GRAD_TOL, rel(got.grad.cpu().numpy(), want)


def test_elastic_misfit_skips_the_model_gradient_when_not_needed(fwi_lib):
    """ElasticMisfit with only the sources requiring grad: the library call gets
    no model-gradient output, and the source gradients still match the oracle."""
    from paper_2003_06027_gb300.autograd import elastic_misfit

    d = synth.random_elastic(55, 25, 34, 90, 2, 4, 6, src_kind=1, nrec=5)
    ins = [np.float64(d[k]) for k in ("vp", "vs", "rho", "stf", "x0", "mt")]
    do = oracle.elastic_forward(_geom(d), *ins)
    obs = (np.random.default_rng(55).standard_normal(do.shape) * np.abs(do).max() * 0.3).astype(np.float32)
    vp, vs, rho = (_cuda(d[k]) for k in ("vp", "vs", "rho"))
    stf = _cuda(d["stf"], True)
    J = elastic_misfit(vp, vs, rho, stf, _cuda(d["x0"]), _cuda(d["mt"]), _cuda(obs), _cuda(d["rec_iz"]),
                       _cuda(d["rec_ix"]), **_kw(d, 30))
    J.backward()
    _, _, _, _, gso, _ = oracle.elastic_misfit_grad(_geom(d), *ins, np.float64(obs))
    assert vp.grad is None
    assert rel(stf.grad.cpu().numpy(), gso) <= GRAD_TOL
