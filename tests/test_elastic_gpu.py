"""Parity of the CUDA elastic path (through the C ABI) with the FP64 oracle.

Bar: seismograms within relative L2 1e-4; misfit and the gradients with
respect to lambda, mu, rho, the source time function and the Gaussian source
position within relative L2 1e-3. Each side runs its own pipeline on the same
seeded inputs."""

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


def _cuda(x):
    import torch

    return torch.as_tensor(np.ascontiguousarray(x)).cuda()


def _args(d):
    return [_cuda(d[k]) for k in ("vp", "vs", "rho", "stf", "x0", "mt", "rec_iz", "rec_ix")]


def gpu_forward(d):
    from paper_2003_06027_gb300 import fwi

    return fwi.forward_elastic(*_args(d), **fwi.problem_kwargs(d)).cpu().numpy()


def gpu_misfit_grad(d, observed, K=None):
    from paper_2003_06027_gb300 import fwi

    J, g, gs, gx, seis = fwi.misfit_grad_elastic(*_args(d), _cuda(observed), ckpt_every=K or d["ckpt_every"],
                                                 want_seis=True, **fwi.problem_kwargs(d))
    return (float(J.cpu().numpy()[0]), g.cpu().numpy(), gs.cpu().numpy(), gx.cpu().numpy(), seis.cpu().numpy())


def oracle_inputs(d):
    return [np.float64(d[k]) for k in ("vp", "vs", "rho", "stf", "x0", "mt")]


CASES = [
    # nz, nx, nt, shots, order, npml, kind, seed
    (37, 71, 140, 2, 4, 10, 1, 31),   # ragged tiles in x and z, Gaussian moment tensors
    (45, 50, 120, 3, 8, 12, 0, 32),   # point sources, 8th order
    (20, 130, 100, 1, 4, 0, 1, 33),   # rigid boundary
    (70, 17, 120, 2, 8, 6, 1, 34),    # tall and narrow
]


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}x{c[1]}-o{c[4]}-pml{c[5]}-k{c[6]}" for c in CASES])
def test_elastic_parity(fwi_lib, case):
    nz, nx, nt, S, order, npml, kind, seed = case
    d = synth.random_elastic(seed, nz, nx, nt, S, order, npml, src_kind=kind, nrec=9)
    d["rec_iz"][:2] = [0, nz - 1]
    d["rec_ix"][:2] = [nx - 1, 0]
    dg = gpu_forward(d)
    do = oracle.elastic_forward(_geom(d), *oracle_inputs(d))
    assert np.abs(do).max() > 0
    assert rel(dg, do) <= SEIS_TOL, rel(dg, do)
    rng = np.random.default_rng(seed)
    obs = (rng.standard_normal(dg.shape) * np.abs(do).max() * 0.3).astype(np.float32)
    Jg, gg, gsg, gxg, _ = gpu_misfit_grad(d, obs, K=max(1, nt // 3 + 1))
    Jo, gl, gm, gr, gso, gxo = oracle.elastic_misfit_grad(_geom(d), *oracle_inputs(d), np.float64(obs))
    assert abs(Jg - Jo) <= SEIS_TOL * Jo
    for k, go in enumerate((gl, gm, gr)):
        assert rel(gg[k], go) <= GRAD_TOL, (k, rel(gg[k], go))
    assert rel(gsg, gso) <= GRAD_TOL, rel(gsg, gso)
    if kind == 1:
        assert rel(gxg, gxo) <= GRAD_TOL, (gxg, gxo)
    else:
        assert np.all(gxg == 0)


def test_elastic_layered_reduced_elementwise(fwi_lib):
    # the 300 x 800 discretisation (dx 5 m, 4th order, 32 CPML cells), 2 shots, 200 steps
    d = synth.elastic_layered(nshots=2, nt=200)
    d["x0"][:, 1] = [150.0, 210.0]  # shallow enough to reach the receivers within 200 steps
    do = oracle.elastic_forward(_geom(d), *oracle_inputs(d))
    dg = gpu_forward(d)
    assert rel(dg, do) <= SEIS_TOL, rel(dg, do)
    rng = np.random.default_rng(1)
    obs = (do * (1 + 0.2 * rng.standard_normal(do.shape))).astype(np.float32)
    Jg, gg, gsg, gxg, _ = gpu_misfit_grad(d, obs, K=50)
    Jo, gl, gm, gr, gso, gxo = oracle.elastic_misfit_grad(_geom(d), *oracle_inputs(d), np.float64(obs))
    assert abs(Jg - Jo) <= GRAD_TOL * Jo
    for k, go in enumerate((gl, gm, gr)):
        assert rel(gg[k], go) <= GRAD_TOL, (k, rel(gg[k], go))
    assert rel(gsg, gso) <= GRAD_TOL
    assert rel(gxg, gxo) <= GRAD_TOL


def test_elastic_checkpoint_invariance(fwi_lib):
    d = synth.random_elastic(41, 30, 40, 97, 2, 4, 8, nrec=5)
    obs = np.zeros((2, 2, 5, 97), np.float32)
    ref = gpu_misfit_grad(d, obs, K=97)
    for K in (1, 10, 33):
        r = gpu_misfit_grad(d, obs, K=K)
        assert r[0] == pytest.approx(ref[0], rel=1e-12)
        assert rel(r[1], ref[1]) <= 1e-6
    a = gpu_misfit_grad(d, obs, K=10)
    b = gpu_misfit_grad(d, obs, K=10)
    assert a[0] == b[0] and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_elastic_errors(fwi_lib):
    from paper_2003_06027_gb300 import fwi

    d = synth.random_elastic(51, 20, 20, 40, 1, 4, 4, nrec=2)
    kw = fwi.problem_kwargs(d)
    args = _args(d)
    with pytest.raises(fwi.FwiError) as e:
        fwi.forward_elastic(*args, **dict(kw, dt=0.05))
    assert e.value.status == 2
    bad = d["vs"].copy()
    bad[2, 2] = d["vp"][2, 2]  # vp^2 < 2 vs^2: negative lambda
    with pytest.raises(fwi.FwiError) as e:
        fwi.forward_elastic(args[0], _cuda(bad), *args[2:], **kw)
    assert e.value.status == 1
    assert rel(gpu_forward(d), oracle.elastic_forward(_geom(d), *oracle_inputs(d))) <= SEIS_TOL
