"""Parity of the CUDA acoustic path (through the C ABI) with the FP64 oracle.

Bar: seismograms within relative L2 1e-4, misfit and gradients within
relative L2 1e-3 (FP32 on the device, FP64 in the oracle). Inputs are the
seeded synthetic problems of paper_2003_06027_gb300.synth; each side runs its
own pipeline (the observed data of each side comes from that side's own
forward map, never from the other side).
"""

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
                dx=d["dx"], dt=d["dt"], src_kind=d["src_kind"], pml_R=d["pml_R"],
                pml_vmax=d["pml_vmax"], pml_f0=d["pml_f0"], rec_iz=d["rec_iz"], rec_ix=d["rec_ix"])


def _cuda(x):
    import torch

    return torch.as_tensor(np.ascontiguousarray(x)).cuda()


def gpu_forward(d, c=None):
    from paper_2003_06027_gb300 import fwi

    c = d["c"] if c is None else c
    out = fwi.forward(_cuda(c), _cuda(d["stf"]), _cuda(d["x0"]), _cuda(d["rec_iz"]),
                      _cuda(d["rec_ix"]), **fwi.problem_kwargs(d))
    return out.cpu().numpy()


def gpu_misfit_grad(d, observed, c=None, K=None):
    from paper_2003_06027_gb300 import fwi

    c = d["c"] if c is None else c
    J, g, gs, gx, seis = fwi.misfit_grad(
        _cuda(c), _cuda(d["stf"]), _cuda(d["x0"]), _cuda(d["rec_iz"]), _cuda(d["rec_ix"]),
        _cuda(observed), ckpt_every=K or d["ckpt_every"], want_seis=True, **fwi.problem_kwargs(d))
    return (float(J.cpu().numpy()[0]), g.cpu().numpy(), gs.cpu().numpy(), gx.cpu().numpy(),
            seis.cpu().numpy())


def oracle_misfit_grad(d, observed, c=None):
    c = d["c"] if c is None else c
    return oracle.acoustic_misfit_grad(_geom(d), np.float64(c), np.float64(d["stf"]),
                                       np.float64(d["x0"]), np.float64(observed))


def test_library_loads_on_gpu(fwi_lib):
    assert fwi_lib is not None


# ------------------------------------------------------------- 100 x 100 two-layer
def test_two_layer_forward_parity(fwi_lib):
    d = synth.acoustic_small()
    dg = gpu_forward(d)
    do = oracle.acoustic_forward(_geom(d), np.float64(d["c"]), np.float64(d["stf"]), np.float64(d["x0"]))
    assert np.abs(do).max() > 0
    assert rel(dg, do) <= SEIS_TOL, rel(dg, do)


def test_two_layer_misfit_grad_parity(fwi_lib):
    d = synth.acoustic_small()
    dp = synth.acoustic_small(perturbed=True)
    obs_g = gpu_forward(dp)
    obs_o = oracle.acoustic_forward(_geom(dp), np.float64(dp["c"]), np.float64(dp["stf"]),
                                    np.float64(dp["x0"]))
    Jg, gg, gsg, _, seis = gpu_misfit_grad(d, obs_g)
    Jo, go, gso, _ = oracle_misfit_grad(d, obs_o)
    assert Jo > 0
    assert abs(Jg - Jo) <= GRAD_TOL * Jo, (Jg, Jo)
    assert rel(gg, go) <= GRAD_TOL, rel(gg, go)
    assert rel(gsg, gso) <= GRAD_TOL, rel(gsg, gso)
    # the seismograms returned by the gradient call are the forward map
    assert rel(seis, gpu_forward(d)) == 0.0


# ------------------------------------------------------------- ragged multi-tile problems
CASES = [
    # nz, nx, nt, shots, order, npml, kind, seed
    (37, 71, 160, 2, 4, 10, 0, 11),   # 57 x 91 padded: ragged tiles in x and z
    (45, 50, 140, 3, 8, 13, 1, 12),   # Gaussian sources, 8th order
    (20, 130, 120, 1, 8, 0, 0, 13),   # no CPML (rigid boundary), wide
    (70, 17, 150, 2, 4, 6, 1, 14),    # tall and narrow
]


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}x{c[1]}-o{c[4]}-pml{c[5]}-k{c[6]}" for c in CASES])
def test_random_problem_parity(fwi_lib, case):
    nz, nx, nt, S, order, npml, kind, seed = case
    d = synth.random_acoustic(seed, nz, nx, nt, S, order, npml, src_kind=kind, nrec=9)
    # receivers on the physical edges too
    d["rec_iz"][:2] = [0, nz - 1]
    d["rec_ix"][:2] = [nx - 1, 0]
    dg = gpu_forward(d)
    do = oracle.acoustic_forward(_geom(d), np.float64(d["c"]), np.float64(d["stf"]), np.float64(d["x0"]))
    assert rel(dg, do) <= SEIS_TOL, rel(dg, do)
    rng = np.random.default_rng(seed)
    obs = (rng.standard_normal(dg.shape) * np.abs(do).max() * 0.3).astype(np.float32)
    Jg, gg, gsg, gxg, _ = gpu_misfit_grad(d, obs, K=max(1, nt // 3 + 1))
    Jo, go, gso, gxo = oracle_misfit_grad(d, obs)
    assert abs(Jg - Jo) <= SEIS_TOL * Jo
    assert rel(gg, go) <= GRAD_TOL, rel(gg, go)
    assert rel(gsg, gso) <= GRAD_TOL, rel(gsg, gso)
    if kind == 1:
        assert rel(gxg, gxo) <= GRAD_TOL, (gxg, gxo)
    else:
        assert np.all(gxg == 0)


def test_checkpoint_interval_invariance_and_determinism(fwi_lib):
    d = synth.random_acoustic(21, 30, 40, 97, 2, 8, 9, nrec=5)
    obs = np.zeros((2, 5, 97), np.float32)
    ref = gpu_misfit_grad(d, obs, K=97)
    for K in (1, 10, 33):
        r = gpu_misfit_grad(d, obs, K=K)
        assert r[0] == pytest.approx(ref[0], rel=1e-12)
        assert rel(r[1], ref[1]) <= 1e-6
        assert rel(r[2], ref[2]) <= 1e-6
    again = gpu_misfit_grad(d, obs, K=10)
    r10 = gpu_misfit_grad(d, obs, K=10)
    for a, b in zip(again[1:], r10[1:]):
        assert np.array_equal(a, b)
    assert again[0] == r10[0]


def test_host_and_device_pointers_agree(fwi_lib):
    from paper_2003_06027_gb300 import fwi

    d = synth.random_acoustic(31, 25, 33, 80, 2, 4, 8, nrec=4)
    kw = fwi.problem_kwargs(d)
    host = fwi.forward(d["c"], d["stf"], d["x0"], d["rec_iz"], d["rec_ix"], **kw)
    dev = gpu_forward(d)
    assert isinstance(host, np.ndarray)
    assert np.array_equal(host, dev)
    obs = np.zeros_like(host)
    J, g, gs, gx, _ = fwi.misfit_grad(d["c"], d["stf"], d["x0"], d["rec_iz"], d["rec_ix"], obs,
                                      ckpt_every=20, **kw)
    Jd, gd, gsd, _, _ = gpu_misfit_grad(d, obs, K=20)
    assert float(J[0]) == Jd and np.array_equal(g, gd) and np.array_equal(gs, gsd)


def test_zero_residual_gives_zero_gradient(fwi_lib):
    d = synth.random_acoustic(41, 20, 24, 60, 1, 4, 5, nrec=3)
    obs = gpu_forward(d)
    J, g, gs, gx, _ = gpu_misfit_grad(d, obs, K=15)
    assert J == 0.0 and np.all(g == 0) and np.all(gs == 0)


def test_single_cell_and_no_receivers(fwi_lib):
    from paper_2003_06027_gb300 import fwi

    d = synth.random_acoustic(51, 1, 1, 30, 1, 4, 3, nrec=1)
    d["x0"][:] = 0.0
    dg = gpu_forward(d)
    do = oracle.acoustic_forward(_geom(d), np.float64(d["c"]), np.float64(d["stf"]), np.float64(d["x0"]))
    assert rel(dg, do) <= SEIS_TOL
    kw = fwi.problem_kwargs(d)
    out = fwi.forward(_cuda(d["c"]), _cuda(d["stf"]), _cuda(d["x0"]), _cuda(np.zeros(0, np.int32)),
                      _cuda(np.zeros(0, np.int32)), **kw)
    assert tuple(out.shape) == (1, 0, 30)


def test_errors_are_reported(fwi_lib):
    from paper_2003_06027_gb300 import fwi

    d = synth.random_acoustic(61, 20, 20, 40, 1, 4, 4, nrec=2)
    kw = fwi.problem_kwargs(d)
    args = (_cuda(d["c"]), _cuda(d["stf"]), _cuda(d["x0"]), _cuda(d["rec_iz"]), _cuda(d["rec_ix"]))
    with pytest.raises(fwi.FwiError) as e:
        fwi.forward(*args, **dict(kw, dt=0.05))
    assert e.value.status == 2  # FWI_ECFL
    with pytest.raises(fwi.FwiError) as e:
        fwi.forward(*args, **dict(kw, order=6))
    assert e.value.status == 1
    bad = d["rec_iz"].copy()
    bad[0] = 20
    with pytest.raises(fwi.FwiError) as e:
        fwi.forward(args[0], args[1], args[2], _cuda(bad), args[4], **kw)
    assert e.value.status == 1
    x0 = d["x0"].copy()
    x0[0, 0] = -50.0
    with pytest.raises(fwi.FwiError) as e:
        fwi.forward(args[0], args[1], _cuda(x0), args[3], args[4], **kw)
    assert e.value.status == 1
    c = d["c"].copy()
    c[3, 3] = np.nan
    with pytest.raises(fwi.FwiError):
        fwi.forward(_cuda(c), *args[1:], **kw)
    # the context stays usable after errors
    assert rel(gpu_forward(d), oracle.acoustic_forward(_geom(d), np.float64(d["c"]), np.float64(d["stf"]),
                                                       np.float64(d["x0"]))) <= SEIS_TOL


# ------------------------------------------------------------- 201 x 601 FWI problem
@pytest.fixture(scope="module")
def fwi_problem():
    return synth.acoustic_fwi()


def test_fwi_reduced_nt_elementwise(fwi_lib):
    # 201 x 601, 8th order, CPML 32: two shots, 300 steps; every output compared
    d = synth.acoustic_fwi(nshots=2, nt=300)
    d["x0"][:, 0] = [1500.0, 4700.0]
    do = oracle.acoustic_forward(_geom(d), np.float64(d["c"]), np.float64(d["stf"]), np.float64(d["x0"]))
    dg = gpu_forward(d)
    assert rel(dg, do) <= SEIS_TOL, rel(dg, do)
    rng = np.random.default_rng(7)
    obs = (do * (1 + 0.2 * rng.standard_normal(do.shape))).astype(np.float32)
    Jg, gg, gsg, _, _ = gpu_misfit_grad(d, obs, K=100)
    Jo, go, gso, _ = oracle_misfit_grad(d, obs)
    assert abs(Jg - Jo) <= GRAD_TOL * Jo
    assert rel(gg, go) <= GRAD_TOL, rel(gg, go)
    assert rel(gsg, gso) <= GRAD_TOL


@pytest.mark.slow
def test_fwi_full_size_sampled(fwi_lib, fwi_problem):
    # Full size as benchmarked (16 shots, 3000 steps, checkpoint 100):
    # seismograms of two shots against the oracle, and the directional
    # derivative of the GPU gradient against a central difference of the
    # oracle's FP64 misfit.
    d = fwi_problem
    true = dict(d, c=d["c_true"])
    obs = gpu_forward(true)
    Jg, gg, _, _, seis = gpu_misfit_grad(d, obs)
    g2 = dict(_geom(d))
    sub = [0, 15]
    do = oracle.acoustic_forward(g2, np.float64(d["c"]), np.float64(d["stf"][sub]), np.float64(d["x0"][sub]))
    assert rel(seis[sub], do) <= SEIS_TOL, rel(seis[sub], do)
    # directional derivative on two shots (the gradient is a sum over shots)
    d2 = dict(d, stf=d["stf"][sub], x0=d["x0"][sub])
    obs2 = oracle.acoustic_forward(g2, np.float64(d["c_true"]), np.float64(d2["stf"]), np.float64(d2["x0"]))
    _, gg2, _, _, _ = gpu_misfit_grad(d2, obs2.astype(np.float32))
    rng = np.random.default_rng(3)
    dirn = synth.smooth(rng.standard_normal(d["c"].shape).astype(np.float32), 8.0).astype(np.float64)
    eps = 0.5

    def Jo(c):
        r = oracle.acoustic_forward(g2, c, np.float64(d2["stf"]), np.float64(d2["x0"])) - np.float64(
            obs2.astype(np.float32))
        return 0.5 * np.sum(r * r)

    c0 = np.float64(d["c"])
    fd = (Jo(c0 + eps * dirn) - Jo(c0 - eps * dirn)) / (2 * eps)
    gd = float(np.sum(np.float64(gg2) * dirn))
    assert abs(gd - fd) <= GRAD_TOL * abs(fd), (gd, fd)


def test_bounded_wait_gives_up_and_context_survives(fwi_lib):
    """The step kernels' bounded tile wait, run on a barrier that nothing
    completes, gives up after about a second with FWI_ETIMEOUT; the context
    then still computes a correct forward."""
    from paper_2003_06027_gb300 import fwi

    st, ns = fwi.selftest_wait_timeout(0)
    assert st == 6, (st, fwi.library().fwi_last_error())  # FWI_ETIMEOUT
    assert 0.5e9 < ns < 5e9, ns
    d = synth.random_acoustic(23, 20, 24, 60, 1, 4, 4, nrec=4)
    do = oracle.acoustic_forward(_geom(d), np.float64(d["c"]), np.float64(d["stf"]), np.float64(d["x0"]))
    assert rel(gpu_forward(d), do) <= SEIS_TOL


# ------------------------------------------------------------- line (plane-wave) sources
LINE_CASES = [  # seed, nz, nx, nt, shots, order, npml, line_len, K
    (21, 30, 70, 160, 3, 8, 8, 40, 40),
    (22, 40, 33, 130, 5, 4, 6, 33, 50),
]


@pytest.mark.parametrize("case", LINE_CASES, ids=[f"{c[1]}x{c[2]}-o{c[5]}-L{c[7]}-S{c[4]}" for c in LINE_CASES])
def test_line_source_parity(fwi_lib, case):
    """Plane-wave (line) sources against the oracle: seismograms (receivers on
    the source row included), misfit, dJ/dc and the per-cell dJ/damp, with
    several shot groups and checkpoint segments."""
    from paper_2003_06027_gb300 import fwi

    seed, nz, nx, nt, S, order, npml, L, K = case
    d = synth.line_source_problem(seed, nz, nx, nt, S, order, npml, line_len=L, nrec=9)
    g = dict(_geom(d), line_len=L)
    kw = fwi.problem_kwargs(d)
    args = [_cuda(d["c"]), _cuda(d["stf"]), _cuda(d["x0"]), _cuda(d["rec_iz"]), _cuda(d["rec_ix"])]
    seis = fwi.forward(*args, **kw).cpu().numpy()
    so = oracle.acoustic_forward(g, np.float64(d["c"]), np.float64(d["stf"]), np.float64(d["x0"]))
    assert rel(seis, so) <= SEIS_TOL, rel(seis, so)
    obs = oracle.acoustic_forward(g, np.float64(d["c"]) * 1.03, np.float64(d["stf"]), np.float64(d["x0"]))
    J, gc, gs, gx, _ = fwi.misfit_grad(*args, _cuda(obs), ckpt_every=K, **kw)
    Jo, gco, gso, _ = oracle.acoustic_misfit_grad(g, np.float64(d["c"]), np.float64(d["stf"]),
                                                  np.float64(d["x0"]), obs)
    assert gx is None and gs.shape == d["stf"].shape
    assert abs(float(J[0]) - Jo) <= GRAD_TOL * Jo
    assert rel(gc.cpu().numpy(), gco) <= GRAD_TOL, rel(gc.cpu().numpy(), gco)
    assert rel(gs.cpu().numpy(), gso) <= GRAD_TOL, rel(gs.cpu().numpy(), gso)


def test_line_source_errors(fwi_lib):
    from paper_2003_06027_gb300 import fwi

    d = synth.line_source_problem(23, 20, 30, 40, 2, 4, 5, line_len=10)
    kw = fwi.problem_kwargs(d)
    x0 = d["x0"].copy()
    x0[1, 0] = (d["nx"] - 5) * d["dx"]  # the line would leave the physical grid
    with pytest.raises(fwi.FwiError):
        fwi.forward(_cuda(d["c"]), _cuda(d["stf"]), _cuda(x0), _cuda(d["rec_iz"]), _cuda(d["rec_ix"]), **kw)
    # the context stays usable
    seis = fwi.forward(_cuda(d["c"]), _cuda(d["stf"]), _cuda(d["x0"]), _cuda(d["rec_iz"]), _cuda(d["rec_ix"]), **kw)
    assert np.isfinite(seis.cpu().numpy()).all()


# ------------------------------------------------------------- c^2 Laplacian operator
LAP_CASES = [  # nz, nx, nt, shots, order, npml, kind, seed, K
    (37, 71, 150, 2, 4, 10, 0, 41, 50),
    (30, 44, 140, 3, 8, 9, 1, 42, 47),
    (80, 200, 120, 2, 8, 10, 1, 45, 40),  # 4 x 4 tiles with interior ones and a ragged tail
]


@pytest.mark.parametrize("case", LAP_CASES, ids=[f"{c[0]}x{c[1]}-o{c[4]}-k{c[6]}" for c in LAP_CASES])
def test_laplacian_operator_parity(fwi_lib, case):
    """FWI_OP_LAPLACIAN (u_tt = c^2 Laplacian u) against the oracle's op 1:
    seismograms, misfit, dJ/dc, dJ/dstf and (Gaussian sources) dJ/dx0 over
    several checkpoint segments; and it differs from the divergence form."""
    nz, nx, nt, S, order, npml, kind, seed, K = case
    d = dict(synth.random_acoustic(seed, nz, nx, nt, S, order, npml, src_kind=kind, nrec=9), op=1)
    d["rec_iz"][:2] = [0, nz - 1]
    dg = gpu_forward(d)
    g = dict(_geom(d), op=1)
    do = oracle.acoustic_forward(g, np.float64(d["c"]), np.float64(d["stf"]), np.float64(d["x0"]))
    assert rel(dg, do) <= SEIS_TOL, rel(dg, do)
    d0 = oracle.acoustic_forward(_geom(d), np.float64(d["c"]), np.float64(d["stf"]), np.float64(d["x0"]))
    assert rel(d0, do) > 100 * SEIS_TOL  # the two operators are different maps in this medium
    rng = np.random.default_rng(seed)
    obs = (rng.standard_normal(dg.shape) * np.abs(do).max() * 0.3).astype(np.float32)
    Jg, gg, gsg, gxg, _ = gpu_misfit_grad(d, obs, K=K)
    Jo, go, gso, gxo = oracle.acoustic_misfit_grad(g, np.float64(d["c"]), np.float64(d["stf"]),
                                                   np.float64(d["x0"]), np.float64(obs))
    assert abs(Jg - Jo) <= SEIS_TOL * Jo
    assert rel(gg, go) <= GRAD_TOL, rel(gg, go)
    assert rel(gsg, gso) <= GRAD_TOL, rel(gsg, gso)
    if kind == 1:
        assert rel(gxg, gxo) <= GRAD_TOL, (gxg, gxo)


def test_laplacian_operator_line_source(fwi_lib):
    from paper_2003_06027_gb300 import fwi

    d = dict(synth.line_source_problem(43, 26, 40, 120, 2, 8, 6, line_len=20, nrec=7), op=1)
    g = dict(_geom(d), line_len=20, op=1)
    kw = fwi.problem_kwargs(d)
    args = [_cuda(d["c"]), _cuda(d["stf"]), _cuda(d["x0"]), _cuda(d["rec_iz"]), _cuda(d["rec_ix"])]
    so = oracle.acoustic_forward(g, np.float64(d["c"]), np.float64(d["stf"]), np.float64(d["x0"]))
    assert rel(fwi.forward(*args, **kw).cpu().numpy(), so) <= SEIS_TOL
    obs = oracle.acoustic_forward(g, np.float64(d["c"]) * 1.03, np.float64(d["stf"]), np.float64(d["x0"]))
    J, gc, gs, _, _ = fwi.misfit_grad(*args, _cuda(obs), ckpt_every=40, **kw)
    Jo, gco, gso, _ = oracle.acoustic_misfit_grad(g, np.float64(d["c"]), np.float64(d["stf"]),
                                                  np.float64(d["x0"]), obs)
    assert abs(float(J[0]) - Jo) <= GRAD_TOL * Jo
    assert rel(gc.cpu().numpy(), gco) <= GRAD_TOL
    assert rel(gs.cpu().numpy(), gso) <= GRAD_TOL


def test_laplacian_operator_graph_replay_and_noalloc(fwi_lib):
    """The c^2 Laplacian operator with receivers that share cells (their
    residuals enter the adjoint in receiver order) against the oracle; through
    a recorded CUDA graph it gives the direct call's misfit and gradients bit
    for bit (same kernels, same order, one stream), on every replay; the
    allocation-free forward refuses it with FWI_ENOTIMPL."""
    import torch

    from paper_2003_06027_gb300 import fwi

    d = dict(synth.random_acoustic(44, 30, 52, 130, 2, 8, 8, src_kind=1, nrec=6), op=1)
    for r in (3, 5):  # receivers 1, 3 and 5 record the same cell
        d["rec_iz"][r], d["rec_ix"][r] = d["rec_iz"][1], d["rec_ix"][1]
    kw = fwi.problem_kwargs(d)
    g64 = dict(_geom(d), op=1)
    args = [_cuda(d["c"]), _cuda(d["stf"]), _cuda(d["x0"]), _cuda(d["rec_iz"]), _cuda(d["rec_ix"])]
    obs64 = oracle.acoustic_forward(g64, np.float64(d["c"]) * 1.02, np.float64(d["stf"]), np.float64(d["x0"]))
    obs64[:, 3] *= 0.5  # different data at the shared cell: the three residuals differ
    obs64[:, 5] *= -1.0
    obs = _cuda(obs64.astype(np.float32))
    J, gc, gs, gx, _ = fwi.misfit_grad(*args, obs, ckpt_every=40, **kw)
    Jo, gco, gso, gxo = oracle.acoustic_misfit_grad(g64, np.float64(d["c"]), np.float64(d["stf"]),
                                                    np.float64(d["x0"]), np.float64(obs64.astype(np.float32)))
    assert abs(float(J[0]) - Jo) <= SEIS_TOL * Jo
    assert rel(gc.cpu().numpy(), gco) <= GRAD_TOL, rel(gc.cpu().numpy(), gco)
    assert rel(gs.cpu().numpy(), gso) <= GRAD_TOL, rel(gs.cpu().numpy(), gso)
    assert rel(gx.cpu().numpy(), gxo) <= GRAD_TOL, (gx, gxo)
    g = fwi.GradGraph(*args, obs, ckpt_every=40, want_src=True, **kw)
    try:
        for _ in range(2):
            g.launch()
            g.check()
            torch.cuda.synchronize()
            assert float(g.misfit[0]) == float(J[0])
            assert torch.equal(g.grad, gc) and torch.equal(g.grad_stf, gs) and torch.equal(g.grad_x0, gx)
    finally:
        g.close()
    with pytest.raises(fwi.FwiError) as e:
        fwi.forward_noalloc(*args, **kw)
    assert e.value.status == 7


# ------------------------------------------------ forward tile shapes (32 / 64 rows)
@pytest.mark.parametrize("shape", [(37, 71, 4, 1), (98, 45, 8, 0), (150, 130, 8, 1)])
def test_forward_tile_shapes_agree_bit_for_bit(fwi_lib, shape):
    """The 64 x 64 forward tiles (512 threads) against the 64 x 32 default:
    seismograms, misfit and gradients must be identical (each cell's arithmetic
    is the same), on grids whose padded height is not a multiple of either tile
    (the last tile row ragged), with receivers in the bottom rows; and the same
    as the oracle."""
    import torch

    from paper_2003_06027_gb300 import fwi

    nz, nx, order, kind = shape
    d = synth.random_acoustic(300 + nz, nz, nx, 140, 2, order, 9, src_kind=kind, nrec=9)
    d["rec_iz"][:3] = [nz - 1, nz - 2, 0]
    d["x0"][1, 1] = (nz - 4) * d["dz"]  # a source near the bottom edge
    rng = np.random.default_rng(nz)
    obs = (rng.standard_normal((2, 9, 140)) * 1e-7).astype(np.float32)
    out = {}
    for rows in (32, 64):
        fwi.set_tile_shape(rows)
        try:
            seis = gpu_forward(d)
            out[rows] = (seis,) + gpu_misfit_grad(d, obs, K=50)
        finally:
            fwi.set_tile_shape(0)
    a, b = out[32], out[64]
    assert np.array_equal(a[0], b[0])
    assert a[1] == b[1]
    for x, y in zip(a[2:], b[2:]):
        assert np.array_equal(x, y)
    do = oracle.acoustic_forward(_geom(d), np.float64(d["c"]), np.float64(d["stf"]), np.float64(d["x0"]))
    assert rel(b[0], do) <= SEIS_TOL
    Jo, go, _, _ = oracle_misfit_grad(d, obs)
    assert abs(b[1] - Jo) <= SEIS_TOL * Jo and rel(b[2], go) <= GRAD_TOL


def test_tile_shape_refusal(fwi_lib):
    from paper_2003_06027_gb300 import fwi

    with pytest.raises(fwi.FwiError) as e:
        fwi.set_tile_shape(48)
    assert e.value.status == 1
