"""Batched uneven-instance FWI: the batched sweep (all shots of an instance in
one call, several instances in flight on their own streams) must give the same
misfits and gradients as the plain per-shot sweep, and an FWI loop driven by
either must follow the same misfit history. Instance-level parity with the FP64
oracle is covered by the acoustic parity tests (the same library call)."""

import numpy as np
import pytest

from paper_2003_06027_gb300 import synth

pytestmark = pytest.mark.gpu


def _small_instances(n=3):
    # the smallest instances of the seeded uneven set, with nt cut to keep the test short
    cands = [synth.uneven_instance(4, i) for i in range(24)]
    cands.sort(key=lambda d: d["stf"].shape[0] * d["nz"] * d["nx"] * d["nt"])
    out = []
    for d in cands[:n]:
        nt = 600
        d = dict(d, nt=nt, stf=np.ascontiguousarray(d["stf"][:, :nt]), ckpt_every=100)
        out.append(d)
    return out


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_batched_equals_per_shot(fwi_lib):
    from paper_2003_06027_gb300 import batch

    inst = batch.prepare(_small_instances())
    Jb, gb, _ = batch.sweep(inst, "batched", workers=3)
    Jp, gp, _ = batch.sweep(inst, "plain")
    for i in range(len(inst)):
        jb, jp = float(Jb[i][0]), float(Jp[i][0])
        assert jb > 0 and abs(jb - jp) <= 1e-6 * jp, (i, jb, jp)
        assert rel(gb[i].cpu().numpy(), gp[i].cpu().numpy()) <= 1e-5


def test_fwi_histories_match(fwi_lib):
    from paper_2003_06027_gb300 import batch

    problems = _small_instances(2)
    a = batch.prepare(problems)
    b = batch.prepare(problems)
    ha = batch.fwi_iterations(a, 3, "batched", workers=2)
    hb = batch.fwi_iterations(b, 3, "plain")
    ja, jb = [h[0] for h in ha], [h[0] for h in hb]
    assert ja[-1] < ja[0]
    np.testing.assert_allclose(ja, jb, rtol=1e-4)


def test_autotune_picks_a_candidate(fwi_lib):
    from paper_2003_06027_gb300 import batch

    inst = batch.prepare(_small_instances(2))
    best, table = batch.autotune(inst, workers=(1, 2), ckpt=(50, 100), modes=("batched", "graph"))
    assert best in table and len(table) == 8
    assert table[best] == min(table.values())
    batch.close_graphs()


def test_graph_sweep_equals_batched(fwi_lib):
    """Recorded CUDA graphs run the same kernels in the same order: the same
    misfits and gradients bit for bit, sweep after sweep, and an in-place model
    update is picked up by the next launch."""
    import torch

    from paper_2003_06027_gb300 import batch, fwi

    inst = batch.prepare(_small_instances(3))
    Jb, gb, _ = batch.sweep(inst, "batched", workers=2)
    for _ in range(2):
        Jg, gg, _ = batch.sweep(inst, "graph", workers=2)
        for i in range(len(inst)):
            assert float(Jg[i][0]) == float(Jb[i][0])
            assert torch.equal(gg[i], gb[i])
    with torch.no_grad():
        inst[0].c.mul_(1.01)
    Jg, gg, _ = batch.sweep(inst, "graph", workers=2)
    J1, g1, _, _, _ = fwi.misfit_grad(inst[0].c, inst[0].stf, inst[0].x0, inst[0].rec_iz, inst[0].rec_ix,
                                      inst[0].observed, ckpt_every=100, want_src=False, **inst[0].kw)
    assert float(Jg[0][0]) == float(J1[0]) and torch.equal(gg[0], g1)
    batch.close_graphs()


def test_graph_replay_reports_phase_times(fwi_lib):
    """A recorded gradient keeps the call's phase marks as event-record nodes:
    after each replay the context reports positive phase and per-step kernel
    times that add up like a direct call's, and the direct call's launch count;
    the replay's results are the direct call's bit for bit."""
    import torch

    from paper_2003_06027_gb300 import batch, fwi

    (a,) = batch.prepare(_small_instances(1))
    J1, g1, _, _, _ = fwi.misfit_grad(a.c, a.stf, a.x0, a.rec_iz, a.rec_ix, a.observed, ckpt_every=100,
                                      want_src=False, **a.kw)
    td = fwi.last_timing(a.c.device.index)
    g = fwi.GradGraph(a.c, a.stf, a.x0, a.rec_iz, a.rec_ix, a.observed, ckpt_every=100, **a.kw)
    try:
        for _ in range(2):
            g.launch()
            g.check()
            t = g.timing()
            assert t.launches == td.launches > 0
            assert t.forward_ms > 0 and t.reverse_ms > 0 and t.total_ms >= 0.999 * (t.forward_ms + t.reverse_ms)
            assert t.fwd_step_ms > 0 and t.adj_step_ms > 0
            assert t.store_step_ms > 0  # the instance has more than one checkpoint segment
            assert float(g.misfit[0]) == float(J1[0]) and torch.equal(g.grad, g1)
    finally:
        g.close()


def test_graph_on_pinned_host_buffers(fwi_lib):
    """A gradient recorded on page-locked host tensors copies its inputs in and
    its results out at every replay: it gives the device-buffer call's misfit
    and gradients bit for bit, follows an in-place update of the host model on
    the next replay, and refuses pageable or mixed inputs."""
    import torch

    from paper_2003_06027_gb300 import batch, fwi

    (a,) = batch.prepare(_small_instances(1))
    pin = lambda t: t.detach().cpu().contiguous().pin_memory()
    h = [pin(a.c), pin(a.stf), pin(a.x0), pin(a.rec_iz.to(torch.int32)), pin(a.rec_ix.to(torch.int32)),
         pin(a.observed)]
    g = fwi.GradGraph(*h, ckpt_every=100, want_src=True, **a.kw)
    try:
        assert not g.grad.is_cuda and g.grad.is_pinned()
        for scale in (1.0, 1.01):
            if scale != 1.0:
                h[0].mul_(scale)  # the next replay reads the updated host model
            st = torch.cuda.current_stream()
            g.launch(st)
            g.check(st)
            J, gc, gs, gx, _ = fwi.misfit_grad(h[0].cuda(), a.stf, a.x0, a.rec_iz, a.rec_ix, a.observed,
                                               ckpt_every=100, **a.kw)
            assert float(g.misfit[0]) == float(J[0])
            assert torch.equal(g.grad, gc.cpu()) and torch.equal(g.grad_stf, gs.cpu())
            assert torch.equal(g.grad_x0, gx.cpu())
    finally:
        g.close()
    with pytest.raises(ValueError):
        fwi.GradGraph(a.c.cpu(), *h[1:], ckpt_every=100, **a.kw)  # pageable model
    with pytest.raises(ValueError):
        fwi.GradGraph(a.c, *h[1:], ckpt_every=100, **a.kw)  # device and host mixed


def test_graph_refuses_a_relaid_workspace(fwi_lib):
    """A graph is tied to its context's workspace: after a call with another
    problem layout on the same context, launching it fails with FWI_EINVAL."""
    import ctypes

    from paper_2003_06027_gb300 import batch, fwi

    a, b = batch.prepare(_small_instances(2))
    g = fwi.GradGraph(a.c, a.stf, a.x0, a.rec_iz, a.rec_ix, a.observed, ckpt_every=100, **a.kw)
    g.launch()
    g.check()
    other = fwi._Call(b.c, b.stf, b.x0, b.rec_iz, b.rec_ix, b.kw["dx"], b.kw["dz"], b.kw["order"], b.kw["npml"],
                      b.kw["pml_R"], b.kw["pml_vmax"], b.kw["pml_f0"], b.kw["src_kind"])
    out = fwi._empty_like_place(b.c, (b.shots, other.nrec, other.nt))
    L = fwi.library()
    fwi._check(L.fwi_forward(g.ctx, ctypes.byref(other.model), ctypes.byref(other.src), ctypes.byref(other.rec),
                             other.nt, float(b.kw["dt"]), fwi._ptr(out), fwi._stream(b.c, None)))
    with pytest.raises(fwi.FwiError):
        g.launch()
    g.close()


def test_lbfgs_fwi_descends_faster_than_normalised_steepest_descent(fwi_lib):
    """The paper's outer loop (L-BFGS) on recorded-graph gradients: every
    accepted step lowers the misfit, and after the same number of iterations it
    is below plain normalised steepest descent's."""
    from paper_2003_06027_gb300 import batch

    problems = _small_instances(1)
    a = batch.prepare(problems)
    b = batch.prepare(problems)
    log = batch.fwi_lbfgs(a[0], 6, step0=20.0)
    assert all(f1 < f0 for f0, f1 in zip(log.f, log.f[1:]))
    assert len(log.f) == 7
    hist = batch.fwi_iterations(b, 7, "batched", workers=1, step=20.0)
    J_sd = hist[-1][0]  # misfit at the start of the 7th steepest-descent iteration, i.e. after 6 steps
    assert log.f[-1] < J_sd, (log.f, [h[0] for h in hist])
    batch.close_graphs()


def test_shot_groups_do_not_change_results(fwi_lib):
    """The launch shape (shot groups of the forward and adjoint steps) changes
    only how the step kernels are launched: the misfit and every gradient are
    bit-identical for any split; values outside [0, 4] are refused."""
    import torch

    from paper_2003_06027_gb300 import batch, fwi

    inst = batch.prepare(_small_instances(1))[0]
    outs = []
    for grp in ((1, 1), (4, 2), (3, 3), (0, 0)):
        fwi.set_shot_groups(*grp)
        outs.append(fwi.misfit_grad(inst.c, inst.stf, inst.x0, inst.rec_iz, inst.rec_ix, inst.observed,
                                    ckpt_every=100, **inst.kw))
    for o in outs[1:]:
        assert float(o[0][0]) == float(outs[0][0][0])
        for a, b in zip(o[1:4], outs[0][1:4]):
            assert torch.equal(a, b)
    with pytest.raises(fwi.FwiError):
        fwi.set_shot_groups(5, 0)
    fwi.set_shot_groups(0, 0)


def test_autotune_over_launch_shapes(fwi_lib):
    from paper_2003_06027_gb300 import batch

    inst = batch.prepare(_small_instances(2))
    best, table = batch.autotune(inst, workers=(2,), ckpt=(100,), modes=("graph",), groups=((1, 1), (4, 2)))
    assert len(table) == 2 and best in table and table[best] == min(table.values())
    Jg, gg, _ = batch.sweep(inst, "graph", 2, 100, best[3])
    Jb, gb, _ = batch.sweep(inst, "batched", 2, 100)
    for i in range(len(inst)):
        assert float(Jg[i][0]) == float(Jb[i][0])
    batch.close_graphs()


# ----------------------------------------------- one persistent launch per step
def _oracle_instances():
    """Three small uneven instances (different grids, nt, shots, receivers;
    one shorter than the checkpoint interval, one not a multiple of it) with the
    same discretisation (8th order, dx = dz = 10 m, dt = 1 ms)."""
    shapes = [(34, 71, 230, 3, 7, 1), (27, 45, 160, 2, 5, 0), (41, 38, 70, 1, 4, 1)]
    out = []
    for k, (nz, nx, nt, S, nrec, kind) in enumerate(shapes):
        d = synth.random_acoustic(90 + k, nz, nx, nt, S, 8, 6, src_kind=kind, nrec=nrec)
        rng = np.random.default_rng(190 + k)
        d["c_obs"] = (d["c"] * (1.0 + 0.03 * rng.standard_normal(d["c"].shape))).astype(np.float32)
        out.append(d)
    return out


def _geom(d):
    return dict(nz=d["nz"], nx=d["nx"], npml=d["npml"], order=d["order"], nt=d["nt"], dz=d["dz"], dx=d["dx"],
                dt=d["dt"], src_kind=d["src_kind"], pml_R=d["pml_R"], pml_vmax=d["pml_vmax"], pml_f0=d["pml_f0"],
                rec_iz=d["rec_iz"], rec_ix=d["rec_ix"])


def _device_instance(fwi, d, obs):
    import torch

    cu = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda()
    return (cu(d["c"]), cu(d["stf"]), cu(d["x0"]), cu(d["rec_iz"]), cu(d["rec_ix"]), cu(obs), fwi.problem_kwargs(d))


def test_persistent_batch_matches_oracle_and_single_calls(fwi_lib):
    """fwi_batch_* (one launch per step over every instance's tiles, recorded as
    one graph) against the FP64 oracle, and bit for bit against fwi_misfit_grad
    of each instance alone (the same per-cell arithmetic and fold order)."""
    import oracle
    from paper_2003_06027_gb300 import fwi

    ds = _oracle_instances()
    K = 100
    obs = [oracle.acoustic_forward(_geom(d), np.float64(d["c_obs"]), np.float64(d["stf"]),
                                   np.float64(d["x0"])).astype(np.float32) for d in ds]
    inst = [_device_instance(fwi, d, o) for d, o in zip(ds, obs)]
    B = fwi.Batch(inst, ckpt_every=K)
    for rep in range(2):  # the creation sweep, then a replay of the recorded graph
        if rep:
            B.misfit.zero_()
            for g in B.grads:
                g.zero_()
            B.launch()
            B.check()
        for i, (d, o) in enumerate(zip(ds, obs)):
            Jo, go, _, _ = oracle.acoustic_misfit_grad(_geom(d), np.float64(d["c"]), np.float64(d["stf"]),
                                                       np.float64(d["x0"]), np.float64(o))
            Jb, gb = float(B.misfit[i].cpu()), B.grads[i].cpu().numpy()
            assert Jo > 0 and abs(Jb - Jo) <= 1e-4 * Jo, (i, Jb, Jo)
            assert rel(gb, go) <= 1e-3, (i, rel(gb, go))
            c, stf, x0, iz, ix, ob, kw = inst[i]
            Js, gs, _, _, _ = fwi.misfit_grad(c, stf, x0, iz, ix, ob, ckpt_every=min(K, d["nt"]), want_src=False, **kw)
            assert float(Js.cpu()[0]) == Jb
            assert np.array_equal(gs.cpu().numpy(), gb), i
    B.close()


def test_persistent_batch_follows_model_updates(fwi_lib):
    """The recorded sweep reads the models again at every launch."""
    from paper_2003_06027_gb300 import fwi

    ds = _oracle_instances()[:2]
    inst = [_device_instance(fwi, d, np.zeros((d["stf"].shape[0], len(d["rec_iz"]), d["nt"]), np.float32))
            for d in ds]
    B = fwi.Batch(inst, ckpt_every=50)
    inst[1][0].mul_(1.01)  # update instance 1's model in place
    B.launch()
    B.check()
    c, stf, x0, iz, ix, ob, kw = inst[1]
    Js, gs, _, _, _ = fwi.misfit_grad(c, stf, x0, iz, ix, ob, ckpt_every=50, want_src=False, **kw)
    assert float(Js.cpu()[0]) == float(B.misfit[1].cpu())
    assert np.array_equal(gs.cpu().numpy(), B.grads[1].cpu().numpy())
    B.close()


def test_persistent_batch_refusals(fwi_lib):
    from paper_2003_06027_gb300 import fwi

    ds = _oracle_instances()[:2]
    inst = [_device_instance(fwi, d, np.zeros((d["stf"].shape[0], len(d["rec_iz"]), d["nt"]), np.float32))
            for d in ds]
    bad = list(inst[1])
    bad[6] = dict(bad[6], dx=12.0, dz=12.0)  # another spacing than instance 0
    with pytest.raises(fwi.FwiError) as e:
        fwi.Batch([inst[0], tuple(bad)])
    assert e.value.status == 1
    fast = list(inst[1])
    fast[0] = fast[0] * 4.0  # CFL violated in instance 1
    with pytest.raises(fwi.FwiError) as e:
        fwi.Batch([inst[0], tuple(fast)])
    assert e.value.status == 2 and "instance 1" in str(e.value)


def test_persistent_sweep_and_fwi_history(fwi_lib):
    """batch.sweep in the persistent mode gives the batched mode's misfits and
    gradients, and an FWI loop on it follows the plain per-shot history."""
    from paper_2003_06027_gb300 import batch

    problems = _small_instances(3)
    a = batch.prepare(problems)
    Jp, gp, _ = batch.sweep(a, "persistent")
    Jb, gb, _ = batch.sweep(a, "batched", workers=2)
    for i in range(len(a)):
        assert float(Jp[i][0]) == float(Jb[i][0])
        assert np.array_equal(gp[i].cpu().numpy(), gb[i].cpu().numpy())
    b = batch.prepare(problems[:2])
    c = batch.prepare(problems[:2])
    hp = batch.fwi_iterations(b, 3, "persistent")
    hq = batch.fwi_iterations(c, 3, "plain")
    np.testing.assert_allclose([h[0] for h in hp], [h[0] for h in hq], rtol=1e-4)
    batch.close_graphs()
    batch.close_pools()
