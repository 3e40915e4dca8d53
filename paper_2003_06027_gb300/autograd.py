"""torch.autograd over the exact discrete adjoint.

The method of the paper differentiates the misfit of the discrete forward
recursion by reverse-mode AD, which it shows equals the adjoint-state method
(Method, the theorem relating reverse-mode AD and the adjoint-state method). The
library computes J and its exact gradient together in one fwi_misfit_grad call
(forward sweep with checkpoints, recompute, adjoint sweep); these Functions
expose that call to torch so a model and its sources can sit in an ordinary
torch optimisation loop:

    c = torch.nn.Parameter(c0)
    opt = torch.optim.Adam([c], lr=5.0)
    for _ in range(iters):
        opt.zero_grad()
        J = acoustic_misfit(c, stf, x0, observed, rec_iz, rec_ix, **geometry)
        J.backward()
        opt.step()

Differentiable inputs: the model (c, or vp, vs, rho), the source time
functions and the source positions (Gaussian sources). The receivers and the
observed data are constants; the moment tensors of elastic sources are too.
The gradient is computed when J is (the adjoint sweep runs inside forward), and
backward only scales it by the upstream gradient, so a graph holding J can be
backpropagated once per evaluation as usual.

The seismogram operators ``acoustic_seismograms`` / ``elastic_seismograms``
are the forward map itself as a differentiable op: forward runs the forward
sweep, and backward is the hand-written adjoint sweep seeded at the receivers
with the incoming gradient dL/dd (fwi_forward_vjp), i.e. the paper's
reverse-mode rule dU_k/dU_{k-1} = A^T (Eq. ad-backward) applied to any torch
loss L of the seismograms. Backward re-runs the forward sweep with checkpoints
(the states are not kept between forward and backward), so a backward costs
one gradient call.
"""

from __future__ import annotations

import torch

from . import fwi


def _scale(g, gJ):
    if g is None:
        return None
    return g * gJ.to(g.dtype)


class AcousticMisfit(torch.autograd.Function):
    """J(c, stf, x0) = 1/2 sum (d - d_obs)^2 of the acoustic scheme."""

    @staticmethod
    def forward(ctx, c, stf, x0, observed, rec_iz, rec_ix, opts):
        want_src = ctx.needs_input_grad[1] or ctx.needs_input_grad[2]
        J, gc, gs, gx, _ = fwi.misfit_grad(c, stf, x0, rec_iz, rec_ix, observed,
                                           want_grad=ctx.needs_input_grad[0], want_src=want_src, **opts)
        ctx.save_for_backward(*(t if t is not None else torch.empty(0) for t in (gc, gs, gx)))
        ctx.has = (gc is not None, gs is not None, gx is not None)
        ctx.shapes = (tuple(c.shape), tuple(stf.shape), tuple(x0.shape))
        return J.reshape(())

    @staticmethod
    def backward(ctx, gJ):
        saved = ctx.saved_tensors
        gc, gs, gx = (saved[k] if ctx.has[k] else None for k in range(3))
        gc = _scale(gc, gJ) if ctx.needs_input_grad[0] else None
        gs = _scale(gs, gJ).reshape(ctx.shapes[1]) if ctx.needs_input_grad[1] and gs is not None else None
        gx = _scale(gx, gJ).reshape(ctx.shapes[2]) if ctx.needs_input_grad[2] and gx is not None else None
        return gc, gs, gx, None, None, None, None


class ElasticMisfit(torch.autograd.Function):
    """J(vp, vs, rho, stf, x0) = 1/2 sum (d - d_obs)^2 of the elastic scheme
    (vx and vz seismograms); the model gradient is taken in (vp, vs, rho)."""

    @staticmethod
    def forward(ctx, vp, vs, rho, stf, x0, mt, observed, rec_iz, rec_ix, opts):
        want_model = any(ctx.needs_input_grad[:3])
        want_src = ctx.needs_input_grad[3] or ctx.needs_input_grad[4]
        J, glame, gs, gx, _ = fwi.misfit_grad_elastic(vp, vs, rho, stf, x0, mt, rec_iz, rec_ix, observed,
                                                      want_grad=want_model, want_src=want_src, **opts)
        gvel = fwi.elastic_velocity_grad(vp, vs, rho, glame, out=glame) if want_model else torch.empty(0)
        ctx.save_for_backward(gvel, *(t if t is not None else torch.empty(0) for t in (gs, gx)))
        ctx.has_src = gs is not None
        ctx.shapes = (tuple(stf.shape), tuple(x0.shape))
        return J.reshape(())

    @staticmethod
    def backward(ctx, gJ):
        gvel, gs, gx = ctx.saved_tensors
        out = [_scale(gvel[k], gJ) if ctx.needs_input_grad[k] else None for k in range(3)]
        gs = _scale(gs, gJ).reshape(ctx.shapes[0]) if ctx.needs_input_grad[3] and ctx.has_src else None
        gx = _scale(gx, gJ).reshape(ctx.shapes[1]) if ctx.needs_input_grad[4] and ctx.has_src else None
        return (*out, gs, gx, None, None, None, None, None)


class AcousticSeismograms(torch.autograd.Function):
    """d(c, stf, x0) = the acoustic seismograms [S][nrec][nt]; backward is the
    adjoint sweep seeded with dL/dd (vector-Jacobian product)."""

    @staticmethod
    def forward(ctx, c, stf, x0, rec_iz, rec_ix, opts):
        fwd = {k: v for k, v in opts.items() if k != "ckpt_every"}
        d = fwi.forward(c, stf, x0, rec_iz, rec_ix, **fwd)
        ctx.save_for_backward(c, stf, x0, rec_iz, rec_ix)
        ctx.opts = opts
        return d

    @staticmethod
    def backward(ctx, gd):
        c, stf, x0, iz, ix = ctx.saved_tensors
        need = ctx.needs_input_grad
        want_src = need[1] or need[2]
        if not (need[0] or want_src):
            return None, None, None, None, None, None
        _, gc, gs, gx, _ = fwi.forward_vjp(c, stf, x0, iz, ix, gd.contiguous(), want_grad=need[0],
                                           want_src=want_src, **ctx.opts)
        return (gc if need[0] else None, gs.reshape(stf.shape) if need[1] else None,
                gx.reshape(x0.shape) if need[2] and gx is not None else None, None, None, None)


class ElasticSeismograms(torch.autograd.Function):
    """d(vp, vs, rho, stf, x0) = the elastic seismograms [S][2][nrec][nt] (vx, vz);
    backward is the adjoint sweep seeded with dL/dd, taken to (vp, vs, rho)."""

    @staticmethod
    def forward(ctx, vp, vs, rho, stf, x0, mt, rec_iz, rec_ix, opts):
        fwd = {k: v for k, v in opts.items() if k != "ckpt_every"}
        d = fwi.forward_elastic(vp, vs, rho, stf, x0, mt, rec_iz, rec_ix, **fwd)
        ctx.save_for_backward(vp, vs, rho, stf, x0, mt, rec_iz, rec_ix)
        ctx.opts = opts
        return d

    @staticmethod
    def backward(ctx, gd):
        vp, vs, rho, stf, x0, mt, iz, ix = ctx.saved_tensors
        need = ctx.needs_input_grad
        want_model = any(need[:3])
        want_src = need[3] or need[4]
        if not (want_model or want_src):
            return (None,) * 9
        _, gl, gs, gx, _ = fwi.forward_vjp_elastic(vp, vs, rho, stf, x0, mt, iz, ix, gd.contiguous(),
                                                   want_grad=want_model, want_src=want_src, **ctx.opts)
        gv = fwi.elastic_velocity_grad(vp, vs, rho, gl, out=gl) if want_model else None
        out = [gv[k] if need[k] else None for k in range(3)]
        return (*out, gs.reshape(stf.shape) if need[3] else None, gx.reshape(x0.shape) if need[4] else None,
                None, None, None, None)


def acoustic_seismograms(c, stf, x0, rec_iz, rec_ix, *, dx, dz, dt, order=4, npml=20, pml_R=1e-3, pml_vmax=4500.0,
                         pml_f0=10.0, src_kind=fwi.FWI_SRC_POINT, op=fwi.FWI_OP_DIVERGENCE, ckpt_every=100):
    """Differentiable acoustic seismograms [S][nrec][nt] (float32, on c's device);
    ``ckpt_every`` is the checkpoint interval of the backward sweep, ``op`` the
    acoustic operator (divergence form or c^2 Laplacian)."""
    opts = dict(dx=dx, dz=dz, dt=dt, order=order, npml=npml, pml_R=pml_R, pml_vmax=pml_vmax, pml_f0=pml_f0,
                src_kind=src_kind, op=op, ckpt_every=ckpt_every)
    return AcousticSeismograms.apply(c, stf, x0, rec_iz, rec_ix, opts)


def elastic_seismograms(vp, vs, rho, stf, x0, mt, rec_iz, rec_ix, *, dx, dz, dt, order=4, npml=20, pml_R=1e-3,
                        pml_vmax=4500.0, pml_f0=10.0, src_kind=fwi.FWI_SRC_GAUSSIAN, ckpt_every=100):
    """Differentiable elastic seismograms [S][2][nrec][nt] (vx, vz)."""
    opts = dict(dx=dx, dz=dz, dt=dt, order=order, npml=npml, pml_R=pml_R, pml_vmax=pml_vmax, pml_f0=pml_f0,
                src_kind=src_kind, ckpt_every=ckpt_every)
    return ElasticSeismograms.apply(vp, vs, rho, stf, x0, mt, rec_iz, rec_ix, opts)


def acoustic_misfit(c, stf, x0, observed, rec_iz, rec_ix, *, dx, dz, dt, order=4, npml=20, pml_R=1e-3,
                    pml_vmax=4500.0, pml_f0=10.0, src_kind=fwi.FWI_SRC_POINT, op=fwi.FWI_OP_DIVERGENCE,
                    ckpt_every=100):
    """Differentiable acoustic misfit (a 0-d float64 tensor on c's device)."""
    opts = dict(dx=dx, dz=dz, dt=dt, order=order, npml=npml, pml_R=pml_R, pml_vmax=pml_vmax, pml_f0=pml_f0,
                src_kind=src_kind, op=op, ckpt_every=ckpt_every)
    return AcousticMisfit.apply(c, stf, x0, observed, rec_iz, rec_ix, opts)


def elastic_misfit(vp, vs, rho, stf, x0, mt, observed, rec_iz, rec_ix, *, dx, dz, dt, order=4, npml=20,
                   pml_R=1e-3, pml_vmax=4500.0, pml_f0=10.0, src_kind=fwi.FWI_SRC_GAUSSIAN, ckpt_every=100):
    """Differentiable elastic misfit (a 0-d float64 tensor on vp's device)."""
    opts = dict(dx=dx, dz=dz, dt=dt, order=order, npml=npml, pml_R=pml_R, pml_vmax=pml_vmax, pml_f0=pml_f0,
                src_kind=src_kind, ckpt_every=ckpt_every)
    return ElasticMisfit.apply(vp, vs, rho, stf, x0, mt, observed, rec_iz, rec_ix, opts)
