"""Source inversions on top of the exact source gradients (Applications:
earthquake location and source time function retrieval; earthquake rupture
imaging).

* ``locate_source``: joint estimate of an earthquake's location x0 and source
  time function g(t) from recorded waveforms, with the source written as a
  Gaussian in space (sigma = half a cell) so that J is differentiable in x0; it
  starts, as in the paper's test, from a given (e.g. random) location and a zero
  source time function.
* ``superposed_misfit``: J = 1/2 || sum_k d_k - d_obs ||^2 for several sources
  active in ONE wavefield (a rupture: sub-sources switched on along a fault).
  The scheme is linear in its source term, so the wavefield of the sum is the
  sum of the per-source wavefields d_k (the sub-sources as the shots of one
  call). The library forms the sum, the residual and J on the device and seeds
  every sub-source's adjoint sweep with the common residual dJ/dd_k =
  sum_k d_k - d_obs (fwi_superposed_misfit_grad), which gives the gradient
  with respect to each sub-source's time function and position.
* ``gaussian_slip``: the rupture time / amplitude parametrisation
  g_k(t) = A_k exp(-(t - t_k)^2 / (2 s^2)), differentiable in (A_k, t_k).

All wave propagation and every gradient runs in the library's kernels; the
optimisation loops are ordinary torch code.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import torch

from . import fwi
from .autograd import acoustic_misfit


class SuperposedMisfit(torch.autograd.Function):
    """J(stf, x0, c) of sub-sources acting together: the library forms the sum
    of the sub-sources' seismograms, the residual and J, and the gradients by the
    adjoint sweep seeded with that residual (fwi_superposed_misfit_grad);
    backward scales them by the upstream gradient."""

    @staticmethod
    def forward(ctx, stf, x0, c, observed, rec_iz, rec_ix, opts):
        want_src = ctx.needs_input_grad[0] or ctx.needs_input_grad[1]
        J, gc, gs, gx = fwi.superposed_misfit_grad(c, stf, x0, rec_iz, rec_ix, observed,
                                                   want_grad=ctx.needs_input_grad[2], want_src=want_src, **opts)
        ctx.grads = (gs, gx, gc)
        return J.reshape(())

    @staticmethod
    def backward(ctx, gJ):
        gs, gx, gc = ctx.grads
        scale = lambda g: None if g is None else g * gJ.to(g.dtype)
        return (scale(gs) if ctx.needs_input_grad[0] else None, scale(gx) if ctx.needs_input_grad[1] else None,
                scale(gc) if ctx.needs_input_grad[2] else None, None, None, None, None)


def superposed_misfit(stf, x0, c, observed, rec_iz, rec_ix, *, dx, dz, dt, order=4, npml=20, pml_R=1e-3,
                      pml_vmax=4500.0, pml_f0=10.0, src_kind=fwi.FWI_SRC_GAUSSIAN, ckpt_every=100):
    """Differentiable misfit of the sources stf [k][nt] at x0 [k][2] acting
    together (a 0-d float64 tensor): J = 1/2 sum (sum_k d_k - observed)^2 for
    observed [nrec][nt], computed by the library."""
    opts = dict(dx=dx, dz=dz, dt=dt, order=order, npml=npml, pml_R=pml_R, pml_vmax=pml_vmax, pml_f0=pml_f0,
                src_kind=src_kind, ckpt_every=ckpt_every)
    return SuperposedMisfit.apply(stf, x0, c, observed, rec_iz, rec_ix, opts)


def gaussian_slip(A, t0, sigma, nt, dt):
    """[k][nt] time functions A_k exp(-(t_n - t0_k)^2 / (2 sigma^2)), t_n = n dt."""
    t = torch.arange(nt, device=A.device, dtype=A.dtype) * dt
    return A[:, None] * torch.exp(-((t[None, :] - t0[:, None]) ** 2) / (2.0 * sigma * sigma))


@dataclass
class LocationResult:
    x0: torch.Tensor
    stf: torch.Tensor
    misfit: list = field(default_factory=list)
    path: list = field(default_factory=list)


def locate_source(c, observed, rec_iz, rec_ix, x0_init, *, nt, dx, dz, dt, iters=200, lr_x0=None,
                  lr_stf=None, order=4, npml=20, pml_R=1e-3, pml_vmax=4500.0, pml_f0=10.0, ckpt_every=100,
                  stf_init=None):
    """Joint inversion of the location x0 [1][2] (metres) and the time function
    g(t) [1][nt] of one Gaussian source from observed [1][nrec][nt], by Adam
    steps on the exact gradients. Starts from x0_init and a zero g unless
    stf_init is given. Returns the estimate and the misfit / location history."""
    dev = c.device
    x0 = torch.nn.Parameter(torch.as_tensor(x0_init, dtype=torch.float32, device=dev).reshape(1, 2).clone())
    g0 = torch.zeros(1, nt, device=dev) if stf_init is None else torch.as_tensor(stf_init, device=dev).reshape(1, nt)
    stf = torch.nn.Parameter(g0.clone().float())
    scale = float(observed.abs().max())
    lr_x0 = 0.5 * min(dx, dz) if lr_x0 is None else lr_x0
    lr_stf = 0.02 if lr_stf is None else lr_stf
    opt = torch.optim.Adam([{"params": [x0], "lr": lr_x0}, {"params": [stf], "lr": lr_stf}])
    opts = dict(dx=dx, dz=dz, dt=dt, order=order, npml=npml, pml_R=pml_R, pml_vmax=pml_vmax, pml_f0=pml_f0,
                src_kind=fwi.FWI_SRC_GAUSSIAN, ckpt_every=ckpt_every)
    res = LocationResult(x0=x0.data, stf=stf.data)
    for _ in range(iters):
        opt.zero_grad()
        J = acoustic_misfit(c, stf, x0, observed, rec_iz, rec_ix, **opts)
        # J in units of the data's peak squared: seismograms of a unit source are
        # tiny (dt^2 / (2 pi sigma^2) per step), and Adam's epsilon would swamp
        # gradients of that size
        loss = J / (scale * scale)
        loss.backward()
        opt.step()
        res.misfit.append(float(loss.detach()))
        res.path.append(x0.detach().cpu().numpy().reshape(2).copy())
    res.x0, res.stf = x0.detach(), stf.detach()
    return res
