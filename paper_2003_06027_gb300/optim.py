"""L-BFGS for the outer FWI loop (the paper minimises its misfit with L-BFGS-B,
Full-waveform Inversion section).

``lbfgs`` is the limited-memory BFGS method with the two-loop recursion for
the inverse-Hessian product (Nocedal & Wright, Numerical Optimization, 2nd ed.,
Algorithms 7.4 and 7.5), a projected step onto box bounds, and a backtracking
line search on the sufficient-decrease (Armijo) condition. A pair (s, y) is kept
only if s.y > 0 (curvature condition), so the implicit inverse Hessian stays
positive definite. The first step of a run (and any step after a reset) is the
steepest-descent direction scaled so that its largest entry is ``step0``: FWI
misfits and gradients are tiny in absolute terms (J ~ 1e-12 here), so only the
shape of the gradient, not its size, sets the first step.

Everything is torch arithmetic on the parameter's device; dot products are
accumulated in FP64. ``fun_grad(x)`` returns (J, dJ/dx) — for FWI one
fwi_misfit_grad call (or a fwi.GradGraph launch).
"""

from __future__ import annotations

from dataclasses import dataclass, field

import torch


def _dot(a: torch.Tensor, b: torch.Tensor) -> float:
    return float(torch.dot(a.reshape(-1).double(), b.reshape(-1).double()))


@dataclass
class LbfgsLog:
    f: list = field(default_factory=list)       # objective after each accepted step (f[0]: start)
    evals: list = field(default_factory=list)   # function/gradient evaluations so far, per entry of f
    resets: int = 0


def lbfgs(fun_grad, x0: torch.Tensor, iters: int, m: int = 5, step0: float = 1.0, lower=None, upper=None,
          c1: float = 1e-4, shrink: float = 0.5, max_ls: int = 12, gtol: float = 0.0):
    """Minimise f over the box [lower, upper] from x0; returns (x, LbfgsLog).

    Each iteration: direction d = -H g by the two-loop recursion over the last
    ``m`` pairs (H0 = (s.y / y.y) I from the newest pair); trial points
    x(t) = P(x + t d), P the projection onto the box, with t = 1, shrink,
    shrink^2, ... until f(x(t)) <= f(x) + c1 g.(x(t) - x). A direction that is
    not a descent direction, or a line search that fails, clears the memory
    and retries along -g (scaled to ``step0``)."""
    proj = (lambda v: v.clamp(lower, upper)) if (lower is not None or upper is not None) else (lambda v: v)
    x = proj(x0.detach().clone())
    f, g = fun_grad(x)
    f = float(f)
    log = LbfgsLog(f=[f], evals=[1])
    nev = 1
    S, Y = [], []
    for _ in range(iters):
        if gtol > 0 and float(g.abs().max()) <= gtol:
            break
        for attempt in range(2):
            if S:
                q = g.clone()
                alphas = []
                for s, y in zip(reversed(S), reversed(Y)):
                    a = _dot(s, q) / _dot(y, s)
                    q.sub_(y, alpha=a)
                    alphas.append(a)
                gamma = _dot(S[-1], Y[-1]) / _dot(Y[-1], Y[-1])
                r = q.mul_(gamma)
                for (s, y), a in zip(zip(S, Y), reversed(alphas)):
                    b = _dot(y, r) / _dot(y, s)
                    r.add_(s, alpha=a - b)
                d = -r
            else:
                d = -g * (step0 / max(float(g.abs().max()), 1e-300))
            if _dot(g, d) >= 0.0:  # not a descent direction: forget the curvature pairs
                S.clear()
                Y.clear()
                log.resets += 1
                continue
            t, accepted = 1.0, False
            for _ls in range(max_ls):
                xn = proj(x + t * d)
                fn, gn = fun_grad(xn)
                fn = float(fn)
                nev += 1
                if fn <= f + c1 * _dot(g, xn - x):
                    accepted = True
                    break
                t *= shrink
            if accepted:
                break
            S.clear()
            Y.clear()
            log.resets += 1
        else:
            break  # no acceptable step along -g either: at a (projected) stationary point to this precision
        s_k, y_k = xn - x, gn - g
        if _dot(s_k, y_k) > 1e-12 * _dot(s_k, s_k) ** 0.5 * _dot(y_k, y_k) ** 0.5:
            S.append(s_k)
            Y.append(y_k)
            if len(S) > m:
                S.pop(0)
                Y.pop(0)
        x, f, g = xn, fn, gn
        log.f.append(f)
        log.evals.append(nev)
    return x, log
