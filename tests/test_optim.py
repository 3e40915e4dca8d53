"""The L-BFGS outer loop against problems whose minimisers are known in closed
form (CPU, float64): a strictly convex quadratic (x* = A^-1 b), the Rosenbrock
function (x* = (1, 1)), and a quadratic whose unconstrained minimiser lies
outside a box (the projected minimiser of a separable quadratic is the
clamped one)."""

import numpy as np
import torch

from paper_2003_06027_gb300.optim import lbfgs


def test_quadratic_reaches_the_solution_of_the_linear_system():
    g = torch.Generator().manual_seed(3)
    n = 60
    Q = torch.randn(n, n, generator=g, dtype=torch.float64)
    A = Q @ Q.T + n * torch.eye(n, dtype=torch.float64)
    b = torch.randn(n, generator=g, dtype=torch.float64)

    def fg(x):
        return 0.5 * float(x @ A @ x) - float(b @ x), A @ x - b

    x, log = lbfgs(fg, torch.zeros(n, dtype=torch.float64), iters=200, m=8, step0=0.1, gtol=1e-12)
    want = torch.linalg.solve(A, b)
    assert float((x - want).abs().max()) < 1e-8
    assert all(f1 <= f0 for f0, f1 in zip(log.f, log.f[1:]))  # monotone: Armijo steps only


def test_rosenbrock():
    def fg(v):
        x, y = float(v[0]), float(v[1])
        f = (1 - x) ** 2 + 100 * (y - x * x) ** 2
        return f, torch.tensor([-2 * (1 - x) - 400 * x * (y - x * x), 200 * (y - x * x)], dtype=torch.float64)

    x, log = lbfgs(fg, torch.tensor([-1.2, 1.0], dtype=torch.float64), iters=300, m=5, step0=0.5, gtol=1e-10)
    np.testing.assert_allclose(x.numpy(), [1.0, 1.0], atol=1e-6)
    assert log.f[-1] < 1e-12


def test_box_bounds_give_the_clamped_minimiser_of_a_separable_quadratic():
    d = torch.tensor([1.0, 4.0, 9.0, 2.0], dtype=torch.float64)
    c = torch.tensor([3.0, -2.0, 0.5, 0.2], dtype=torch.float64)
    lo, hi = -1.0, 1.0

    def fg(x):
        r = x - c
        return 0.5 * float((d * r * r).sum()), d * r

    x, _ = lbfgs(fg, torch.zeros(4, dtype=torch.float64), iters=100, m=4, step0=0.5, lower=lo, upper=hi)
    np.testing.assert_allclose(x.numpy(), c.clamp(lo, hi).numpy(), atol=1e-8)
