"""Memory planning of the gradient calls (CPU, host arithmetic only):
fwi_workspace_bytes against the field sizes the header documents, and
fwi_choose_ckpt against a brute-force search over every checkpoint interval
with the objective the header states (fewest recomputed forward steps, then
fewest segments, then least memory, among the intervals that fit)."""

import math

import numpy as np
import pytest

from paper_2003_06027_gb300 import fwi, synth


def _field_bytes(d, S, row_align):
    Nz, Nx = d["nz"] + 2 * d["npml"], d["nx"] + 2 * d["npml"]
    rows = math.ceil(Nz / row_align) * row_align + 16
    pitch = math.ceil(Nx / 64) * 64 + 16
    return S * rows * pitch * 4


def _acoustic(nt=60, S=3):
    d = synth.random_acoustic(5, 45, 90, nt, S, 8, 12, nrec=7)  # 69 padded rows: 128 with the 64-row padding
    args = [d["c"], d["stf"], d["x0"], d["rec_iz"], d["rec_ix"]]
    return d, args, fwi.problem_kwargs(d)


def _elastic(nt=50, S=2):
    d = synth.random_elastic(6, 30, 70, nt, S, 4, 10, nrec=5)
    args = [d[k] for k in ("vp", "vs", "rho", "stf", "x0", "mt", "rec_iz", "rec_ix")]
    kw = dict(dx=d["dx"], dz=d["dz"], order=d["order"], npml=d["npml"], pml_R=d["pml_R"],
              pml_vmax=d["pml_vmax"], pml_f0=d["pml_f0"], src_kind=d["src_kind"])
    return d, args, kw


@pytest.mark.parametrize("physics", ["acoustic", "laplacian", "elastic"])
def test_workspace_grows_by_the_documented_fields(physics):
    """Between two intervals K and K + 1 the workspace changes by the segment
    fields of one more step, less the checkpoints of the segments saved:
    (2, 1 for the c^2 Laplacian operator, or 5) F per step and (6 or 13) F per
    checkpoint, F one field of all shots on the tile-aligned slice (to the
    256-byte alignment of the layout)."""
    if physics in ("acoustic", "laplacian"):
        d, args, kw = _acoustic()
        ws, per_step, per_ckpt, S, align = fwi.workspace_bytes, 2, 6, d["stf"].shape[0], 64
        if physics == "laplacian":
            kw = dict(kw, op=fwi.FWI_OP_LAPLACIAN)
            per_step = 1
    else:
        d, args, kw = _elastic()
        ws, per_step, per_ckpt, S, align = fwi.workspace_bytes_elastic, 5, 13, d["stf"].shape[0], 32
    nt = d["stf"].shape[1]
    F = _field_bytes(d, S, align)
    W = {K: ws(*args, ckpt_every=K, **kw) for K in range(1, nt + 1)}
    for K in range(1, nt):
        dseg = math.ceil(nt / (K + 1)) - math.ceil(nt / K)
        want = per_step * F + per_ckpt * F * dseg
        assert abs(W[K + 1] - W[K] - want) < 512, (K, W[K + 1] - W[K], want)
    assert ws(*args, ckpt_every=0, **kw) < min(W.values())  # the forward call holds no gradient fields


def _brute(W, nt, budget):
    best = None
    for K, w in W.items():
        if w > budget:
            continue
        nseg = math.ceil(nt / K)
        key = ((nseg - 1) * K, nseg, w)  # both physics store the last segment in the forward sweep
        if best is None or key < best[0]:
            best = (key, K)
    return None if best is None else best[1]


@pytest.mark.parametrize("physics", ["acoustic", "elastic"])
def test_choose_ckpt_is_the_best_interval_that_fits(physics):
    if physics == "acoustic":
        d, args, kw = _acoustic()
        ws, choose = fwi.workspace_bytes, fwi.choose_ckpt
    else:
        d, args, kw = _elastic()
        ws, choose = fwi.workspace_bytes_elastic, fwi.choose_ckpt_elastic
    nt = d["stf"].shape[1]
    W = {K: ws(*args, ckpt_every=K, **kw) for K in range(1, nt + 1)}
    lo, hi = min(W.values()), max(W.values())
    assert choose(*args, budget_bytes=W[nt], **kw) == nt  # one segment fits: no checkpoint but the start
    budgets = [hi, W[nt], W[nt] - 1, lo, lo + 1] + [int(b) for b in np.linspace(lo, hi, 9)]
    for b in budgets:
        want = _brute(W, nt, b)
        if want is None:
            continue
        got = choose(*args, budget_bytes=b, **kw)
        assert got == want, (b, got, want)
        assert W[got] <= b
    with pytest.raises(fwi.FwiError) as e:
        choose(*args, budget_bytes=lo - 1, **kw)
    assert e.value.status == 3 and str(lo) in str(e.value)


def test_acoustic_no_recomputation_when_everything_fits():
    """With room for every step's fields the choice is K = nt (the forward
    sweep keeps all of them, nothing is recomputed); one byte less and it is
    the interval with the fewest recomputed steps that still fits."""
    d, args, kw = _acoustic(nt=48)
    nt = 48
    W = {K: fwi.workspace_bytes(*args, ckpt_every=K, **kw) for K in range(1, nt + 1)}
    assert fwi.choose_ckpt(*args, budget_bytes=max(W.values()), **kw) == nt
    K = fwi.choose_ckpt(*args, budget_bytes=W[nt] - 1, **kw)
    assert K < nt and W[K] < W[nt]
    assert (math.ceil(nt / K) - 1) * K == min((math.ceil(nt / k) - 1) * k for k in W if W[k] < W[nt])


def test_invalid_requests():
    d, args, kw = _acoustic()
    nt = d["stf"].shape[1]
    with pytest.raises(fwi.FwiError) as e:
        fwi.workspace_bytes(*args, ckpt_every=nt + 1, **kw)
    assert e.value.status == 1
    with pytest.raises(fwi.FwiError) as e:
        fwi.workspace_bytes(*args, ckpt_every=-1, **kw)
    assert e.value.status == 1
    bad = dict(kw, order=6)
    with pytest.raises(fwi.FwiError) as e:
        fwi.workspace_bytes(*args, **bad)
    assert e.value.status == 1
