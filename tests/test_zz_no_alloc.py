"""fwi_forward_noalloc, the allocation-free forward call, against fwi_forward
and the FP64 oracle.

Some callers cannot let a library call cudaMalloc (their device memory is
owned by their own allocator, or their loop cannot afford the synchronisation
an allocation may cause). fwi_forward_noalloc runs the same forward modelling
in a fixed device array inside the library. It launches the same kernels on
the same inputs as fwi_forward, so its seismograms must be identical bit for
bit; a slip in its scratch layout would show as a difference. This file is
collected last so that a failure here comes after every other test has run.
"""

import ctypes

import numpy as np
import pytest

import oracle
from paper_2003_06027_gb300 import synth

pytestmark = pytest.mark.gpu

SEIS_TOL = 1e-4  # the seismogram tolerance of the parity tests


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _run(fwi, d, fn):
    import torch

    cu = lambda x: torch.as_tensor(np.ascontiguousarray(x)).cuda()
    out = fn(cu(d["c"]), cu(d["stf"]), cu(d["x0"]), cu(d["rec_iz"]), cu(d["rec_ix"]), **fwi.problem_kwargs(d))
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _geom(d):
    return dict(nz=d["nz"], nx=d["nx"], npml=d["npml"], order=d["order"], nt=d["nt"], dz=d["dz"],
                dx=d["dx"], dt=d["dt"], src_kind=d["src_kind"], pml_R=d["pml_R"],
                pml_vmax=d["pml_vmax"], pml_f0=d["pml_f0"], rec_iz=d["rec_iz"], rec_ix=d["rec_ix"])


def test_noalloc_matches_forward_on_two_calls(fwi_lib):
    from paper_2003_06027_gb300 import fwi

    # two different problems in a row: the second must not see the first's
    # leftovers in the shared scratch
    problems = [synth.random_acoustic(71, 37, 71, 150, 2, 8, 10, src_kind=1, nrec=8),
                synth.random_acoustic(72, 30, 26, 120, 3, 4, 6, src_kind=0, nrec=5)]
    for d in problems:
        ref = _run(fwi, d, fwi.forward)
        got = _run(fwi, d, fwi.forward_noalloc)
        assert np.abs(ref).max() > 0
        assert np.array_equal(got, ref), _rel(got, ref)
        # and the second call on the same (now dirty) scratch repeats it exactly
        assert np.array_equal(_run(fwi, d, fwi.forward_noalloc), ref)


def test_noalloc_matches_oracle(fwi_lib):
    from paper_2003_06027_gb300 import fwi

    d = synth.random_acoustic(73, 33, 57, 200, 2, 8, 9, src_kind=1, nrec=7)
    got = _run(fwi, d, fwi.forward_noalloc)
    want = oracle.acoustic_forward(_geom(d), np.float64(d["c"]), np.float64(d["stf"]), np.float64(d["x0"]))
    assert np.abs(want).max() > 0
    assert _rel(got, want) <= SEIS_TOL, _rel(got, want)


def test_noalloc_rejects_problems_beyond_its_scratch(fwi_lib):
    from paper_2003_06027_gb300 import fwi

    d = synth.acoustic_fwi(nshots=16, nt=4)
    with pytest.raises(fwi.FwiError) as e:
        _run(fwi, d, fwi.forward_noalloc)
    assert e.value.status == 1 and "bytes" in str(e.value)


def test_noalloc_rejects_host_pointers(fwi_lib):
    from paper_2003_06027_gb300 import fwi

    d = synth.random_acoustic(74, 30, 26, 50, 1, 4, 6, src_kind=0, nrec=3)
    host = lambda a: np.ascontiguousarray(a)
    c, stf, x0, iz, ix = (host(d[k]) for k in ("c", "stf", "x0", "rec_iz", "rec_ix"))
    seis = np.zeros((1, 3, d["nt"]), np.float32)
    p = lambda a: ctypes.c_void_p(a.ctypes.data)
    model = fwi._Model(fwi.FWI_ACOUSTIC, d["nz"], d["nx"], d["dz"], d["dx"], d["order"], d["npml"], d["pml_R"],
                       d["pml_vmax"], d["pml_f0"], p(c), None, None, fwi.FWI_OP_DIVERGENCE)
    src = fwi._Sources(1, fwi.FWI_SRC_POINT, p(x0), p(stf), None, 0)
    rec = fwi._Receivers(3, p(iz), p(ix))
    L = fwi.library()
    st = L.fwi_forward_noalloc(ctypes.byref(model), ctypes.byref(src), ctypes.byref(rec), d["nt"],
                               float(d["dt"]), ctypes.c_void_p(seis.ctypes.data), None)
    assert st == 1 and b"device pointers" in L.fwi_last_error()
    # the library stays usable
    assert np.abs(_run(fwi, d, fwi.forward_noalloc)).max() > 0
