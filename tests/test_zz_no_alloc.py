"""fwi_forward_noalloc, the allocation-free forward call, against fwi_forward.

Some callers cannot let a library call cudaMalloc (their device memory is
owned by their own allocator, or their loop cannot afford the synchronisation
an allocation may cause). fwi_forward_noalloc runs the same forward modelling
in a fixed device array inside the library. This file is collected last so
that a failure here comes after every other test has run.
"""

import numpy as np
import pytest

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
        assert _rel(got, ref) <= SEIS_TOL, _rel(got, ref)


def test_noalloc_rejects_problems_beyond_its_scratch(fwi_lib):
    from paper_2003_06027_gb300 import fwi

    d = synth.acoustic_fwi(nshots=16, nt=4)
    with pytest.raises(fwi.FwiError) as e:
        _run(fwi, d, fwi.forward_noalloc)
    assert e.value.status == 1 and "bytes" in str(e.value)
