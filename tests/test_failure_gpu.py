"""Failure handling on the GPU, made on the host side (no fault, trap or hang):
a workspace larger than the device (cudaMalloc fails cleanly: FWI_ENOMEM) and
non-finite inputs (NaN in a source time function: FWI_EUNSTABLE). After each
refusal the same context must still compute correct results."""

import numpy as np
import pytest

import oracle
from paper_2003_06027_gb300 import synth

pytestmark = pytest.mark.gpu

ENOMEM, EUNSTABLE = 3, 5


def _cuda(x):
    import torch

    return torch.as_tensor(np.ascontiguousarray(x)).cuda()


def _geom(d):
    return dict(nz=d["nz"], nx=d["nx"], npml=d["npml"], order=d["order"], nt=d["nt"], dz=d["dz"],
                dx=d["dx"], dt=d["dt"], src_kind=d["src_kind"], pml_R=d["pml_R"], pml_vmax=d["pml_vmax"],
                pml_f0=d["pml_f0"], rec_iz=d["rec_iz"], rec_ix=d["rec_ix"])


def _still_correct(fwi):
    d = synth.random_acoustic(81, 30, 40, 100, 2, 4, 6, src_kind=0, nrec=5)
    got = fwi.forward(*[_cuda(d[k]) for k in ("c", "stf", "x0", "rec_iz", "rec_ix")],
                      **fwi.problem_kwargs(d)).cpu().numpy()
    want = oracle.acoustic_forward(_geom(d), np.float64(d["c"]), np.float64(d["stf"]), np.float64(d["x0"]))
    assert np.linalg.norm(got - want) <= 1e-4 * np.linalg.norm(want)


def test_workspace_beyond_the_device_gives_enomem(fwi_lib):
    import torch

    from paper_2003_06027_gb300 import fwi

    total = torch.cuda.get_device_properties(0).total_memory
    # the 201 x 601 discretisation with no recomputation (ckpt_every = nt): the
    # stored fluxes of every step for enough shots to need ~1.5x the device
    nt = 3000
    d1 = synth.acoustic_fwi(nshots=1, nt=nt)
    one = fwi.workspace_bytes(d1["c"], d1["stf"], d1["x0"], d1["rec_iz"], d1["rec_ix"], ckpt_every=nt,
                              **fwi.problem_kwargs(d1))
    S = int(1.5 * total / one) + 1
    d = synth.acoustic_fwi(nshots=S, nt=nt)
    need = fwi.workspace_bytes(d["c"], d["stf"], d["x0"], d["rec_iz"], d["rec_ix"], ckpt_every=nt,
                               **fwi.problem_kwargs(d))
    assert need > 1.4 * total
    # one receiver keeps the host-side inputs small
    iz, ix = d["rec_iz"][:1], d["rec_ix"][:1]
    obs = np.zeros((S, 1, nt), np.float32)
    with pytest.raises(fwi.FwiError) as e:
        fwi.misfit_grad(_cuda(d["c"]), _cuda(d["stf"]), _cuda(d["x0"]), _cuda(iz), _cuda(ix), _cuda(obs),
                        ckpt_every=nt, want_src=False, **fwi.problem_kwargs(d))
    assert e.value.status == ENOMEM and "workspace" in str(e.value)
    _still_correct(fwi)


@pytest.mark.parametrize("call", ["forward", "gradient"])
def test_nonfinite_source_gives_eunstable(fwi_lib, call):
    from paper_2003_06027_gb300 import fwi

    d = synth.random_acoustic(82, 30, 40, 100, 2, 4, 6, src_kind=0, nrec=5)
    stf = d["stf"].copy()
    stf[1, 20] = np.nan
    args = [_cuda(d["c"]), _cuda(stf), _cuda(d["x0"]), _cuda(d["rec_iz"]), _cuda(d["rec_ix"])]
    with pytest.raises(fwi.FwiError) as e:
        if call == "forward":
            fwi.forward(*args, **fwi.problem_kwargs(d))
        else:
            fwi.misfit_grad(*args, _cuda(np.zeros((2, 5, 100), np.float32)), ckpt_every=25, **fwi.problem_kwargs(d))
    assert e.value.status == EUNSTABLE
    _still_correct(fwi)


def test_nonfinite_elastic_source_gives_eunstable(fwi_lib):
    from paper_2003_06027_gb300 import fwi

    d = synth.random_elastic(83, 25, 34, 80, 2, 4, 6, src_kind=1, nrec=5)
    stf = d["stf"].copy()
    stf[0, 10] = np.inf
    args = [_cuda(d[k]) for k in ("vp", "vs", "rho")] + [_cuda(stf)] + [_cuda(d[k]) for k in
                                                                       ("x0", "mt", "rec_iz", "rec_ix")]
    with pytest.raises(fwi.FwiError) as e:
        fwi.forward_elastic(*args, **fwi.problem_kwargs(d))
    assert e.value.status == EUNSTABLE
    _still_correct(fwi)
