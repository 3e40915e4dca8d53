"""CPU checks of the C-ABI library: it builds, loads, and exports every entry
point declared in include/fwi.h. No compute call (no GPU here)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fwi_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared("fwi.h")
    for n in ("fwi_create", "fwi_destroy", "fwi_forward", "fwi_misfit_grad", "fwi_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2003_06027_gb300 import build

    path = build.build()
    lib = ctypes.CDLL(path)
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            for n in _declared(h):
                assert hasattr(lib, n), f"{n} declared in include/{h} but not exported"


def test_binding_fails_loudly_without_a_device():
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2003_06027_gb300 import fwi

    with pytest.raises(fwi.FwiError):
        fwi.context(0)


def test_recorded_graph_refuses_pageable_or_mixed_inputs_on_the_host():
    """GradGraph's host-side checks run before the library is touched: host
    inputs must be page-locked, of the call's dtypes (a converted copy would not
    see the caller's in-place model updates), and not mixed with device ones."""
    torch = pytest.importorskip("torch")
    from paper_2003_06027_gb300 import fwi

    args = [torch.zeros(4, 4), torch.zeros(1, 5), torch.zeros(1, 2), torch.zeros(2, dtype=torch.int32),
            torch.zeros(2, dtype=torch.int32), torch.zeros(1, 2, 5)]
    with pytest.raises(ValueError):
        fwi.GradGraph(*args, dx=1.0, dz=1.0, dt=0.1)  # pageable host tensors
    with pytest.raises(ValueError):
        fwi.GradGraph(*args[:3], args[3].long(), *args[4:], dx=1.0, dz=1.0, dt=0.1)  # int64 receivers
