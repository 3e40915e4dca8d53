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
