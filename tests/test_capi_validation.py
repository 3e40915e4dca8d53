"""Argument validation at the C ABI (CPU): fwi_workspace_bytes checks its
arguments with the same functions as fwi_forward / fwi_misfit_grad (acoustic
and elastic) before any device work, so every documented error case can be
exercised without a GPU. Each case changes one field of a valid request and
expects the documented status; the valid request itself must pass."""

import ctypes

import numpy as np
import pytest

from paper_2003_06027_gb300 import fwi

EINVAL, ENOTIMPL = 1, 7


class Req:
    """A valid small request, with its arrays kept alive."""

    def __init__(self, elastic=False, kind=None):
        nz, nx, S, nt, nrec = 20, 30, 2, 40, 4
        self.c = np.full((nz, nx), 2000.0, np.float32)
        self.stf = np.zeros((S, nt), np.float32)
        self.x0 = np.array([[50.0, 50.0], [100.0, 80.0]], np.float32)
        self.mt = np.ones((S, 3), np.float32)
        self.iz = np.zeros(nrec, np.int32)
        self.ix = np.arange(nrec, dtype=np.int32)
        p = lambda a: ctypes.c_void_p(a.ctypes.data)
        phys = fwi.FWI_ELASTIC if elastic else fwi.FWI_ACOUSTIC
        self.model = fwi._Model(phys, nz, nx, 10.0, 10.0, 4, 5, 1e-3, 4500.0, 10.0, p(self.c),
                                p(self.c) if elastic else None, p(self.c) if elastic else None, 0)
        if kind is None:
            kind = fwi.FWI_SRC_GAUSSIAN if elastic else fwi.FWI_SRC_POINT
        self.src = fwi._Sources(S, kind, p(self.x0), p(self.stf), p(self.mt) if elastic else None, 0)
        self.rec = fwi._Receivers(nrec, p(self.iz), p(self.ix))
        self.nt = nt

    def status(self, nt=None, K=0):
        b = ctypes.c_uint64()
        return fwi.library().fwi_workspace_bytes(ctypes.byref(self.model), ctypes.byref(self.src),
                                                 ctypes.byref(self.rec), self.nt if nt is None else nt, K,
                                                 ctypes.byref(b))


ACOUSTIC_CASES = [
    ("nz", 0, EINVAL), ("nx", -3, EINVAL), ("dx", 0.0, EINVAL), ("dz", -1.0, EINVAL), ("order", 6, EINVAL),
    ("npml", -1, EINVAL), ("pml_R", 0.0, EINVAL), ("pml_R", 1.0, EINVAL), ("pml_vmax", 0.0, EINVAL),
    ("pml_f0", -1.0, EINVAL), ("vp", None, EINVAL), ("op", 2, EINVAL), ("physics", 7, ENOTIMPL),
    ("nz", 1 << 21, EINVAL),
]
SOURCE_CASES = [("nshots", 0, EINVAL), ("kind", fwi.FWI_SRC_MOMENT, EINVAL), ("kind", 9, EINVAL),
                ("x0", None, EINVAL), ("stf", None, EINVAL)]
RECEIVER_CASES = [("nrec", -1, EINVAL), ("iz", None, EINVAL), ("ix", None, EINVAL)]


def test_valid_requests_pass():
    for r in (Req(), Req(elastic=True), Req(elastic=True, kind=fwi.FWI_SRC_MOMENT)):
        assert r.status() == 0 and r.status(K=10) == 0 and r.status(K=r.nt) == 0


@pytest.mark.parametrize("field,value,want", ACOUSTIC_CASES)
def test_acoustic_model_fields(field, value, want):
    r = Req()
    setattr(r.model, field, value)
    assert r.status() == want
    assert fwi.library().fwi_last_error()  # a message for every refusal


@pytest.mark.parametrize("field,value,want", SOURCE_CASES)
def test_source_fields(field, value, want):
    r = Req()
    setattr(r.src, field, value)
    assert r.status() == want


@pytest.mark.parametrize("field,value,want", RECEIVER_CASES)
def test_receiver_fields(field, value, want):
    r = Req()
    setattr(r.rec, field, value)
    assert r.status() == want


def test_line_source_length():
    for L, want in ((0, EINVAL), (31, EINVAL), (30, 0), (1, 0)):
        r = Req(kind=fwi.FWI_SRC_LINE)
        r.src.line_len = L
        # a line source's stf is [S][nt][line_len]: size the array so a valid request is a real one
        r.stf = np.zeros((2, r.nt, max(L, 1)), np.float32)
        r.src.stf = ctypes.c_void_p(r.stf.ctypes.data)
        assert r.status() == want, L


def test_time_and_checkpoint_ranges():
    r = Req()
    assert r.status(nt=0) == EINVAL
    assert r.status(K=-1) == EINVAL and r.status(K=r.nt + 1) == EINVAL
    assert fwi.library().fwi_workspace_bytes(ctypes.byref(r.model), ctypes.byref(r.src), ctypes.byref(r.rec),
                                             r.nt, 0, None) == EINVAL  # no output pointer


def test_null_structs():
    r = Req()
    b = ctypes.c_uint64()
    L = fwi.library()
    assert L.fwi_workspace_bytes(None, ctypes.byref(r.src), ctypes.byref(r.rec), r.nt, 0, ctypes.byref(b)) == EINVAL
    assert L.fwi_workspace_bytes(ctypes.byref(r.model), None, ctypes.byref(r.rec), r.nt, 0, ctypes.byref(b)) == EINVAL
    assert L.fwi_workspace_bytes(ctypes.byref(r.model), ctypes.byref(r.src), None, r.nt, 0, ctypes.byref(b)) == EINVAL


@pytest.mark.parametrize("field,value", [("vs", None), ("rho", None)])
def test_elastic_model_fields(field, value):
    r = Req(elastic=True)
    setattr(r.model, field, value)
    assert r.status() == EINVAL


def test_elastic_sources():
    r = Req(elastic=True)
    r.src.mt = None
    assert r.status() == EINVAL
    r = Req(elastic=True, kind=fwi.FWI_SRC_LINE)
    assert r.status() == EINVAL  # line sources are acoustic only


# fwi_forward_noalloc checks the padded grid in 64-bit arithmetic before any
# device work or pointer query, so these refusals need no GPU.
@pytest.mark.parametrize("field,value", [("npml", 0x7FFFFFFF), ("npml", 0x40000000), ("nz", 1 << 21),
                                         ("nx", (1 << 20) - 9)])
def test_noalloc_grid_bound(field, value):
    r = Req()
    setattr(r.model, field, value)
    seis = np.zeros((2, 4, r.nt), np.float32)
    L = fwi.library()
    st = L.fwi_forward_noalloc(ctypes.byref(r.model), ctypes.byref(r.src), ctypes.byref(r.rec), r.nt, 1e-3,
                               ctypes.c_void_p(seis.ctypes.data), None)
    assert st == EINVAL
    assert b"grid too large" in L.fwi_last_error()
