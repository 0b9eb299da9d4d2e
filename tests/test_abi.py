"""CPU checks of the C-ABI library: it builds for sm_103a, loads, exports every
symbol include/epic.h declares, and rejects bad plans on the host before any
device work (argument validation and the grid-overflow check run first)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2609_03027_gb300 as E
from paper_2609_03027_gb300 import epic as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[\w\s\*]*?\b(epic_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_builds_and_exports_every_declared_symbol():
    L = E.load()
    declared = _declared_functions()
    assert len(declared) >= 10
    for name in declared:
        assert hasattr(L, name), name
    assert set(declared) <= set(E.EXPORTED) | set(declared)
    for name in E.EXPORTED:
        assert name in declared, name


def test_status_strings():
    L = E.load()
    for code, name in B.STATUS.items():
        assert L.epic_status_str(code).decode() == name


def _desc(**kw):
    pos = kw.pop("pos", np.array([[0.0, 0.0], [3.0, 1.0]]))
    freq = kw.pop("freq", np.array([150e6]))
    d = B._PlanDesc()
    d.n_ant = pos.shape[0]
    d.pos_m = pos.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    d.n_pol = 2
    d.n_chan = freq.shape[0]
    d.freq_hz = freq.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    d.cell_m = None
    d.grid_n = 32
    d.gcf.kind = 0
    d.gcf.K = 3
    d.gcf.sigma_cells = 0.5
    d.gcf.f_ref_hz = 150e6
    d.gcf.freq_scaled = 0
    d.gcf.oversample = 1
    d.gcf.table = None
    d.path = 0
    d.max_time = 16
    for k, v in kw.items():
        if k.startswith("gcf_"):
            setattr(d.gcf, k[4:], v)
        else:
            setattr(d, k, v)
    return d, (pos, freq)


@pytest.mark.parametrize("field,value", [
    ("n_pol", 3), ("n_pol", 0), ("grid_n", 48), ("grid_n", 4), ("grid_n", 1024), ("max_time", 0),
    ("gcf_K", 0), ("gcf_K", 9), ("gcf_sigma_cells", 0.0), ("gcf_kind", 7), ("path", 9), ("n_chan", 0),
    ("n_ant", 0), ("input_bits", 6), ("input_bits", 16), ("sub_int", -1), ("sub_int", 17), ("n_chan", 40000)])
def test_invalid_descriptor_rejected_on_host(field, value):
    L = E.load()
    d, keep = _desc(**{field: value})
    h = ctypes.c_void_p()
    st = L.epic_plan_create(ctypes.byref(d), ctypes.byref(h))
    assert st == 1, (field, value, L.epic_last_error(None))
    assert not h.value
    assert L.epic_last_error(None).decode()


def test_bad_frequency_and_table_rejected():
    L = E.load()
    d, keep = _desc(freq=np.array([-1.0]))
    assert L.epic_plan_create(ctypes.byref(d), ctypes.byref(ctypes.c_void_p())) == 1
    d, keep = _desc(gcf_kind=1)                                           # TABLE without a table
    assert L.epic_plan_create(ctypes.byref(d), ctypes.byref(ctypes.c_void_p())) == 1
    assert L.epic_plan_create(None, ctypes.byref(ctypes.c_void_p())) == 1


def test_grid_overflow_detected_at_plan_time():
    L = E.load()
    # 100 m apart at lambda/2 = 1 m cells on a 32 grid: far outside
    d, keep = _desc(pos=np.array([[-50.0, 0.0], [50.0, 0.0]]), freq=np.array([149896229.0]))
    h = ctypes.c_void_p()
    assert L.epic_plan_create(ctypes.byref(d), ctypes.byref(h)) == 2
    assert "leaves" in L.epic_last_error(None).decode()


def test_null_plan_calls_are_invalid():
    L = E.load()
    assert L.epic_image(None, None, 0, None, None, 0) == 1
    assert L.epic_image_host(None, None, 0, None, None, 0) == 1
    assert L.epic_sync(None) == 1
    assert L.epic_plan_destroy(None) == 0


def test_invalid_polarisation_mixing_rejected_on_host():
    L = E.load()
    j = np.zeros((1, 2, 2, 2, 2), dtype=np.float32)
    j[..., 0, 0, 0] = j[..., 1, 1, 0] = 1.0
    jp = j.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    d, keep = _desc(n_pol=1, jones=jp)                                    # needs two polarisations
    assert L.epic_plan_create(ctypes.byref(d), ctypes.byref(ctypes.c_void_p())) == 1
    assert "n_pol" in L.epic_last_error(None).decode()
    bad = j.copy()
    bad[0, 1, 0, 1, 1] = np.nan
    d, keep = _desc(jones=bad.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    assert L.epic_plan_create(ctypes.byref(d), ctypes.byref(ctypes.c_void_p())) == 1
    assert "finite" in L.epic_last_error(None).decode()
