"""The C-ABI library loads and exports every entry point include/hemo.h
declares; host-only entry points and argument validation work without a GPU."""
import ctypes as C
import fractions
import os
import re

import numpy as np
import pytest

import __graft_entry__
from paper_2305_02752_gb300 import build as B
from paper_2305_02752_gb300 import hemo

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope='module', autouse=True)
def built():
    B.build()


def header_functions():
    src = open(os.path.join(ROOT, 'include', 'hemo.h')).read()
    src = re.sub(r'/\*.*?\*/', '', src, flags=re.S)
    return sorted(set(re.findall(r'\b(hemo_[a-z0-9_]+)\s*\(', src)))


def test_header_symbols_are_exported():
    names = header_functions()
    assert len(names) >= 15
    L = C.CDLL(hemo.LIB_PATH)
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(hemo.exported_symbols())


def test_library_velocity_set_is_d3q19():
    """The library's own D3Q19 table (Sec. 2.2) satisfies the exact lattice
    moment identities."""
    c, w = hemo.velocity_set()
    wf = [fractions.Fraction(x).limit_denominator(100) for x in w]
    assert sum(wf) == 1
    for a in range(3):
        assert sum(wf[i] * c[i, a] for i in range(19)) == 0
        for b in range(3):
            assert sum(wf[i] * c[i, a] * c[i, b] for i in range(19)) == (fractions.Fraction(1, 3) if a == b else 0)
    assert len({tuple(x) for x in c}) == 19


def _desc(**kw):
    d = hemo.hemo_lattice_desc()
    d.nx, d.ny, d.nz, d.tau, d.precision = 8, 8, 8, 1.0, 1
    for k in range(3):
        d.periodic[k] = 1
    for k, v in kw.items():
        setattr(d, k, v)
    return d


@pytest.mark.parametrize('kw,msg', [
    (dict(nx=0), 'sizes'),
    (dict(tau=0.5), 'tau'),
    (dict(precision=7), 'precision'),
])
def test_create_rejects_bad_arguments(kw, msg):
    L = hemo.lib()
    h = C.c_void_p()
    assert L.hemo_create_lattice(C.byref(_desc(**kw)), C.byref(h)) == hemo.HEMO_ERR_ARG
    assert msg in L.hemo_last_error().decode()
    assert not h.value


def test_create_rejects_bad_mask_and_flags():
    L = hemo.lib()
    h = C.c_void_p()
    mask = np.full(512, 4, np.uint8)
    d = _desc()
    d.wall_mask = mask.ctypes.data
    assert L.hemo_create_lattice(C.byref(d), C.byref(h)) == hemo.HEMO_ERR_ARG
    d = _desc()
    d.periodic[1] = 2
    assert L.hemo_create_lattice(C.byref(d), C.byref(h)) == hemo.HEMO_ERR_ARG
    assert L.hemo_create_lattice(None, C.byref(h)) == hemo.HEMO_ERR_ARG


def test_null_handles():
    L = hemo.lib()
    assert L.hemo_step(None, 1) == hemo.HEMO_ERR_ARG
    assert L.hemo_sync(None) == hemo.HEMO_ERR_ARG
    assert L.hemo_get_fields(None, 1, None, None, None, None, None) == hemo.HEMO_ERR_ARG
    assert L.hemo_velocity_set(None, None) == hemo.HEMO_ERR_ARG
    assert L.hemo_set_time_scales(None, 2, hemo.HEMO_AB2) == hemo.HEMO_ERR_ARG
    assert L.hemo_set_viscosity_ratio(None, 5.0) == hemo.HEMO_ERR_ARG
    assert L.hemo_get_inside(None, None) == hemo.HEMO_ERR_ARG
    assert L.hemo_set_lees_edwards(None, 0.01) == hemo.HEMO_ERR_ARG
    L.hemo_destroy(None)


def test_build_entry_point_exists():
    assert callable(__graft_entry__.build) and callable(__graft_entry__.smoke)
