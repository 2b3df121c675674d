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
    (dict(tau=float('nan')), 'tau'),
    (dict(nx=1024, ny=1024, nz=1024), 'too large'),  # 2^30 nodes: one past the limit
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


def test_create_rejects_half_an_allocator():
    L = hemo.lib()
    h = C.c_void_p()
    d = _desc()
    d.alloc = hemo.ALLOC_FN(lambda n, ctx: None)
    assert L.hemo_create_lattice(C.byref(d), C.byref(h)) == hemo.HEMO_ERR_ARG
    assert 'alloc and release' in L.hemo_last_error().decode()
    assert not h.value


def test_allocation_failure_is_oom():
    """A device memory provider that refuses makes create return
    HEMO_ERR_OOM with no handle (no CUDA call is reached)."""
    L = hemo.lib()
    h = C.c_void_p()
    calls = []
    d = _desc()
    d.alloc = hemo.ALLOC_FN(lambda n, ctx: calls.append(n) or None)
    d.release = hemo.FREE_FN(lambda p, ctx: None)
    assert L.hemo_create_lattice(C.byref(d), C.byref(h)) == hemo.HEMO_ERR_OOM
    assert not h.value and len(calls) >= 1


@pytest.mark.skipif(__import__('torch').cuda.is_available(), reason='hands the library placeholder device addresses')
def test_partial_allocation_failure_releases_everything():
    """The provider grants the first allocations (placeholder addresses the
    library never dereferences: the lattice's allocations all come before
    its first CUDA call) and refuses the last: every granted block is
    released exactly once."""
    L = hemo.lib()
    granted, released = [], []

    def alloc(n, ctx):
        if len(granted) == 5:
            return None
        granted.append(0x10000 * (len(granted) + 1))
        return granted[-1]

    d = _desc()
    d.alloc = hemo.ALLOC_FN(alloc)
    d.release = hemo.FREE_FN(lambda p, ctx: released.append(p))
    h = C.c_void_p()
    assert L.hemo_create_lattice(C.byref(d), C.byref(h)) == hemo.HEMO_ERR_OOM
    assert not h.value
    assert sorted(released) == granted


def test_noalloc_binning_limits():
    """The allocation-free binning refuses sizes beyond its fixed scratch
    (1,048,576 vertices, 131,072 blocks of 8^3) and missing outputs before
    touching the GPU."""
    L = hemo.lib()
    per = (C.c_int * 3)(1, 1, 1)
    dummy = C.c_void_p(16)  # never dereferenced: the arguments are refused first
    args = lambda nv, nx, ny, nz, start=dummy: (dummy, nv, nx, ny, nz, per, dummy, dummy, start, None)  # noqa: E731
    assert L.hemo_bin_vertices_noalloc(*args(1048577, 64, 64, 64)) == hemo.HEMO_ERR_ARG
    assert L.hemo_bin_vertices_noalloc(*args(10, 8 * 64, 8 * 64, 8 * 33)) == hemo.HEMO_ERR_ARG
    assert L.hemo_bin_vertices_noalloc(*args(10, 64, 64, 64, start=None)) == hemo.HEMO_ERR_ARG
    assert L.hemo_bin_vertices_noalloc(*args(-1, 64, 64, 64)) == hemo.HEMO_ERR_ARG
    assert L.hemo_bin_vertices_noalloc(*args(10, 0, 64, 64)) == hemo.HEMO_ERR_ARG
    # block counts whose product would overflow 64 bits, or one axis alone
    # beyond the limit (the sizes are checked axis by axis before the product)
    big = 2 ** 31 - 1
    assert L.hemo_bin_vertices_noalloc(*args(10, big, big, big)) == hemo.HEMO_ERR_ARG
    assert L.hemo_bin_vertices_noalloc(*args(10, 2 ** 30, 2 ** 30, 2 ** 30)) == hemo.HEMO_ERR_ARG
    assert L.hemo_bin_vertices_noalloc(*args(10, big, 1, 1)) == hemo.HEMO_ERR_ARG
    assert L.hemo_bin_vertices_noalloc(*args(10, 1, 1, 8 * 131073)) == hemo.HEMO_ERR_ARG


def test_noalloc_binding_checks_buffers():
    """The binding is the only place that can check the caller's buffers
    (the C ABI takes bare pointers): wrong dtypes, host tensors,
    non-contiguous or too-small buffers are refused with HEMO_ERR_ARG
    before the library is called."""
    import torch
    nv, dims = 10, (16, 16, 16)
    nbins = 8
    good = dict(verts=torch.zeros((nv, 3), dtype=torch.float64), key=torch.zeros(nv, dtype=torch.int32),
                perm=torch.zeros(nv, dtype=torch.int32), start=torch.zeros(nbins + 1, dtype=torch.int32))
    bad_cases = [
        dict(verts=torch.zeros((nv, 3), dtype=torch.float32)),
        dict(verts=torch.zeros((nv, 2), dtype=torch.float64)),
        dict(verts=torch.zeros((3, nv), dtype=torch.float64).t()),
        dict(key=torch.zeros(nv - 1, dtype=torch.int32)),
        dict(perm=torch.zeros(nv, dtype=torch.int64)),
        dict(start=torch.zeros(nbins, dtype=torch.int32)),
    ]
    for case in bad_cases:
        a = dict(good, **case)
        with pytest.raises(hemo.HemoError) as e:
            hemo.bin_vertices_noalloc(a['verts'], dims, (1, 1, 1), a['key'], a['perm'], a['start'],
                                      _require_cuda=False)
        assert e.value.code == hemo.HEMO_ERR_ARG, case
    # host tensors are refused too (the kernels need device memory)
    with pytest.raises(hemo.HemoError) as e:
        hemo.bin_vertices_noalloc(good['verts'], dims, (1, 1, 1), good['key'], good['perm'], good['start'])
    assert e.value.code == hemo.HEMO_ERR_ARG


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
    assert L.hemo_set_force_tolerance(None, 0.1) == hemo.HEMO_ERR_ARG
    cnt = C.c_longlong(-5)
    assert L.hemo_get_force_evaluations(None, C.byref(cnt)) == hemo.HEMO_ERR_ARG and cnt.value == -5
    n = C.c_size_t(7)
    assert L.hemo_state_bytes(None, C.byref(n)) == hemo.HEMO_ERR_ARG and n.value == 7
    assert L.hemo_save_state(None, None, 0) == hemo.HEMO_ERR_ARG
    assert L.hemo_load_state(None, None, 0) == hemo.HEMO_ERR_ARG
    L.hemo_destroy(None)


def test_build_entry_point_exists():
    assert callable(__graft_entry__.build) and callable(__graft_entry__.smoke)


def test_binding_layouts_match_the_header(tmp_path):
    """The ctypes structures and constants of the binding against the C
    header, as a C compiler lays them out (sizes, field offsets, enum
    values)."""
    lat = [f for f, _ in hemo.hemo_lattice_desc._fields_]
    mesh = [f for f, _ in hemo.hemo_mesh_desc._fields_]
    consts = ['HEMO_OK', 'HEMO_ERR_ARG', 'HEMO_ERR_OOM', 'HEMO_ERR_CUDA', 'HEMO_ERR_NUMERIC', 'HEMO_ERR_DOMAIN',
              'HEMO_ERR_STATE', 'HEMO_RHO', 'HEMO_U', 'HEMO_VERTS', 'HEMO_FORCES', 'HEMO_CELLSTATS',
              'HEMO_OPT_STAGED_COLLISION', 'HEMO_OPT_NODE_COLLISION', 'HEMO_OPT_TEST_STALLED_WAIT',
              'HEMO_OPT_PAIR_COLLISION', 'HEMO_OPT_WIDE_INDEX', 'HEMO_OPT_NODE_STAGING',
              'HEMO_OPT_UNSTAGED_COLLISION', 'HEMO_EULER',
              'HEMO_AB2']
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "hemo.h"', 'int main(void) {',
             'printf("lat %zu\\n", sizeof(hemo_lattice_desc));', 'printf("mesh %zu\\n", sizeof(hemo_mesh_desc));']
    lines += [f'printf("lat.{f} %zu\\n", offsetof(hemo_lattice_desc, {f}));' for f in lat]
    lines += [f'printf("mesh.{f} %zu\\n", offsetof(hemo_mesh_desc, {f}));' for f in mesh]
    lines += [f'printf("{c} %d\\n", (int){c});' for c in consts]
    lines += ['printf("prec %d %d %d %d\\n", HEMO_F64, HEMO_F32, HEMO_F16DEV, HEMO_BF16DEV);',
              'printf("phases %d\\n", HEMO_NUM_PHASES);', 'return 0; }']
    src = tmp_path / 'layout.c'
    src.write_text('\n'.join(lines) + '\n')
    exe = tmp_path / 'layout'
    import subprocess
    subprocess.run(['gcc', '-std=c99', '-Wall', '-Werror', '-I', os.path.join(ROOT, 'include'), str(src), '-o', str(exe)],
                   check=True)
    got = dict(line.split(' ', 1) for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                            text=True).stdout.splitlines())
    assert int(got['lat']) == C.sizeof(hemo.hemo_lattice_desc)
    assert int(got['mesh']) == C.sizeof(hemo.hemo_mesh_desc)
    for f in lat:
        assert int(got[f'lat.{f}']) == getattr(hemo.hemo_lattice_desc, f).offset, f
    for f in mesh:
        assert int(got[f'mesh.{f}']) == getattr(hemo.hemo_mesh_desc, f).offset, f
    for c in consts:
        assert int(got[c]) == getattr(hemo, c), c
    assert [int(x) for x in got['prec'].split()] == [hemo.PRECISIONS[p] for p in ('f64', 'f32', 'f16', 'bf16')]
    assert int(got['phases']) == len(hemo.Simulation.PHASES)


def _c_kind(param):
    p = param.strip()
    if '*' in p or '[' in p:
        return 'ptr'
    p = re.sub(r'\b(const|enum|struct)\b', '', p).split()
    if p[:2] == ['long', 'long']:
        return 'll'
    return {'int': 'int', 'unsigned': 'uint', 'double': 'double', 'void': 'void', 'size_t': 'size'}[p[0]]


def _ctypes_kind(t):
    if t is None:
        return 'void'
    if t in (C.c_void_p, C.c_char_p) or hasattr(t, '_type_') and isinstance(t._type_, type):
        return 'ptr'
    return {C.c_int: 'int', C.c_uint: 'uint', C.c_double: 'double', C.c_longlong: 'll', C.c_size_t: 'size'}[t]


def test_binding_signatures_match_the_header():
    """Argument count and kinds (pointer, int, unsigned, long long, double)
    and the return kind of every prototype in the header against the
    binding's ctypes declarations."""
    src = re.sub(r'/\*.*?\*/', '', open(os.path.join(ROOT, 'include', 'hemo.h')).read(), flags=re.S)
    protos = re.findall(r'\b(int|void|const char\s*\*)\s*(hemo_[a-z0-9_]+)\s*\(([^)]*)\)\s*;', src)
    assert len(protos) == len(header_functions())
    L = hemo.lib()
    for ret, name, params in protos:
        fn = getattr(L, name)
        want = [] if params.strip() in ('', 'void') else [_c_kind(p) for p in params.split(',')]
        assert [_ctypes_kind(t) for t in fn.argtypes] == want, name
        assert _ctypes_kind(fn.restype) == ('ptr' if '*' in ret else _c_kind(ret)), name


def test_bounds_checked_library_is_built():
    """build() also makes the bounds-checked library; it exports the same
    symbols."""
    from paper_2305_02752_gb300 import build as B
    assert os.path.exists(B.LIB_CHECKED)
    L = C.CDLL(B.LIB_CHECKED)
    for n in header_functions():
        assert hasattr(L, n), n
