"""Build libhemo.so in-tree for sm_103a with nvcc (translation units compiled
in parallel, then linked as a shared library against the shared CUDA
runtime), and its bounds-checked twin libhemo_checked.so (HEMO_BOUNDS_CHECK:
the data-driven indices of the vertex, bin and membrane kernels are tested
on the device; a failed test is reported through the status word)."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, 'csrc')
BUILD = os.path.join(HERE, '_build')
LIB = os.path.join(HERE, 'libhemo.so')
BUILD_CHECKED = os.path.join(HERE, '_build_checked')
LIB_CHECKED = os.path.join(HERE, 'libhemo_checked.so')
SOURCES = ['hemo_api.cu', 'k_lattice.cu', 'k_ibm.cu', 'k_membrane.cu', 'k_adjoint.cu', 'k_inside.cu', 'k_lees.cu']
HEADERS = [os.path.join(CSRC, 'hemo_internal.cuh'), os.path.join(CSRC, 'lattice_core.cuh'),
           os.path.join(os.path.dirname(HERE), 'include', 'hemo.h')]
ARCH = ['-gencode', 'arch=compute_103a,code=sm_103a']
FLAGS = ['-O3', '-lineinfo', '-std=c++17', '-Xcompiler', '-fPIC', '-Xcompiler', '-fno-strict-aliasing']


def nvcc() -> str:
    for cand in (os.environ.get('NVCC'), shutil.which('nvcc'), '/usr/local/cuda/bin/nvcc'):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError('nvcc not found')


def _cuda_lib_dir(nv: str) -> str:
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nv))), 'lib64')


def build(force: bool = False, verbose: bool = False, extra_flags=(), checked: bool = False) -> str:
    """Compile what changed and link; checked=True builds the bounds-checked
    library instead."""
    build_dir, lib = (BUILD_CHECKED, LIB_CHECKED) if checked else (BUILD, LIB)
    if checked:
        extra_flags = (*extra_flags, '-DHEMO_BOUNDS_CHECK=1')
    os.makedirs(build_dir, exist_ok=True)
    nv = nvcc()
    hdr_mtime = max(os.path.getmtime(h) for h in HEADERS)
    jobs = []
    objs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(build_dir, src.replace('.cu', '.o'))
        objs.append(o)
        if force or not os.path.exists(o) or os.path.getmtime(o) < max(os.path.getmtime(s), hdr_mtime):
            jobs.append([nv, *ARCH, *FLAGS, *extra_flags, '-c', s, '-o', o])

    def run(cmd):
        if verbose:
            print(' '.join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f'nvcc failed:\n{" ".join(cmd)}\n{r.stdout}\n{r.stderr}')
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr, flush=True)

    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            list(ex.map(run, jobs))
    if jobs or force or not os.path.exists(lib) or os.path.getmtime(lib) < max(os.path.getmtime(o) for o in objs):
        tmp = lib + f'.{os.getpid()}.tmp'
        run([nv, *ARCH, '-shared', '-cudart', 'shared', '-o', tmp, *objs,
             '-Xlinker', '-rpath=' + _cuda_lib_dir(nv)])
        os.replace(tmp, lib)
    return lib


def build_all(force: bool = False, verbose: bool = False) -> tuple:
    """Both libraries, built side by side."""
    with cf.ThreadPoolExecutor(max_workers=2) as ex:
        a = ex.submit(build, force, verbose)
        b = ex.submit(build, force, verbose, (), True)
        return a.result(), b.result()


if __name__ == '__main__':
    print(build_all(verbose=True))
