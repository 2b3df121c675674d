"""Python binding of libhemo (include/hemo.h): argument marshalling only.

Every step of the coupled lattice-Boltzmann / immersed-boundary time step
runs in the library's CUDA kernels.  The library is loaded from this package
directory; if it has not been built the import of the binding fails loudly
(there is no CPU fallback).  PyTorch provides device memory (through the
allocator callbacks below) and streams.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# HEMO_BOUNDS_CHECK=1 in the environment loads the bounds-checked build
LIB_PATH = os.path.join(_HERE, 'libhemo_checked.so' if os.environ.get('HEMO_BOUNDS_CHECK') == '1' else 'libhemo.so')

HEMO_OK, HEMO_ERR_ARG, HEMO_ERR_OOM, HEMO_ERR_CUDA, HEMO_ERR_NUMERIC, HEMO_ERR_DOMAIN, HEMO_ERR_STATE = \
    0, -1, -2, -3, -4, -5, -6
PRECISIONS = {'f64': 0, 'f32': 1, 'f16': 2, 'bf16': 3}
HEMO_RHO, HEMO_U, HEMO_VERTS, HEMO_FORCES, HEMO_CELLSTATS = 1, 2, 4, 8, 16

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class hemo_lattice_desc(C.Structure):
    _fields_ = [('nx', C.c_int), ('ny', C.c_int), ('nz', C.c_int), ('tau', C.c_double),
                ('precision', C.c_int), ('periodic', C.c_int * 3), ('wall_mask', C.c_void_p),
                ('wall_velocity', (C.c_double * 3) * 2), ('body_force', C.c_double * 3),
                ('cuda_stream', C.c_void_p), ('alloc', ALLOC_FN), ('release', FREE_FN),
                ('alloc_ctx', C.c_void_p), ('options', C.c_uint)]

HEMO_OPT_STAGED_COLLISION = 1
HEMO_OPT_NODE_COLLISION = 2
HEMO_OPT_TEST_STALLED_WAIT = 4
HEMO_OPT_PAIR_COLLISION = 8
HEMO_OPT_WIDE_INDEX = 16
HEMO_OPT_NODE_STAGING = 32
HEMO_OPT_UNSTAGED_COLLISION = 64
HEMO_EULER, HEMO_AB2 = 0, 1
INTEGRATORS = {'euler': HEMO_EULER, 'ab2': HEMO_AB2}


class hemo_mesh_desc(C.Structure):
    _fields_ = [('nv', C.c_int), ('nt', C.c_int), ('tri', C.c_void_p), ('rest_xyz', C.c_void_p),
                ('k_link', C.c_double), ('k_bend', C.c_double), ('k_area', C.c_double),
                ('k_volume', C.c_double), ('kbt', C.c_double), ('persistence', C.c_double),
                ('max_strain', C.c_double), ('k_local', C.c_double), ('theta_m', C.c_double)]


class HemoError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f'hemo error {code}: {msg}')
        self.code = code


_lib = None


def lib():
    """Load libhemo.so (raises if it is missing: build it with
    `python -c "import __graft_entry__ as g; g.build()"`)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f'{LIB_PATH} is missing: the CUDA library must be built first '
                          '(python -c "import __graft_entry__ as g; g.build()")')
    L = C.CDLL(LIB_PATH)
    vp, i, ll, d = C.c_void_p, C.c_int, C.c_longlong, C.c_double
    sig = {
        'hemo_create_lattice': ([C.POINTER(hemo_lattice_desc), C.POINTER(vp)], i),
        'hemo_set_velocity': ([vp, vp], i),
        'hemo_add_cells': ([vp, C.POINTER(hemo_mesh_desc), i, vp, vp, C.POINTER(i)], i),
        'hemo_step': ([vp, i], i),
        'hemo_set_time_scales': ([vp, i, i], i),
        'hemo_set_force_tolerance': ([vp, d], i),
        'hemo_get_force_evaluations': ([vp, C.POINTER(ll)], i),
        'hemo_set_viscosity_ratio': ([vp, d], i),
        'hemo_set_lees_edwards': ([vp, d], i),
        'hemo_get_inside': ([vp, vp], i),
        'hemo_sync': ([vp], i),
        'hemo_get_fields': ([vp, C.c_uint, vp, vp, vp, vp, vp], i),
        'hemo_get_sizes': ([vp, C.POINTER(ll), C.POINTER(ll), C.POINTER(i), C.POINTER(i)], i),
        'hemo_get_lattice_plan': ([vp, vp], i),
        'hemo_velocity_set': ([vp, vp], i),
        'hemo_get_populations': ([vp, vp], i),
        'hemo_get_links': ([vp, vp], i),
        'hemo_get_edges': ([vp, i, vp, C.POINTER(i)], i),
        'hemo_set_vertices': ([vp, vp], i),
        'hemo_get_bins': ([vp, vp, vp, vp], i),
        'hemo_set_phase_timing': ([vp, i], i),
        'hemo_get_phase_times': ([vp, vp, C.POINTER(i)], i),
        'hemo_bin_vertices_noalloc': ([vp, i, i, i, i, vp, vp, vp, vp, vp], i),
        'hemo_state_bytes': ([vp, C.POINTER(C.c_size_t)], i),
        'hemo_save_state': ([vp, vp, C.c_size_t], i),
        'hemo_load_state': ([vp, vp, C.c_size_t], i),
        'hemo_record': ([vp, i], i),
        'hemo_deformation_loss': ([vp, vp, vp], i),
        'hemo_backward': ([vp, vp, vp, i], i),
        'hemo_destroy': ([vp], None),
        'hemo_last_error': ([], C.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def exported_symbols():
    """Names the header declares (used by the load test)."""
    return ['hemo_create_lattice', 'hemo_set_velocity', 'hemo_add_cells', 'hemo_step', 'hemo_set_time_scales',
            'hemo_set_force_tolerance', 'hemo_get_force_evaluations',
            'hemo_set_viscosity_ratio', 'hemo_get_inside', 'hemo_set_lees_edwards', 'hemo_sync',
            'hemo_get_fields', 'hemo_get_sizes', 'hemo_get_lattice_plan', 'hemo_velocity_set', 'hemo_get_populations',
            'hemo_get_links', 'hemo_get_edges', 'hemo_set_vertices', 'hemo_get_bins',
            'hemo_set_phase_timing', 'hemo_get_phase_times', 'hemo_bin_vertices_noalloc', 'hemo_state_bytes',
            'hemo_save_state', 'hemo_load_state', 'hemo_record',
            'hemo_deformation_loss', 'hemo_backward', 'hemo_destroy', 'hemo_last_error']


def check(rc):
    if rc != HEMO_OK:
        raise HemoError(rc, lib().hemo_last_error().decode())
    return rc


def bin_vertices_noalloc(verts, dims, periodic, key, perm, start, stream=None, _require_cuda=True):
    """Bin absolute vertex positions without any allocation by the library
    (for callers that cannot let it allocate device memory).  verts: CUDA
    float64 tensor [nv, 3]; key, perm: CUDA int32 [nv]; start: CUDA int32
    [nbins + 1] with nbins = ceil(nx/8) ceil(ny/8) ceil(nz/8), all
    caller-owned and contiguous.  Same binning as Simulation.bins() for
    absolute FP64 positions; asynchronous on `stream` (default: current
    stream).  The C ABI receives bare pointers and cannot check the buffers,
    so their types, devices and sizes are checked here (HemoError with
    HEMO_ERR_ARG)."""
    import torch
    nx, ny, nz = (int(x) for x in dims)
    nb = [(n + 7) // 8 for n in (nx, ny, nz)]
    nbins = nb[0] * nb[1] * nb[2]

    def need(ok, what):
        if not ok:
            raise HemoError(HEMO_ERR_ARG, f'bin_vertices_noalloc: {what}')

    def tensor(t, name, dtype, min_numel):
        need(isinstance(t, torch.Tensor), f'{name} must be a torch tensor')
        need(t.dtype == dtype, f'{name} must be {dtype}')
        need(t.is_contiguous(), f'{name} must be contiguous')
        need(not _require_cuda or t.is_cuda, f'{name} must be a CUDA tensor')
        need(t.numel() >= min_numel, f'{name} needs at least {min_numel} entries')

    need(isinstance(verts, torch.Tensor) and verts.dim() == 2 and verts.shape[1] == 3, 'verts must be [nv, 3]')
    nv = int(verts.shape[0])
    tensor(verts, 'verts', torch.float64, 3 * nv)
    tensor(key, 'key', torch.int32, nv)
    tensor(perm, 'perm', torch.int32, nv)
    tensor(start, 'start', torch.int32, nbins + 1)
    per = np.ascontiguousarray(periodic, dtype=np.int32)
    need(per.shape == (3,), 'periodic must have 3 entries')
    st = (stream or torch.cuda.current_stream()).cuda_stream
    check(lib().hemo_bin_vertices_noalloc(verts.data_ptr(), int(verts.shape[0]), nx, ny, nz, per.ctypes.data,
                                          key.data_ptr(), perm.data_ptr(), start.data_ptr(), st))


def velocity_set():
    c = np.zeros((19, 3), np.int32)
    w = np.zeros(19)
    check(lib().hemo_velocity_set(c.ctypes.data, w.ctypes.data))
    return c, w


def _ptr(a):
    """Data pointer of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


class Simulation:
    """One coupled LBM-IBM simulation on the current CUDA device."""

    def __init__(self, nx, ny, nz, tau=1.0, precision='f32', periodic=(1, 1, 1), wall_mask=None,
                 wall_velocity=None, body_force=None, stream=None, torch_allocator=True, options=0):
        import torch
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        self.precision = precision
        self._rdtype = np.float64 if precision == 'f64' else np.float32
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        d = hemo_lattice_desc()
        d.nx, d.ny, d.nz = nx, ny, nz
        d.tau = tau
        d.precision = PRECISIONS[precision]
        for k in range(3):
            d.periodic[k] = int(periodic[k])
        self._mask = None
        if wall_mask is not None:
            self._mask = np.ascontiguousarray(wall_mask, dtype=np.uint8).reshape(-1)
            assert self._mask.size == self.N
            d.wall_mask = self._mask.ctypes.data
        wv = np.zeros((2, 3)) if wall_velocity is None else np.asarray(wall_velocity, float)
        for a in range(2):
            for b in range(3):
                d.wall_velocity[a][b] = wv[a, b]
        g = np.zeros(3) if body_force is None else np.asarray(body_force, float)
        for k in range(3):
            d.body_force[k] = g[k]
        d.cuda_stream = self._stream.cuda_stream
        d.options = int(options)
        if torch_allocator:
            dev = torch.cuda.current_device()
            stream = self._stream

            def _alloc(nbytes, ctx):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream)
                except Exception:
                    return None

            def _free(ptr, ctx):
                torch.cuda.caching_allocator_delete(ptr)

            self._alloc_cb = ALLOC_FN(_alloc)
            self._free_cb = FREE_FN(_free)
            d.alloc = self._alloc_cb
            d.release = self._free_cb
        self._desc = d
        self.handle = C.c_void_p()
        check(lib().hemo_create_lattice(C.byref(d), C.byref(self.handle)))
        self._meshes = []

    # -- construction ------------------------------------------------------
    @classmethod
    def from_config(cls, cfg, precision='f32', **kw):
        s = cls(cfg.nx, cfg.ny, cfg.nz, cfg.tau, precision, cfg.periodic, cfg.mask, cfg.wall_velocity,
                cfg.body_force, **kw)
        if cfg.init_velocity is not None:
            s.set_velocity(cfg.init_velocity)
        types = np.asarray(cfg.cell_type)
        # cells are added in configuration order (one call per run of equal
        # type) so the global vertex numbering is the configuration's
        runs = []
        for k, t in enumerate(types):
            if runs and runs[-1][0] == t:
                runs[-1][1].append(k)
            else:
                runs.append((t, [k]))
        for t, idx in runs:
            s.add_cells(cfg.meshes[t], cfg.centers[idx], cfg.rotations[idx])
        if not runs:
            for mt in cfg.meshes:
                s.add_cells(mt, np.zeros((0, 3)), np.zeros((0, 3, 3)))
        return s

    def set_velocity(self, u):
        if u is None:
            check(lib().hemo_set_velocity(self.handle, None))
        else:
            u = np.ascontiguousarray(u, dtype=np.float64)
            assert u.size == 3 * self.N
            check(lib().hemo_set_velocity(self.handle, u.ctypes.data))

    def add_cells(self, mesh, centers, rots):
        """Add cells of one mesh type (an `inputs.MeshType`)."""
        tri = np.ascontiguousarray(mesh.tri, dtype=np.int32)
        rest = np.ascontiguousarray(mesh.rest, dtype=np.float64)
        centers = np.ascontiguousarray(centers, dtype=np.float64).reshape(-1, 3)
        rots = np.ascontiguousarray(rots, dtype=np.float64).reshape(-1, 3, 3)
        m = hemo_mesh_desc(len(rest), len(tri), tri.ctypes.data, rest.ctypes.data, mesh.k_link, mesh.k_bend,
                           mesh.k_area, mesh.k_volume, mesh.kbt, mesh.persistence, mesh.max_strain,
                           getattr(mesh, 'k_local', 0.0), getattr(mesh, 'theta_m', 0.0))
        first = C.c_int(-1)
        check(lib().hemo_add_cells(self.handle, C.byref(m), len(centers), centers.ctypes.data,
                                   rots.ctypes.data, C.byref(first)))
        self._meshes.append(mesh)
        return first.value

    # -- stepping ----------------------------------------------------------
    def step(self, n=1):
        check(lib().hemo_step(self.handle, int(n)))

    def set_time_scales(self, force_every=1, integrator='euler'):
        """Membrane forces every `force_every` steps, held in between, and
        the vertex integrator 'euler' or 'ab2' (Sec. 2.6), from this step on."""
        check(lib().hemo_set_time_scales(self.handle, int(force_every), INTEGRATORS[integrator]))

    def set_force_tolerance(self, delta):
        """Adaptive separation: evaluate the membrane forces when a vertex
        has moved more than delta since the last evaluation (or
        force_every steps have passed); delta < 0: constant schedule."""
        check(lib().hemo_set_force_tolerance(self.handle, float(delta)))

    @property
    def force_evaluations(self):
        """Membrane-force evaluations since creation (every schedule)."""
        n = C.c_longlong(0)
        check(lib().hemo_get_force_evaluations(self.handle, C.byref(n)))
        return n.value

    def set_viscosity_ratio(self, ratio):
        """Viscosity inside cells relative to the plasma (1 = off): inside
        nodes relax with tau_in = 1/2 + ratio (tau - 1/2)."""
        check(lib().hemo_set_viscosity_ratio(self.handle, float(ratio)))

    def set_lees_edwards(self, U):
        """Lees-Edwards boundary along z with image velocity U (before the
        first step; lattice periodic on every axis without walls)."""
        check(lib().hemo_set_lees_edwards(self.handle, float(U)))

    def inside(self):
        """Inside/outside indicator of the current vertex positions [z, y, x]."""
        out = np.zeros(self.shape, np.uint8)
        check(lib().hemo_get_inside(self.handle, out.ctypes.data))
        return out

    def sync(self):
        return check(lib().hemo_sync(self.handle))

    def sizes(self):
        n, v, c, b = C.c_longlong(), C.c_longlong(), C.c_int(), C.c_int()
        check(lib().hemo_get_sizes(self.handle, C.byref(n), C.byref(v), C.byref(c), C.byref(b)))
        return n.value, v.value, c.value, b.value

    def lattice_plan(self):
        """(tiles staged through shared memory, rows for the per-node
        kernel, rows per tile, ring stages); zeros without staging."""
        plan = (C.c_int * 4)()
        check(lib().hemo_get_lattice_plan(self.handle, plan))
        return tuple(plan)

    # -- read-out ----------------------------------------------------------
    def get_fields(self, what=HEMO_RHO | HEMO_U | HEMO_VERTS | HEMO_FORCES | HEMO_CELLSTATS, out=None):
        """Copy fields to host numpy arrays (or into the given host/device
        buffers `out` = dict of arrays or tensors)."""
        _, nv, nc, _ = self.sizes()
        out = dict(out or {})
        if what & HEMO_RHO and 'rho' not in out:
            out['rho'] = np.zeros(self.shape, self._rdtype)
        if what & HEMO_U and 'u' not in out:
            out['u'] = np.zeros(self.shape + (3,), self._rdtype)
        if what & HEMO_VERTS and 'X' not in out:
            out['X'] = np.zeros((nv, 3))
        if what & HEMO_FORCES and 'Fv' not in out:
            out['Fv'] = np.zeros((nv, 3))
        if what & HEMO_CELLSTATS and 'cellstats' not in out:
            out['cellstats'] = np.zeros((nc, 6))
        check(lib().hemo_get_fields(self.handle, what, _ptr(out.get('rho')), _ptr(out.get('u')),
                                    _ptr(out.get('X')), _ptr(out.get('Fv')), _ptr(out.get('cellstats'))))
        return out

    def populations(self):
        f = np.zeros(self.shape + (19,))
        check(lib().hemo_get_populations(self.handle, f.ctypes.data))
        return f

    def links(self):
        out = np.zeros(self.shape, np.uint64)
        check(lib().hemo_get_links(self.handle, out.ctypes.data))
        return out

    def edges(self, type_id):
        mesh = self._meshes[type_id]
        buf = np.zeros(4 * (3 * len(mesh.tri) // 2 + 1), np.int32)
        ne = C.c_int()
        check(lib().hemo_get_edges(self.handle, int(type_id), buf.ctypes.data, C.byref(ne)))
        return buf[:4 * ne.value].reshape(-1, 4)

    def set_vertices(self, X):
        X = np.ascontiguousarray(X, dtype=np.float64)
        check(lib().hemo_set_vertices(self.handle, X.ctypes.data))

    def bins(self):
        _, nv, _, nb = self.sizes()
        key = np.zeros(nv, np.int32)
        perm = np.zeros(nv, np.int32)
        start = np.zeros(nb + 1, np.int32)
        check(lib().hemo_get_bins(self.handle, key.ctypes.data, perm.ctypes.data, start.ctypes.data))
        return key, perm, start

    # -- checkpoint and resume -------------------------------------------
    def save_state(self):
        """The simulation's dynamic state as a host byte array (see
        hemo_save_state)."""
        n = C.c_size_t()
        check(lib().hemo_state_bytes(self.handle, C.byref(n)))
        buf = np.zeros(n.value, np.uint8)
        check(lib().hemo_save_state(self.handle, buf.ctypes.data, n.value))
        return buf

    def load_state(self, buf):
        """Continue from a state saved by save_state() of a simulation
        created and filled with cells the same way."""
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        check(lib().hemo_load_state(self.handle, buf.ctypes.data, buf.size))

    # -- differentiation form --------------------------------------------
    def record(self, checkpoint_every=100):
        check(lib().hemo_record(self.handle, int(checkpoint_every)))

    def deformation_loss(self):
        """(loss, dL/dX [nv, 3]) of the current vertices."""
        _, nv, _, _ = self.sizes()
        loss = np.zeros(1)
        g = np.zeros((nv, 3))
        check(lib().hemo_deformation_loss(self.handle, loss.ctypes.data, g.ctypes.data))
        return float(loss[0]), g

    def backward(self, dL_dX):
        """Gradient of a loss of the current vertices with respect to the
        recorded steps' parameters: per mesh type (k_link, k_bend, k_area,
        k_volume), then the wall-velocity scale and g (3)."""
        dL = np.ascontiguousarray(dL_dX, dtype=np.float64)
        ng = 4 * len(self._meshes) + 4
        out = np.zeros(ng)
        check(lib().hemo_backward(self.handle, dL.ctypes.data, out.ctypes.data, ng))
        return out

    PHASES = ('membrane', 'bins', 'spread', 'collide', 'moments', 'interp')

    def set_phase_timing(self, on=True):
        check(lib().hemo_set_phase_timing(self.handle, int(bool(on))))

    def phase_times(self):
        """Device ms of each phase of the most recent step, and the kernel
        launches per step."""
        ms = np.zeros(len(self.PHASES), np.float32)
        k = C.c_int()
        check(lib().hemo_get_phase_times(self.handle, ms.ctypes.data, C.byref(k)))
        return dict(zip(self.PHASES, ms.astype(float))), k.value

    def close(self):
        if getattr(self, 'handle', None) and self.handle.value:
            lib().hemo_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# torch.autograd wrapper
# ---------------------------------------------------------------------------
def parameter_vector(cfg):
    """Parameters in the order of the gradient: per mesh type (k_link,
    k_bend, k_area, k_volume), wall-velocity scale (1), body force (3)."""
    vals = []
    for mt in cfg.meshes:
        vals += [mt.k_link, mt.k_bend, mt.k_area, mt.k_volume]
    return np.array(vals + [1.0] + list(np.asarray(cfg.body_force, float)))


def config_with(cfg, params):
    """Copy of an input configuration with the parameters replaced."""
    import copy
    c = copy.deepcopy(cfg)
    p = np.asarray(params, float)
    for t, mt in enumerate(c.meshes):
        mt.k_link, mt.k_bend, mt.k_area, mt.k_volume = (float(x) for x in p[4 * t:4 * t + 4])
    k = 4 * len(c.meshes)
    c.wall_velocity = np.asarray(cfg.wall_velocity, float) * p[k]
    c.body_force = p[k + 1:k + 4].copy()
    return c


def coupled_run(cfg, steps, precision='f64', checkpoint_every=100):
    """A torch.autograd.Function mapping the parameter vector (see
    parameter_vector) to the final vertex positions after `steps` coupled
    steps; backward runs hemo_backward."""
    import torch

    class CoupledRun(torch.autograd.Function):
        @staticmethod
        def forward(ctx, params):
            sim = Simulation.from_config(config_with(cfg, params.detach().cpu().numpy()), precision)
            sim.record(checkpoint_every)
            sim.step(steps)
            X = sim.get_fields(HEMO_VERTS)['X']
            ctx.sim = sim
            ctx.device = params.device
            return torch.from_numpy(X).to(params.device)

        @staticmethod
        def backward(ctx, dX):
            g = ctx.sim.backward(dX.detach().cpu().numpy())
            ctx.sim.close()
            return torch.from_numpy(g).to(ctx.device)

    return CoupledRun.apply
