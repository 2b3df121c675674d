"""Python wrapper of the CPU oracle (plain FP64 C, `hemo_oracle.c`).

TEST INFRASTRUCTURE ONLY: used by the test-suite, by the smoke check and by
the benchmark's CPU-baseline / reference leg.  It imports nothing from the
CUDA package; both receive the same inputs from the seeded input generators.

Every function cites the paper passage it follows in `hemo_oracle.c`.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, 'hemo_oracle.c')
_LIB = os.path.join(_HERE, 'libhemo_oracle.so')
_lib = None

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags='C_CONTIGUOUS')
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags='C_CONTIGUOUS')
_up = np.ctypeslib.ndpointer(dtype=np.uint32, flags='C_CONTIGUOUS')
_bp = np.ctypeslib.ndpointer(dtype=np.uint8, flags='C_CONTIGUOUS')


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, strict IEEE: no fast-math and
    no FMA contraction, so x86 and Arm hosts give the same results), with
    OpenMP where the compiler has it."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f'.{os.getpid()}.tmp'
        base = ['gcc', '-O2', '-std=c99', '-fPIC', '-shared', '-ffp-contract=off', '-o', tmp, _SRC, '-lm']
        try:
            subprocess.check_call(base[:1] + ['-fopenmp'] + base[1:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        L.ora_d3q19.argtypes = [_ip, _dp, _ip]
        L.ora_equilibrium.argtypes = [C.c_double, _dp, _dp]
        L.ora_storage_reference.argtypes = [C.c_double, _dp]
        L.ora_set_force_tolerance.argtypes = [C.c_void_p, C.c_double]
        L.ora_set_force_tolerance.restype = C.c_int
        L.ora_force_evaluations.argtypes = [C.c_void_p]
        L.ora_force_evaluations.restype = C.c_long
        L.ora_phi.argtypes = [C.c_double]
        L.ora_phi.restype = C.c_double
        L.ora_build_edges.argtypes = [C.c_int, C.c_int, _ip, _ip]
        L.ora_build_edges.restype = C.c_int
        L.ora_membrane.argtypes = [C.c_int, C.c_int, _ip, _dp, _dp, _dp, _dp, _dp, _dp]
        L.ora_membrane.restype = C.c_int
        L.ora_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, _ip, C.c_void_p, _dp, _dp]
        L.ora_create.restype = C.c_void_p
        L.ora_destroy.argtypes = [C.c_void_p]
        L.ora_add_mesh.argtypes = [C.c_void_p, C.c_int, C.c_int, _ip, _dp, _dp]
        L.ora_add_mesh.restype = C.c_int
        L.ora_add_cells.argtypes = [C.c_void_p, C.c_int, C.c_int, _dp, _dp, _dp]
        L.ora_add_cells.restype = C.c_int
        L.ora_set_vertices.argtypes = [C.c_void_p, _dp]
        L.ora_set_velocity.argtypes = [C.c_void_p, C.c_void_p]
        L.ora_wall_links.argtypes = [C.c_void_p, _up]
        L.ora_step.argtypes = [C.c_void_p, C.c_int]
        L.ora_set_time_scales.argtypes = [C.c_void_p, C.c_int, C.c_int]
        L.ora_set_time_scales.restype = C.c_int
        L.ora_get.argtypes = [C.c_void_p] + [C.c_void_p] * 6
        L.ora_get_populations.argtypes = [C.c_void_p, _dp]
        L.ora_spread.argtypes = [C.c_void_p, C.c_long, _dp, _dp, _dp]
        L.ora_interpolate.argtypes = [C.c_void_p, C.c_long, _dp, _dp, _dp]
        L.ora_bins.argtypes = [C.c_void_p, C.c_long, _dp, C.c_int, _ip, _ip, _ip]
        L.ora_bins.restype = C.c_int
        L.ora_deformation_index.argtypes = [_dp, C.c_int]
        L.ora_deformation_index.restype = C.c_double
        L.ora_loss.argtypes = [C.c_void_p]
        L.ora_loss.restype = C.c_double
        L.ora_num_vertices.argtypes = [C.c_void_p]
        L.ora_num_vertices.restype = C.c_long
        L.ora_num_cells.argtypes = [C.c_void_p]
        L.ora_num_cells.restype = C.c_int
        L.ora_inside.argtypes = [C.c_void_p, _bp]
        L.ora_set_viscosity_ratio.argtypes = [C.c_void_p, C.c_double]
        L.ora_set_viscosity_ratio.restype = C.c_int
        L.ora_force_inside.argtypes = [C.c_void_p, C.c_void_p]
        L.ora_set_lees_edwards.argtypes = [C.c_void_p, C.c_double]
        L.ora_set_lees_edwards.restype = C.c_int
        L.ora_set_threads.argtypes = [C.c_int]
        L.ora_get_threads.restype = C.c_int
        L.ora_set_threads(1)
        _lib = L
    return _lib


INTEGRATORS = {'euler': 0, 'ab2': 1}


def set_threads(n: int) -> int:
    """Threads of the oracle's loops over independent nodes, cells and
    vertices (1 unless set; results do not depend on it).  Returns the
    number in effect (1 when the oracle was built without OpenMP)."""
    lib().ora_set_threads(int(n))
    return lib().ora_get_threads()


def _c(a, dt=np.float64):
    return np.ascontiguousarray(a, dtype=dt)


# ---------------------------------------------------------------------------
# pieces (pins)
# ---------------------------------------------------------------------------
def d3q19():
    c = np.zeros(57, np.int32)
    w = np.zeros(19)
    o = np.zeros(19, np.int32)
    lib().ora_d3q19(c, w, o)
    return c.reshape(19, 3), w, o


def equilibrium(rho, u):
    out = np.zeros(19)
    lib().ora_equilibrium(float(rho), _c(u), out)
    return out


def storage_reference(U):
    """K_i of the 16-bit storage form for a row reference velocity (U, 0, 0):
    f_i^eq(1, (U, 0, 0)) - w_i where c_i,x != 0, else 0 (oracle order)."""
    out = np.zeros(19)
    lib().ora_storage_reference(float(U), out)
    return out


def phi(r):
    return np.array([lib().ora_phi(float(x)) for x in np.ravel(r)]).reshape(np.shape(r))


def build_edges(nv, tri):
    tri = _c(tri, np.int32)
    out = np.zeros(4 * (3 * len(tri) // 2 + 1), np.int32)
    ne = lib().ora_build_edges(int(nv), len(tri), tri.ravel(), out)
    if ne < 0:
        raise ValueError('mesh is not an oriented closed 2-manifold')
    return out[:4 * ne].reshape(ne, 4)


def membrane_params(mt):
    """[k_link, k_bend, k_area, k_volume, kbt, persistence, max_strain,
    k_local, theta_m] of a mesh type (the last two 0 unless set)."""
    return np.array([mt.k_link, mt.k_bend, mt.k_area, mt.k_volume, mt.kbt, mt.persistence,
                     mt.max_strain, getattr(mt, 'k_local', 0.0), getattr(mt, 'theta_m', 0.0)], float)


def _params9(params):
    p = np.zeros(9)
    p[:len(params)] = params
    return p


def membrane(rest, tri, params, X):
    """Forces [nv, 3], energies (link, bend, area, volume), (A, V, A0, V0)."""
    rest = _c(rest)
    tri = _c(tri, np.int32)
    F = np.zeros(rest.size)
    E = np.zeros(4)
    AV = np.zeros(4)
    rc = lib().ora_membrane(len(rest), len(tri), tri.ravel(), rest.ravel(), _params9(params),
                            _c(X).ravel(), F, E, AV)
    if rc != 0:
        raise ValueError('bad mesh')
    return F.reshape(-1, 3), E, AV


def deformation_index(X):
    X = _c(X)
    return lib().ora_deformation_index(X.ravel(), len(X))


# ---------------------------------------------------------------------------
# simulation
# ---------------------------------------------------------------------------
class OracleSim:
    """FP64 CPU reference of the coupled step; fields indexed [z, y, x]."""

    def __init__(self, nx, ny, nz, tau, periodic, mask=None, wall_velocity=None, body_force=None):
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        self._mask = None if mask is None else _c(mask, np.uint8).ravel()
        wv = _c(np.zeros((2, 3)) if wall_velocity is None else wall_velocity).ravel()
        g = _c(np.zeros(3) if body_force is None else body_force)
        mptr = None if self._mask is None else self._mask.ctypes.data
        self.h = lib().ora_create(nx, ny, nz, float(tau), _c(periodic, np.int32), mptr, wv, g)
        self._rest = []

    def close(self):
        if self.h:
            lib().ora_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_mesh(self, rest, tri, params):
        t = lib().ora_add_mesh(self.h, len(rest), len(tri), _c(tri, np.int32).ravel(),
                               _c(rest).ravel(), _params9(params))
        if t < 0:
            raise ValueError('bad mesh')
        self._rest.append(_c(rest))
        return t

    def add_cells(self, type_id, centers, rots):
        centers = _c(centers).reshape(-1, 3)
        rots = _c(rots).reshape(-1, 3, 3)
        rc = lib().ora_add_cells(self.h, int(type_id), len(centers), centers.ravel(), rots.ravel(),
                                 self._rest[type_id].ravel())
        if rc != 0:
            raise ValueError('bad cell type')

    def set_velocity(self, u):
        if u is None:
            lib().ora_set_velocity(self.h, None)
        else:
            self._u0 = _c(u).ravel()
            lib().ora_set_velocity(self.h, self._u0.ctypes.data)

    def set_vertices(self, X):
        lib().ora_set_vertices(self.h, _c(X).ravel())

    def set_time_scales(self, force_every=1, integrator='euler'):
        """Membrane forces every `force_every` steps (held in between) and
        the vertex integrator, 'euler' or 'ab2' (Sec. 2.6)."""
        rc = lib().ora_set_time_scales(self.h, int(force_every), INTEGRATORS[integrator])
        if rc != 0:
            raise ValueError('force_every must be >= 1')

    def set_force_tolerance(self, delta):
        """Adaptive separation: from the next step the membrane forces are
        evaluated on the first step, then whenever the largest vertex
        displacement since the last evaluation exceeds delta at the start of
        a step, or force_every steps have passed; delta < 0: the constant
        schedule."""
        if lib().ora_set_force_tolerance(self.h, float(delta)) != 0:
            raise ValueError('delta must not be NaN')

    @property
    def force_evaluations(self):
        return lib().ora_force_evaluations(self.h)

    def set_lees_edwards(self, U):
        """Lees-Edwards boundary along z: the image above the box is displaced
        by U n (mod nx) in x at step n and moves with U x^ (before the first
        step; fully periodic lattice without walls)."""
        if lib().ora_set_lees_edwards(self.h, float(U)) != 0:
            raise ValueError('Lees-Edwards needs a fully periodic lattice without walls, before the first step')

    def set_viscosity_ratio(self, ratio):
        """Internal viscosity ratio: nodes inside cells relax with
        tau_in = 1/2 + ratio (tau - 1/2); 1 = off."""
        if lib().ora_set_viscosity_ratio(self.h, float(ratio)) != 0:
            raise ValueError('ratio must be > 0')

    def inside(self):
        """Inside/outside indicator of the current vertex positions [z, y, x]."""
        out = np.zeros(self.N, np.uint8)
        lib().ora_inside(self.h, out)
        return out.reshape(self.shape)

    def force_inside(self, ind):
        """Tests: use the given indicator instead of the cells' (None: back
        to the cells')."""
        if ind is None:
            lib().ora_force_inside(self.h, None)
        else:
            self._forced = _c(ind, np.uint8).ravel()
            lib().ora_force_inside(self.h, self._forced.ctypes.data)

    def step(self, n=1):
        lib().ora_step(self.h, int(n))

    @property
    def n_vertices(self):
        return lib().ora_num_vertices(self.h)

    @property
    def n_cells(self):
        return lib().ora_num_cells(self.h)

    def get(self):
        nv = self.n_vertices
        rho = np.zeros(self.N)
        u = np.zeros(3 * self.N)
        X = np.zeros(3 * nv)
        Fv = np.zeros(3 * nv)
        cs = np.zeros(6 * self.n_cells)
        disc = np.zeros(3)
        lib().ora_get(self.h, rho.ctypes.data, u.ctypes.data, X.ctypes.data, Fv.ctypes.data,
                      cs.ctypes.data, disc.ctypes.data)
        return dict(rho=rho.reshape(self.shape), u=u.reshape(self.shape + (3,)),
                    X=X.reshape(-1, 3), Fv=Fv.reshape(-1, 3), cellstats=cs.reshape(-1, 6),
                    discarded=disc)

    def populations(self):
        f = np.zeros(19 * self.N)
        lib().ora_get_populations(self.h, f)
        return f.reshape(self.shape + (19,))

    def wall_links(self):
        out = np.zeros(self.N, np.uint32)
        lib().ora_wall_links(self.h, out)
        return out.reshape(self.shape)

    def spread(self, X, Fv):
        X = _c(X)
        out = np.zeros(3 * self.N)
        lib().ora_spread(self.h, len(X), X.ravel(), _c(Fv).ravel(), out)
        return out.reshape(self.shape + (3,))

    def interpolate(self, X, u):
        X = _c(X)
        out = np.zeros(X.size)
        lib().ora_interpolate(self.h, len(X), X.ravel(), _c(u).ravel(), out)
        return out.reshape(-1, 3)

    def bins(self, X, B=8):
        X = _c(X)
        nz, ny, nx = self.shape
        nb = ((nx + B - 1) // B) * ((ny + B - 1) // B) * ((nz + B - 1) // B)
        key = np.zeros(len(X), np.int32)
        perm = np.zeros(len(X), np.int32)
        start = np.zeros(nb + 1, np.int32)
        lib().ora_bins(self.h, len(X), X.ravel(), int(B), key, perm, start)
        return key, perm, start

    def loss(self):
        return lib().ora_loss(self.h)


def from_config(cfg, steps=None):
    """Build an oracle simulation from an input configuration."""
    s = OracleSim(cfg.nx, cfg.ny, cfg.nz, cfg.tau, cfg.periodic, cfg.mask, cfg.wall_velocity,
                  cfg.body_force)
    for mt in cfg.meshes:
        s.add_mesh(mt.rest, mt.tri, membrane_params(mt))
    # cells are added in configuration order, one at a time, so the global
    # vertex numbering is the configuration's cell order
    for t, c, r in zip(cfg.cell_type, cfg.centers, cfg.rotations):
        s.add_cells(int(t), c[None], r[None])
    s.set_velocity(cfg.init_velocity)
    return s
