"""Seeded synthetic inputs for the coupled lattice-Boltzmann / immersed-boundary step.

This module is shared by the CUDA path and by the CPU oracle: it produces the
*inputs* of a simulation (membrane meshes at rest, cell placements, wall masks,
initial velocity profiles, model parameters) and nothing of the method's own
arithmetic.  Rest lengths, rest angles, rest area and volume, edge tables,
wall links, binning, forces and the time step are computed independently by
each side from these inputs.

Workloads follow the paper's physiological settings: red blood cells (RBCs)
with the biconcave shape and haematocrits of Section 1, platelets as small
oblate spheroids, a parallel-plate shear cell (Section 2.5, periodic in two
directions), a wall-bounded periodic channel and a straight periodic pipe
(Section 3, diabetic-blood study geometry).  Initial placements use random
uniform positions and orientations (Section 2.4) relaxed by a force-bias
repulsion proportional to an overlap estimate of bounding ellipsoids
(Section 2.4, force-bias equation).

Units are lattice units (LU): dx = 1, dt = 1.  With the plasma properties
below, dx = 0.5 um and tau = 1 give dt = 3.788e-8 s.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

# ---------------------------------------------------------------------------
# physical parameters (inputs, not method arithmetic)
# ---------------------------------------------------------------------------
DX_UM = 0.5                    # lattice spacing in micrometres
PLASMA_RHO = 1025.0            # kg / m^3
PLASMA_NU = 1.1e-6             # m^2 / s
BODY_T = 310.0                 # K
K_BOLTZMANN = 1.380649e-23     # J / K


def kbt_lattice(tau: float = 1.0, dx_um: float = DX_UM) -> float:
    """k_B T at body temperature expressed in lattice energy units."""
    dx = dx_um * 1e-6
    nu_lu = (tau - 0.5) / 3.0
    dt = nu_lu * dx * dx / PLASMA_NU
    mass = PLASMA_RHO * dx ** 3
    energy = mass * dx * dx / (dt * dt)
    return K_BOLTZMANN * BODY_T / energy


# Evans-Fung (1972) biconcave profile coefficients, D = 7.82 um
RBC_DIAMETER_UM = 7.82
EF_A0, EF_A1, EF_A2 = 0.0518, 2.0026, -4.491
PLATELET_SEMI_AXES_UM = (1.8, 1.8, 0.5)
LINK_PERSISTENCE_UM = 0.0075     # spectrin persistence length p
LINK_MAX_STRAIN = 3.0            # strain at which the link energy diverges


# ---------------------------------------------------------------------------
# meshes
# ---------------------------------------------------------------------------
def _icosahedron():
    phi = (1.0 + 5.0 ** 0.5) / 2.0
    v = []
    for a in (-1.0, 1.0):
        for b in (-phi, phi):
            v.append((0.0, a, b))
            v.append((a, b, 0.0))
            v.append((b, 0.0, a))
    v = np.array(v, dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    d = np.linalg.norm(v[:, None, :] - v[None, :, :], axis=2)
    edge_len = np.min(d[d > 1e-9])
    adj = np.abs(d - edge_len) < 1e-6
    tris = []
    n = len(v)
    for i in range(n):
        for j in range(i + 1, n):
            if not adj[i, j]:
                continue
            for k in range(j + 1, n):
                if adj[i, k] and adj[j, k]:
                    nrm = np.cross(v[j] - v[i], v[k] - v[i])
                    if np.dot(nrm, v[i] + v[j] + v[k]) > 0:
                        tris.append((i, j, k))
                    else:
                        tris.append((i, k, j))
    return v, np.array(tris, dtype=np.int32)


def icosphere(subdivisions: int):
    """Unit-sphere triangulation: the icosahedron split `subdivisions` times.

    Each split replaces a triangle (a, b, c) by (a, ab, ca), (ab, b, bc),
    (ca, bc, c), (ab, bc, ca); new midpoint vertices get ids in the order in
    which their edge is first met (triangles in order, edges ab, bc, ca).
    Triangles are counter-clockwise seen from outside.  Returns
    (vertices float64 [nv, 3], triangles int32 [nt, 3]).
    """
    v, t = _icosahedron()
    verts = [tuple(x) for x in v]
    tris = [tuple(x) for x in t]
    for _ in range(subdivisions):
        mid = {}
        new_tris = []

        def midpoint(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in mid:
                p = np.add(verts[a], verts[b]) * 0.5
                p = p / np.linalg.norm(p)
                verts.append(tuple(p))
                mid[key] = len(verts) - 1
            return mid[key]

        for (a, b, c) in tris:
            ab = midpoint(a, b)
            bc = midpoint(b, c)
            ca = midpoint(c, a)
            new_tris += [(a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca)]
        tris = new_tris
    return np.array(verts, dtype=np.float64), np.array(tris, dtype=np.int32)


def evans_fung(unit_verts: np.ndarray, diameter: float) -> np.ndarray:
    """Map unit-sphere vertices onto the Evans-Fung biconcave surface.

    (x, y) <- (sx, sy) * D / 2 and z <- sz * D * (a0 + a1 q / 4 + a2 q^2 / 16)
    with q = 1 - sz^2 (the squared normalised radius), which equals
    sign(sz) * D * sqrt(1 - q) * (a0 + a1 q/4 + a2 q^2/16).
    """
    s = unit_verts
    q = 1.0 - s[:, 2] ** 2
    out = np.empty_like(s)
    out[:, 0] = s[:, 0] * diameter * 0.5
    out[:, 1] = s[:, 1] * diameter * 0.5
    out[:, 2] = s[:, 2] * diameter * (EF_A0 + EF_A1 * q / 4.0 + EF_A2 * q * q / 16.0)
    return out


def spheroid(unit_verts: np.ndarray, a: float, c: float) -> np.ndarray:
    """Map unit-sphere vertices onto a spheroid with semi-axes (a, a, c)."""
    return unit_verts * np.array([a, a, c])


def locality_order(verts: np.ndarray, tris: np.ndarray):
    """Renumber a mesh's vertices along a Morton (Z-order) curve of their
    positions, so that neighbouring vertices get nearby ids (on the
    subdivided icosahedron of 642 vertices the median id gap between the two
    ends of an edge drops from 140 to 4).  The surface is unchanged; returns
    (vertices, triangles) renumbered."""
    bits = 10
    lo = verts.min(axis=0)
    span = float((verts.max(axis=0) - lo).max()) or 1.0
    q = np.floor((verts - lo) / span * ((1 << bits) - 1)).astype(np.int64)
    code = np.zeros(len(verts), np.int64)
    for b in range(bits):
        for d in range(3):
            code |= ((q[:, d] >> b) & 1) << (3 * b + d)
    order = np.argsort(code, kind='stable')  # new id k is old vertex order[k]
    new_id = np.empty_like(order)
    new_id[order] = np.arange(len(order))
    return verts[order], new_id[tris].astype(np.int32)


def rbc_mesh(subdivisions: int = 3, dx_um: float = DX_UM):
    v, t = locality_order(*icosphere(subdivisions))
    return evans_fung(v, RBC_DIAMETER_UM / dx_um), t


def platelet_mesh(subdivisions: int = 2, dx_um: float = DX_UM):
    v, t = locality_order(*icosphere(subdivisions))
    a, _, c = PLATELET_SEMI_AXES_UM
    return spheroid(v, a / dx_um, c / dx_um), t


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniformly distributed rotation matrix from a uniform unit quaternion."""
    u1, u2, u3 = rng.random(3)
    w = math.sqrt(1 - u1) * math.sin(2 * math.pi * u2)
    x = math.sqrt(1 - u1) * math.cos(2 * math.pi * u2)
    y = math.sqrt(u1) * math.sin(2 * math.pi * u3)
    z = math.sqrt(u1) * math.cos(2 * math.pi * u3)
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


# ---------------------------------------------------------------------------
# geometry: wall masks and initial velocity profiles
# ---------------------------------------------------------------------------
# mask values: 0 fluid, 1 resting wall, 2 / 3 moving walls (velocities given
# separately).  Arrays are indexed [z, y, x] (x fastest in memory).
FLUID, WALL, WALL_A, WALL_B = 0, 1, 2, 3


def plate_mask(nx, ny, nz, axis: int, lo_id=WALL, hi_id=WALL) -> np.ndarray:
    """Solid planes at index 0 and n-1 along `axis` (0 = x, 1 = y, 2 = z)."""
    m = np.zeros((nz, ny, nx), dtype=np.uint8)
    sl_lo = [slice(None)] * 3
    sl_hi = [slice(None)] * 3
    ax = 2 - axis
    sl_lo[ax] = 0
    sl_hi[ax] = m.shape[ax] - 1
    m[tuple(sl_lo)] = lo_id
    m[tuple(sl_hi)] = hi_id
    return m


def cylinder_mask(nx, ny, nz, radius: float, cy: float, cz: float) -> np.ndarray:
    """Pipe along x: nodes with (y-cy)^2 + (z-cz)^2 >= radius^2 are walls."""
    y = np.arange(ny, dtype=np.float64)[None, :, None]
    z = np.arange(nz, dtype=np.float64)[:, None, None]
    solid = (y - cy) ** 2 + (z - cz) ** 2 >= radius ** 2
    m = np.zeros((nz, ny, nx), dtype=np.uint8)
    m[np.broadcast_to(solid, m.shape)] = WALL
    return m


def channel_profile(nx, ny, nz, axis_wall: int, lo: float, hi: float, umax: float):
    """Parabolic x-velocity between planes at `lo` and `hi` along `axis_wall`
    with centreline value `umax`; zero outside.  Returned as [z, y, x, 3]."""
    u = np.zeros((nz, ny, nx, 3))
    coord = np.arange([nx, ny, nz][axis_wall], dtype=np.float64)
    s = (coord - lo) * (hi - coord) / ((hi - lo) / 2.0) ** 2
    s = np.clip(s, 0.0, None) * umax
    shape = [1, 1, 1]
    shape[2 - axis_wall] = -1
    u[..., 0] = s.reshape(shape)
    return u


def pipe_profile(nx, ny, nz, radius, cy, cz, umax):
    y = np.arange(ny, dtype=np.float64)[None, :, None]
    z = np.arange(nz, dtype=np.float64)[:, None, None]
    r2 = ((y - cy) ** 2 + (z - cz) ** 2) / radius ** 2
    s = np.clip(1.0 - r2, 0.0, None) * umax
    u = np.empty((nz, ny, nx, 3))
    u[..., 1:] = 0.0
    u[..., 0] = s
    return u


# ---------------------------------------------------------------------------
# placement: seeded random positions/orientations + force-bias relaxation
# ---------------------------------------------------------------------------
def _ellipsoid_inside(points, center, rot, axes):
    """points [n, p, 3] in the world frame, centers [n, 3], rotations
    [n, 3, 3] (columns = body axes), semi-axes [n, 3] -> normalised radius^2
    [n, p] in the body frame (< 1 inside)."""
    loc = np.einsum('npj,njk->npk', points - center[:, None, :], rot)
    return np.sum((loc / axes[:, None, :]) ** 2, axis=-1)


def contact_function(r, rot_a, axes_a, rot_b, axes_b, iters=40):
    """Perram-Wertheim contact function of pairs of ellipsoids (Perram and
    Wertheim, J. Comput. Phys. 58, 1985), vectorised over pairs.

    Ellipsoid a is centred at the origin and b at r [n, 3]; rotations
    [n, 3, 3] (columns = body axes), semi-axes [n, 3].  F = max over lambda in
    [0, 1] of lambda (1 - lambda) r^T C(lambda)^-1 r with C(lambda) =
    (1 - lambda) A^-1 + lambda B^-1, A^-1 = R diag(axes^2) R^T: the
    ellipsoids overlap exactly when F < 1, touch at F = 1, and since F is
    quadratic in r they touch once the centre distance is scaled by
    1 / sqrt(F).  The maximum of the single-peaked function of lambda is
    found by golden-section search (`iters` steps).
    """
    ai = np.einsum('nij,nj,nkj->nik', rot_a, axes_a ** 2, rot_a)
    bi = np.einsum('nij,nj,nkj->nik', rot_b, axes_b ** 2, rot_b)

    def f(lam):
        c = (1.0 - lam)[:, None, None] * ai + lam[:, None, None] * bi
        x = np.linalg.solve(c, r[..., None])[..., 0]
        return lam * (1.0 - lam) * np.einsum('ni,ni->n', r, x)

    g = (math.sqrt(5.0) - 1.0) / 2.0
    lo, hi = np.zeros(len(r)), np.ones(len(r))
    a, b = hi - g * (hi - lo), lo + g * (hi - lo)
    fa, fb = f(a), f(b)
    for _ in range(iters):
        left = fa > fb                      # the maximum lies in [lo, b]
        hi = np.where(left, b, hi)
        lo = np.where(left, lo, a)
        na = np.where(left, hi - g * (hi - lo), b)
        nb = np.where(left, a, lo + g * (hi - lo))
        fa, fb = np.where(left, f(na), fb), np.where(left, fa, f(nb))
        a, b = na, nb
    return np.maximum(fa, fb)


def _keep_in_cylinder(centers, rots, axes, cylinder):
    """Moves centres radially (about the x axis through (cy, cz)) so that
    each ellipsoid lies within the cylinder of the given radius: the
    distance of a centre from the axis is at most radius minus the largest
    semi-axis of the ellipsoid's projection onto the (y, z) plane (the
    largest eigenvalue's root of the (y, z) block of R diag(axes^2) R^T),
    which bounds every surface point's distance from the centre in that
    plane."""
    cy, cz, radius = cylinder
    dy, dz = centers[:, 1] - cy, centers[:, 2] - cz
    r = np.hypot(dy, dz)
    M = np.einsum('nij,nj,nkj->nik', rots, axes ** 2, rots)
    a, b, d = M[:, 1, 1], M[:, 1, 2], M[:, 2, 2]
    ext = np.sqrt(0.5 * (a + d) + np.sqrt(0.25 * (a - d) ** 2 + b * b))
    rmax = np.maximum(radius - ext, 0.0)
    scale = np.where(r > rmax, rmax / np.maximum(r, 1e-12), 1.0)
    centers[:, 1] = cy + dy * scale
    centers[:, 2] = cz + dz * scale


def pack_cells(rng, box_lo, box_hi, periodic, kinds, axes_by_kind, max_iter=400, exact_iter=0,
               margin=0.01, cylinder=None, sample_level=1):
    """Force-bias style packing of bounding ellipsoids (Section 2.4).

    Ellipsoids start at random uniform positions and orientations; every
    iteration each overlapping pair (i, j) is pushed apart along r_j - r_i by
    an amount proportional to its estimated overlap (the mean fraction of one
    ellipsoid's 42 surface samples found inside the other, a proxy for the
    overlap volume), and ellipsoids are pushed back inside the allowed box on
    non-periodic axes.  The surface samples are the vertices of the
    icosphere of `sample_level` splits (1: 42 samples, 0: 12).

    The sample proxy misses shallow overlaps.  With `exact_iter` > 0 a second
    phase follows that detects overlap exactly (`contact_function`) and
    moves the two centres of every overlapping pair apart along r_j - r_i,
    each by half the distance that would make the pair touch with a relative
    gap `margin`, for at most `exact_iter` rounds; the final centres satisfy
    the box constraints.  Returns (centers [n, 3], rotations [n, 3, 3],
    number of pairs still overlapping: by the proxy after the first phase
    alone, exactly when the second phase ran).  `cylinder` = (cy, cz,
    radius): every ellipsoid is also kept inside that cylinder about the x
    axis (a pipe), in both phases.
    """
    from scipy.spatial import cKDTree

    n = len(kinds)
    box_lo = np.asarray(box_lo, float)
    box_hi = np.asarray(box_hi, float)
    span = box_hi - box_lo
    per = np.asarray(periodic, bool)
    axes = np.array([axes_by_kind[k] for k in kinds], float).reshape(n, 3)
    rmax = axes.max(axis=1)
    centers = box_lo + rng.random((n, 3)) * span
    if cylinder is not None and n:  # uniform in the disc that keeps a cell's bounding sphere inside
        cy, cz, radius = cylinder
        rr = max(radius - float(rmax.max()), 0.0) * np.sqrt(rng.random(n))
        ang = 2.0 * math.pi * rng.random(n)
        centers[:, 1] = cy + rr * np.cos(ang)
        centers[:, 2] = cz + rr * np.sin(ang)
    rots = np.stack([random_rotation(rng) for _ in range(n)]) if n else np.zeros((0, 3, 3))
    sv, _ = icosphere(sample_level)
    cutoff = 2.0 * (rmax.max() if n else 1.0)
    # toroidal tree on periodic axes; a box far larger than the data elsewhere
    boxsize = np.where(per, span, 4.0 * span + 4.0 * cutoff)
    residual = 0
    for _ in range(max_iter):
        ext = np.sqrt(np.einsum('njk,nk->nj', rots ** 2, axes ** 2))
        for d in range(3):
            if per[d]:
                centers[:, d] = box_lo[d] + np.mod(centers[:, d] - box_lo[d], span[d])
            else:
                lo = box_lo[d] + ext[:, d]
                hi = box_hi[d] - ext[:, d]
                centers[:, d] = np.where(lo > hi, 0.5 * (box_lo[d] + box_hi[d]),
                                         np.clip(centers[:, d], lo, hi))
        if cylinder is not None:
            _keep_in_cylinder(centers, rots, axes, cylinder)
        local = centers - box_lo
        local = np.where(per, np.mod(local, span), local + 1.5 * span + cutoff)
        local = np.minimum(local, np.nextafter(boxsize, 0))
        tree = cKDTree(local, boxsize=boxsize)
        pairs = tree.query_pairs(cutoff, output_type='ndarray')
        if len(pairs) == 0:
            residual = 0
            break
        I, J = pairs[:, 0], pairs[:, 1]
        dvec = centers[J] - centers[I]
        dvec = np.where(per, dvec - span * np.round(dvec / span), dvec)
        dist = np.linalg.norm(dvec, axis=1)
        close = dist < rmax[I] + rmax[J]
        I, J, dvec, dist = I[close], J[close], dvec[close], dist[close]
        if len(I) == 0:
            residual = 0
            break
        cj = centers[I] + dvec
        si = centers[I][:, None, :] + np.einsum('pk,nk,njk->npj', sv, axes[I], rots[I])
        sj = cj[:, None, :] + np.einsum('pk,nk,njk->npj', sv, axes[J], rots[J])
        in_j = _ellipsoid_inside(si, cj, rots[J], axes[J]) < 1.0
        in_i = _ellipsoid_inside(sj, centers[I], rots[I], axes[I]) < 1.0
        p = 0.5 * (in_j.mean(axis=1) + in_i.mean(axis=1))
        deep = dist < 0.5 * np.minimum(axes[I].min(axis=1), axes[J].min(axis=1))
        p = np.where(deep, 1.0, p)
        ov = p > 0
        residual = int(ov.sum())
        if residual == 0:
            break
        I, J, p, dvec, dist = I[ov], J[ov], p[ov], dvec[ov], dist[ov]
        unit = dvec / np.maximum(dist, 1e-9)[:, None]
        tiny = dist < 1e-6
        if tiny.any():
            rnd = rng.normal(size=(int(tiny.sum()), 3))
            unit[tiny] = rnd / np.linalg.norm(rnd, axis=1, keepdims=True)
        step = (0.5 * (0.05 + p) * np.minimum(rmax[I], rmax[J]))[:, None] * unit
        disp = np.zeros_like(centers)
        np.add.at(disp, I, -step)
        np.add.at(disp, J, step)
        centers += disp
    if exact_iter <= 0 or n < 2:
        if cylinder is not None and n:  # the last round moved the centres after the constraint
            ext = np.sqrt(np.einsum('njk,nk->nj', rots ** 2, axes ** 2))
            for d in range(3):
                if per[d]:
                    centers[:, d] = box_lo[d] + np.mod(centers[:, d] - box_lo[d], span[d])
                else:
                    centers[:, d] = np.clip(centers[:, d], box_lo[d] + ext[:, d], box_hi[d] - ext[:, d])
            _keep_in_cylinder(centers, rots, axes, cylinder)
        return centers, rots, residual
    ext = np.sqrt(np.einsum('njk,nk->nj', rots ** 2, axes ** 2))
    for it in range(exact_iter + 1):
        for d in range(3):
            if per[d]:
                centers[:, d] = box_lo[d] + np.mod(centers[:, d] - box_lo[d], span[d])
            else:
                lo = box_lo[d] + ext[:, d]
                hi = box_hi[d] - ext[:, d]
                centers[:, d] = np.where(lo > hi, 0.5 * (box_lo[d] + box_hi[d]),
                                         np.clip(centers[:, d], lo, hi))
        if cylinder is not None:
            _keep_in_cylinder(centers, rots, axes, cylinder)
        local = centers - box_lo
        local = np.where(per, np.mod(local, span), local + 1.5 * span + cutoff)
        local = np.minimum(local, np.nextafter(boxsize, 0))
        pairs = cKDTree(local, boxsize=boxsize).query_pairs(cutoff, output_type='ndarray')
        residual = 0
        if len(pairs) == 0:
            break
        I, J = pairs[:, 0], pairs[:, 1]
        dvec = centers[J] - centers[I]
        dvec = np.where(per, dvec - span * np.round(dvec / span), dvec)
        dist = np.linalg.norm(dvec, axis=1)
        close = dist < rmax[I] + rmax[J]
        I, J, dvec, dist = I[close], J[close], dvec[close], dist[close]
        if len(I) == 0:
            break
        F = contact_function(dvec, rots[I], axes[I], rots[J], axes[J])
        ov = F < 1.0
        residual = int(ov.sum())
        if residual == 0 or it == exact_iter:
            break
        I, J, F, dvec, dist = I[ov], J[ov], F[ov], dvec[ov], dist[ov]
        unit = dvec / np.maximum(dist, 1e-9)[:, None]
        tiny = dist < 1e-6
        if tiny.any():
            rnd = rng.normal(size=(int(tiny.sum()), 3))
            unit[tiny] = rnd / np.linalg.norm(rnd, axis=1, keepdims=True)
            dist = np.where(tiny, 1e-6, dist)
            F = np.where(tiny, 1e-12, F)
        grow = (1.0 + margin) / np.sqrt(np.maximum(F, 1e-12)) - 1.0
        step = (0.5 * grow * dist)[:, None] * unit
        disp = np.zeros_like(centers)
        np.add.at(disp, I, -step)
        np.add.at(disp, J, step)
        centers += disp
    return centers, rots, residual


# ---------------------------------------------------------------------------
# configurations
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class MeshType:
    name: str
    rest: np.ndarray          # [nv, 3] float64, centred at the origin
    tri: np.ndarray           # [nt, 3] int32, outward counter-clockwise
    k_link: float             # in kBT
    k_bend: float             # in kBT
    k_area: float             # lattice units
    k_volume: float           # lattice units
    kbt: float
    persistence: float        # LU
    max_strain: float
    k_local: float = 0.0      # local (per-triangle) area modulus, lattice energy per lattice area; 0 = off
    theta_m: float = 0.0      # maximum bending deviation of the nonlinear bending term (rad); 0 = harmonic


@dataclasses.dataclass
class Config:
    name: str
    nx: int
    ny: int
    nz: int
    tau: float
    periodic: tuple
    mask: Optional[np.ndarray]            # uint8 [nz, ny, nx] or None
    wall_velocity: np.ndarray             # [2, 3]: velocities of mask ids 2 and 3
    body_force: np.ndarray                # [3]
    init_velocity: Optional[np.ndarray]   # [nz, ny, nx, 3] or None (rest)
    meshes: List[MeshType]
    cell_type: np.ndarray                 # [ncell] int
    centers: np.ndarray                   # [ncell, 3]
    rotations: np.ndarray                 # [ncell, 3, 3]
    steps: int
    seed: int
    note: str = ""

    @property
    def n_nodes(self):
        return self.nx * self.ny * self.nz

    @property
    def n_fluid(self):
        return self.n_nodes if self.mask is None else int((self.mask == 0).sum())

    @property
    def n_vertices(self):
        return int(sum(len(self.meshes[t].rest) for t in self.cell_type))


def _rbc_type(kbt, k_link=15.0, k_bend=80.0, k_area=5.0, k_volume=20.0, subdiv=3):
    v, t = rbc_mesh(subdiv)
    return MeshType('rbc', v, t, k_link, k_bend, k_area, k_volume, kbt,
                    LINK_PERSISTENCE_UM / DX_UM, LINK_MAX_STRAIN)


def _platelet_type(kbt, subdiv=2):
    v, t = platelet_mesh(subdiv)
    # stiffness x10 on link and bending moduli (platelets are much stiffer)
    return MeshType('platelet', v, t, 150.0, 800.0, 5.0, 20.0, kbt,
                    LINK_PERSISTENCE_UM / DX_UM, LINK_MAX_STRAIN)


RBC_BOUND = (7.82, 7.82, 4.3)          # LU semi-axes enclosing the biconcave shape
PLATELET_BOUND = (3.6, 3.6, 1.0)


def shear_cell(n=32, ncell=1, seed=20230500, steps=500, wall_speed=0.01, tau=1.0,
               k=(15.0, 80.0, 5.0, 20.0), name='shear', exact_iter=400):
    """Parallel plates at z=0 and z=n-1 moving at -/+ wall_speed along x."""
    rng = np.random.default_rng(seed)
    kbt = kbt_lattice(1.0)
    mask = plate_mask(n, n, n, axis=2, lo_id=WALL_A, hi_id=WALL_B)
    wv = np.array([[-wall_speed, 0, 0], [wall_speed, 0, 0]], float)
    mt = _rbc_type(kbt, *k)
    if ncell == 1:
        centers = np.array([[n / 2.0, n / 2.0, (n - 1) / 2.0]])
        rots = random_rotation(rng)[None]
    else:
        centers, rots, _ = pack_cells(rng, (0, 0, 1.5), (n, n, n - 2.5), (1, 1, 0),
                                      [0] * ncell, {0: RBC_BOUND}, exact_iter=exact_iter)
    return Config(name, n, n, n, tau, (1, 1, 0), mask, wv, np.zeros(3), None, [mt],
                  np.zeros(len(centers), np.int64), centers, rots, steps, seed)


def channel(nx=64, ny=64, nz=256, ncell=440, seed=20230501, steps=1000, umax=0.02,
            tau=1.0, platelet_ratio=0.0, name='channel', pack_iter=400, exact_iter=400):
    """Walls at y=0 and y=ny-1, periodic in x and z, body force along x giving
    centreline velocity `umax` (effective walls at y=0.5 and y=ny-1.5).
    `pack_iter` and `exact_iter` bound the two phases of `pack_cells`; the
    note records the bounding-ellipsoid pairs still overlapping."""
    rng = np.random.default_rng(seed)
    kbt = kbt_lattice(tau)
    mask = plate_mask(nx, ny, nz, axis=1)
    nu = (tau - 0.5) / 3.0
    H = ny - 2.0
    g = np.array([8.0 * nu * umax / H ** 2, 0.0, 0.0])
    meshes = [_rbc_type(kbt)]
    nplt = int(round(ncell * platelet_ratio))
    kinds = [0] * ncell
    if nplt:
        meshes.append(_platelet_type(kbt))
        kinds += [1] * nplt
    bounds = {0: RBC_BOUND, 1: PLATELET_BOUND}
    centers, rots, resid = pack_cells(rng, (0, 2.5, 0), (nx, ny - 3.5, nz), (1, 0, 1),
                                      kinds, bounds, max_iter=pack_iter, exact_iter=exact_iter)
    u0 = channel_profile(nx, ny, nz, 1, 0.5, ny - 1.5, umax)
    return Config(name, nx, ny, nz, tau, (1, 0, 1), mask, np.zeros((2, 3)), g, u0, meshes,
                  np.array(kinds, np.int64), centers, rots, steps, seed,
                  note=f'residual overlapping bounding-ellipsoid pairs: {resid}')


def pipe_placement(rng, length, cy, cz, r_in, ncell, pack_iter, exact_iter):
    """Red-cell centres and rotations inside the cylinder of radius r_in
    about the x axis through (cy, cz), periodic over `length` in x."""
    return pack_cells(rng, (0, cy - r_in, cz - r_in), (length, cy + r_in, cz + r_in), (1, 0, 0),
                      [0] * ncell, {0: RBC_BOUND}, max_iter=pack_iter, exact_iter=exact_iter,
                      cylinder=(cy, cz, r_in), sample_level=0)


def pipe(nx=1000, ny=208, nz=208, radius=100.0, ncell=19600, seed=20230504, steps=200,
         umax=0.02, tau=1.0, name='pipe', pack_iter=3, exact_iter=0):
    """Straight pipe along x (periodic ends), voxelised wall, body-force
    driven.  Cells start uniformly in the pipe's cross-section and are
    packed inside the cylinder 3 nodes within the wall (`pack_cells` with
    the cylinder constraint and 12 surface samples, `pack_iter` /
    `exact_iter` bounding its two phases).  At 19,600 red cells the
    bounding ellipsoids (7.82 x 7.82 x 4.3) fill about 73 % of that
    cylinder, above the density at which randomly oriented ellipsoids of
    this aspect ratio jam, so the placement cannot be free of ellipsoid
    overlap and further relaxation rounds do not reduce it (about 6 overlaps
    per cell after 4 or 8 rounds alike); the note records the pairs still
    overlapping."""
    rng = np.random.default_rng(seed)
    kbt = kbt_lattice(tau)
    cy = cz = (ny - 1) / 2.0
    mask = cylinder_mask(nx, ny, nz, radius, cy, cz)
    nu = (tau - 0.5) / 3.0
    g = np.array([4.0 * nu * umax / radius ** 2, 0.0, 0.0])
    meshes = [_rbc_type(kbt)]
    kinds = [0] * ncell
    centers, rots, resid = pipe_placement(rng, nx, cy, cz, radius - 3.0, ncell, pack_iter, exact_iter)
    u0 = pipe_profile(nx, ny, nz, radius, cy, cz, umax)
    how = 'exactly' if exact_iter > 0 else 'by the sampled estimate'
    return Config(name, nx, ny, nz, tau, (1, 0, 0), mask, np.zeros((2, 3)), g, u0, meshes,
                  np.array(kinds, np.int64), centers, rots, steps, seed,
                  note=f'residual overlapping bounding-ellipsoid pairs ({how}): {resid}')


def cell_vertices(cfg: Config) -> np.ndarray:
    """Initial absolute vertex positions [nv_total, 3] (rest shape rotated and
    translated), in cell order."""
    out = []
    for t, c, r in zip(cfg.cell_type, cfg.centers, cfg.rotations):
        out.append(cfg.meshes[t].rest @ r.T + c)
    return np.concatenate(out) if out else np.zeros((0, 3))
