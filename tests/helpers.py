"""Shared helpers for the GPU parity tests (comparison only: no method
arithmetic)."""
import numpy as np

import oracle as O
from paper_2305_02752_gb300 import inputs as I


def rel_l2(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def assert_close(got, exp, tol, what='', max_tol=None):
    """Parity check of one field: relative L2 error <= tol (the measure the
    tolerances are stated in) and, so that an error confined to a few
    elements (next to a wall, on a bin face, across a periodic or shifted
    boundary) is not diluted by the whole-field norm, the largest
    per-element error <= max_tol (default tol) times the field's largest
    magnitude."""
    a = np.asarray(got, float)
    b = np.asarray(exp, float)
    assert a.shape == b.shape, (what, a.shape, b.shape)
    err = rel_l2(a, b)
    assert err < tol, (what, 'relative L2', err, tol)
    scale = np.abs(b).max() if b.size else 0.0
    worst = np.abs(a - b).max() if b.size else 0.0
    mt = tol if max_tol is None else max_tol
    assert worst <= mt * (scale if scale > 0 else 1.0), (what, 'max abs', worst, mt * scale)


def direction_map():
    """perm with oracle_index = perm[library_index] (same velocity vector)."""
    from paper_2305_02752_gb300 import hemo
    cg, _ = hemo.velocity_set()
    co, _, _ = O.d3q19()
    return np.array([int(np.where((co == cg[i]).all(axis=1))[0][0]) for i in range(19)])


def small_cell_shear(n=16, seed=7, steps=20, diameter=8.0, sub=2, center=None):
    cfg = I.shear_cell(n=n, ncell=1, seed=seed, steps=steps)
    v, t = I.icosphere(sub)
    cfg.meshes[0].rest = I.evans_fung(v, diameter)
    cfg.meshes[0].tri = t
    cfg.centers = np.array([center if center is not None else [n / 2.0, n / 2.0, (n - 1) / 2.0]])
    return cfg


def run_both(cfg, precision, steps):
    from paper_2305_02752_gb300 import hemo
    sim = hemo.Simulation.from_config(cfg, precision)
    sim.step(steps)
    got = sim.get_fields()
    got['f'] = sim.populations() if sim.N <= 2_000_000 else None
    sim.close()
    ref = O.from_config(cfg)
    ref.step(steps)
    exp = ref.get()
    exp['f'] = ref.populations() if ref.N <= 2_000_000 else None
    return got, exp


def forces_close(got, exp, cfg, rtol=1e-12):
    """Membrane forces agree to `rtol` relative L2, or, near the rest shape,
    to an absolute floor set by conditioning: the area and volume terms scale
    with (A - A0)/A0^2, whose absolute rounding error (~1e-16 A0 sqrt(nt),
    summation order) does not shrink with the deformation; times |grad A| ~
    sqrt(A0/nt) this leaves ~1e-16 k / sqrt(A0) per component.  The floor is
    100x that."""
    if rel_l2(got, exp) < rtol:
        return True
    floor = 0.0
    for mt in cfg.meshes:
        A0 = mesh_area(mt.rest, mt.tri)
        floor = max(floor, 1e-14 * (mt.k_area + mt.k_volume) / np.sqrt(A0))
    return np.abs(np.asarray(got) - np.asarray(exp)).max() < floor


def mesh_area(rest, tri):
    a, b, c = rest[tri[:, 0]], rest[tri[:, 1]], rest[tri[:, 2]]
    return 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1).sum()
