"""Pins of the oracle's internal viscosity (Sec. 1: the cytosol is five
times as viscous as the plasma; Sec. 3: the red-cell model carries an
internal viscosity ratio): the inside/outside indicator and the relaxation
time tau_in = 1/2 + lambda (tau - 1/2) at inside nodes.

The indicator (upward-ray crossing count) is pinned against an independent
definition for convex cells (inside every face plane, over the periodic
images), against the volume of a non-convex red cell (the expected number of
lattice nodes inside a randomly translated body is its volume), and against
integer translations with periodic wrap.  The relaxation time is pinned by a
run with every node forced inside, which must equal a run with tau_in as the
fluid's own relaxation time, and by the decay of a shear wave whose rate
scales with the viscosity."""
import numpy as np
import pytest

import oracle as O
from paper_2305_02752_gb300 import inputs as I

FREE = np.array([0.0, 0.0, 0.0, 0.0, 1e-3, 0.015, 3.0])


def _box_with_cells(n, rest, tri, centers, rots, periodic=(1, 1, 1), tau=1.0):
    s = O.OracleSim(n, n, n, tau, periodic)
    s.add_mesh(rest, tri, FREE)
    for c, r in zip(centers, rots):
        s.add_cells(0, np.array([c]), np.array([r]))
    return s


def _halfspace_inside(X, tri, n, periodic):
    """Independent definition for a convex cell: a node is inside when it
    lies strictly on the inner side of every face plane, for some periodic
    image of the cell."""
    a, b, c = X[tri[:, 0]], X[tri[:, 1]], X[tri[:, 2]]
    nrm = np.cross(b - a, c - a)
    g = np.arange(n)
    pts = np.stack(np.meshgrid(g, g, g, indexing='ij'), -1).reshape(-1, 3)[:, ::-1]  # (x, y, z) in [z, y, x] order
    inside = np.zeros(len(pts), bool)
    shifts = [(kx, ky, kz) for kx in (-1, 0, 1) for ky in (-1, 0, 1) for kz in (-1, 0, 1)
              if (kx == 0 or periodic[0]) and (ky == 0 or periodic[1]) and (kz == 0 or periodic[2])]
    for k in shifts:
        p = pts.astype(float) - np.array(k) * n
        side = np.einsum('tk,ptk->pt', nrm, p[:, None, :] - a[None, :, :])
        inside |= (side < 0).all(axis=1)
    return inside.reshape(n, n, n)


@pytest.mark.parametrize('seed', range(3))
def test_convex_cell_matches_halfspace_definition(seed):
    rng = np.random.default_rng(seed)
    n = 16
    v, t = I.icosphere(2)
    rest = v * np.array([5.0, 4.0, 3.0])
    R = I.random_rotation(rng)
    c = rng.random(3) * n if seed else np.array([0.7, 15.2, 8.4])  # seed 0 straddles two periodic edges
    s = _box_with_cells(n, rest, t, [c], [R])
    X = s.get()['X']
    ins = s.inside()
    ref = _halfspace_inside(X, t, n, (1, 1, 1))
    assert ins.sum() > 100
    assert np.array_equal(ins.astype(bool), ref)


def test_red_cell_node_count_matches_volume():
    """Non-convex (biconcave) cell: averaged over random translations and
    rotations the number of inside nodes is the cell's volume."""
    rng = np.random.default_rng(3)
    n = 32
    rest, t = I.rbc_mesh()
    rest = rest * 2.0  # about 31 lattice units across
    counts, vols = [], []
    for _ in range(12):
        s = _box_with_cells(n, rest, t, [rng.random(3) * n], [I.random_rotation(rng)])
        counts.append(s.inside().sum())
        vols.append(s.get()['cellstats'][0, 4])
    assert abs(np.mean(counts) / np.mean(vols) - 1) < 0.01


def test_integer_translation_with_wrap():
    rng = np.random.default_rng(4)
    n = 20
    rest, t = I.rbc_mesh()
    R = I.random_rotation(rng)
    c = np.array([18.3, 1.7, 10.2])  # across the x and y edges
    a = _box_with_cells(n, rest, t, [c], [R]).inside()
    shift = np.array([5, -7, 9])
    b = _box_with_cells(n, rest, t, [c + shift], [R]).inside()
    assert a.sum() > 200
    assert np.array_equal(np.roll(a, shift=(9, -7, 5), axis=(0, 1, 2)), b)


def test_forced_inside_equals_fluid_with_tau_in():
    """Every node forced inside with ratio lambda: the same run as the fluid
    alone with tau_in = 1/2 + lambda (tau - 1/2), bit for bit."""
    rng = np.random.default_rng(5)
    n, tau, lam = 12, 0.8, 3.0
    u0 = 0.02 * rng.normal(size=(n, n, n, 3))
    a = O.OracleSim(n, n, n, tau, (1, 1, 1), None, None, np.array([1e-5, 0, 0]))
    a.set_velocity(u0)
    a.set_viscosity_ratio(lam)
    a.force_inside(np.ones((n, n, n), np.uint8))
    a.step(7)
    b = O.OracleSim(n, n, n, 0.5 + lam * (tau - 0.5), (1, 1, 1), None, None, np.array([1e-5, 0, 0]))
    b.set_velocity(u0)
    b.step(7)
    assert np.array_equal(a.populations(), b.populations())
    c = O.OracleSim(n, n, n, tau, (1, 1, 1), None, None, np.array([1e-5, 0, 0]))
    c.set_velocity(u0)
    c.step(7)
    assert not np.array_equal(a.populations(), c.populations())


def test_shear_wave_decay_scales_with_viscosity():
    """u_x = u0 sin(2 pi y / L) decays as exp(-nu k^2 t) with nu = (tau - 1/2)/3;
    with every node inside and ratio 2 the decay exponent doubles."""
    L, tau = 64, 0.8
    y = np.arange(L)
    u0 = np.zeros((1, L, 1, 3))
    u0[0, :, 0, 0] = 1e-3 * np.sin(2 * np.pi * y / L)
    rates = []
    for lam in (1.0, 2.0):
        s = O.OracleSim(1, L, 1, tau, (1, 1, 1))
        s.set_velocity(u0)
        if lam != 1.0:
            s.set_viscosity_ratio(lam)
            s.force_inside(np.ones((1, L, 1), np.uint8))
        amp = []
        for steps in (50, 250):  # after the start-up transient of the equilibrium start
            s.step(steps - (50 if amp else 0))
            amp.append(2 * np.mean(s.get()['u'][0, :, 0, 0] * np.sin(2 * np.pi * y / L)))
        rates.append(np.log(amp[0] / amp[1]) / 200)
    k2 = (2 * np.pi / L) ** 2
    assert abs(rates[0] / (k2 * (tau - 0.5) / 3) - 1) < 5e-3
    assert abs(rates[1] / rates[0] - 2) < 5e-3


def test_ratio_one_is_the_default_step():
    cfg = I.shear_cell(n=16, ncell=1, seed=3, steps=5)
    v, t = I.icosphere(2)
    cfg.meshes[0].rest = I.evans_fung(v, 8.0)
    cfg.meshes[0].tri = t
    cfg.centers = np.array([[8.0, 8.0, 7.5]])
    u0 = 0.01 * np.random.default_rng(6).normal(size=(16, 16, 16, 3))
    u0[cfg.mask != 0] = 0.0
    cfg.init_velocity = u0  # inside nodes away from equilibrium from the start
    a = O.from_config(cfg)
    a.set_viscosity_ratio(1.0)
    a.step(5)
    b = O.from_config(cfg)
    b.step(5)
    c = O.from_config(cfg)
    c.set_viscosity_ratio(5.0)
    c.step(5)
    assert np.array_equal(a.populations(), b.populations())
    assert not np.array_equal(a.populations(), c.populations())
