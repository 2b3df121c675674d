"""Pins of the oracle's Lees-Edwards boundary (Sec. 2.5: a fully periodic
domain with opposing velocities imposed on two parallel boundaries, so that
a uniform shear needs no walls; cells crossing the boundary continue on the
other side).  Along z the image above the box is displaced by D_n = U n
(mod nx) and moves with U x^.

Closed forms: the steady state from rest is the linear profile
u_x(z) = (U / nz) (z - (nz - 1) / 2) (the jump across the plane is U and the
mean momentum stays zero); started at that profile the fluid stays on it
exactly (the Galilean-shifted image populations are the equilibrium of the
continued profile), so a force-free cell anywhere, also across the plane,
moves with the continued profile, and the 4-point kernel interpolates that
linear field exactly.  U = 0 is the periodic lattice bit for bit."""
import numpy as np

import oracle as O
from paper_2305_02752_gb300 import inputs as I

FREE = np.array([0.0, 0.0, 0.0, 0.0, 1e-3, 0.015, 3.0])


def _profile(nz, U):
    return (U / nz) * (np.arange(nz) - (nz - 1) / 2.0)


def test_steady_linear_profile_from_rest():
    nx, ny, nz, U = 6, 2, 16, 0.05
    s = O.OracleSim(nx, ny, nz, 1.0, (1, 1, 1))
    s.set_lees_edwards(U)
    s.set_velocity(None)
    s.step(1500)
    u = s.get()['u']
    assert np.abs(u[..., 0] - _profile(nz, U)[:, None, None]).max() < 1e-9
    assert np.abs(u[..., 1:]).max() < 1e-12


def test_linear_profile_is_exactly_steady():
    nx, ny, nz, U = 7, 3, 12, 0.04
    s = O.OracleSim(nx, ny, nz, 0.9, (1, 1, 1))
    s.set_lees_edwards(U)
    u0 = np.zeros((nz, ny, nx, 3))
    u0[..., 0] = _profile(nz, U)[:, None, None]
    s.set_velocity(u0)
    s.step(37)  # the displacement D_n takes non-integer values
    assert np.abs(s.get()['u'] - u0).max() < 1e-15


def test_zero_velocity_is_the_periodic_lattice():
    rng = np.random.default_rng(1)
    n = 8
    u0 = 0.02 * rng.normal(size=(n, n, n, 3))
    a = O.OracleSim(n, n, n, 0.8, (1, 1, 1))
    a.set_lees_edwards(0.0)
    a.set_velocity(u0)
    a.step(9)
    b = O.OracleSim(n, n, n, 0.8, (1, 1, 1))
    b.set_velocity(u0)
    b.step(9)
    assert np.array_equal(a.populations(), b.populations())


def _tracer_box(nz, U, center, tau=1.0):
    nx, ny = 16, 16
    s = O.OracleSim(nx, ny, nz, tau, (1, 1, 1))
    s.set_lees_edwards(U)
    u0 = np.zeros((nz, ny, nx, 3))
    u0[..., 0] = _profile(nz, U)[:, None, None]
    s.set_velocity(u0)
    v, t = I.icosphere(2)
    s.add_mesh(v * 2.5, t, FREE)
    s.add_cells(0, np.array([center]), np.eye(3)[None])
    return s


def test_force_free_cell_across_the_plane_follows_the_continued_profile():
    """Vertices on both sides of the plane (stencils in the image) move with
    u_x = (U / nz)(z - (nz - 1)/2) continued beyond the box."""
    nz, U, K = 16, 0.06, 9
    s = _tracer_box(nz, U, [7.3, 8.2, nz - 0.7])  # centroid in the box, cell across z = nz
    X0 = s.get()['X']
    assert (X0[:, 2] >= nz).any() and (X0[:, 2] < nz - 2).any()
    s.step(K)
    X = s.get()['X']
    vx = (U / nz) * (X0[:, 2] - (nz - 1) / 2.0)
    assert np.abs(X[:, 0] - (X0[:, 0] + K * vx)).max() < 1e-12
    assert np.abs(X[:, 1:] - X0[:, 1:]).max() < 1e-13


def test_cell_crossing_moves_it_by_the_displacement():
    """A cell whose centroid is above the box at the start of step n moves by
    (-D_n, 0, -nz) and then follows the profile from its new place."""
    nz, U, k = 16, 0.06, 23
    s = _tracer_box(nz, U, [7.3, 8.2, 5.0])
    s.step(k)
    Xa = s.get()['X'] + np.array([0.0, 0.0, nz + 0.1 - 5.0])  # lift the cell above the box
    s.set_vertices(Xa)
    s.step(1)
    D = (U * k) % 16
    Xr = Xa - np.array([D, 0.0, nz])
    vx = (U / nz) * (Xr[:, 2] - (nz - 1) / 2.0)
    X = s.get()['X']
    assert np.abs(X[:, 2] - Xr[:, 2]).max() < 1e-13
    assert np.abs(X[:, 0] - (Xr[:, 0] + vx)).max() < 1e-12


def test_arguments():
    s = O.OracleSim(4, 4, 4, 1.0, (1, 1, 0))
    try:
        s.set_lees_edwards(0.1)
    except ValueError:
        pass
    else:
        raise AssertionError('a non-periodic z axis must be refused')
    s = O.OracleSim(4, 4, 4, 1.0, (1, 1, 1))
    s.set_lees_edwards(0.1)
    try:
        s.set_viscosity_ratio(5.0)  # the indicator's rays would cross the displaced plane
    except ValueError:
        pass
    else:
        raise AssertionError('the internal viscosity must be refused with the boundary')
