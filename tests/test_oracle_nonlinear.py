"""Pins of the oracle's fuller constitutive model (Sec. 2.3: the response to
large deformations is highly non-linear, from membrane and cytoskeleton):
the nonlinear bending term (maximum bending deviation theta_m) and the local
(per-triangle) area term, both off unless their parameter is set.

Pinned by the energy-gradient identity (central differences), the rest
state, rigid motions, the closed-form local-area energy of a uniformly
scaled mesh (every triangle area scales by s^2, dihedral angles do not
change), the harmonic limit theta_m -> infinity, and the bound
-ln(1 - r^2) >= r^2 of the bending energy."""
import numpy as np

import oracle as O
from paper_2305_02752_gb300 import inputs as I

# k_link, k_bend, k_area, k_volume, kBT, persistence, max strain, k_local, theta_m
PARAMS = np.array([15.0, 80.0, 5.0, 20.0, 1e-3, 0.015, 3.0, 0.7, 0.6])


def _fd(rest, tri, params, X, idx, h):
    fd = np.zeros((len(idx), 3))
    for a, i in enumerate(idx):
        for k in range(3):
            Xp = X.copy()
            Xp[i, k] += h
            Xm = X.copy()
            Xm[i, k] -= h
            fd[a, k] = -(O.membrane(rest, tri, params, Xp)[1].sum() - O.membrane(rest, tri, params, Xm)[1].sum()) / (2 * h)
    return fd


def test_forces_are_energy_gradient_icosahedron():
    """Each new term alone, then all terms: F = -grad E on a perturbed
    12-vertex icosahedron."""
    rng = np.random.default_rng(5)
    v, t = I.icosphere(0)
    rest = v * 3.0
    X = rest + 0.15 * rng.normal(size=rest.shape)
    only_bend = PARAMS.copy()
    only_bend[[0, 2, 3, 7]] = 0.0
    only_local = PARAMS.copy()
    only_local[[0, 1, 2, 3]] = 0.0
    for p in (only_bend, only_local, PARAMS):
        F, E, _ = O.membrane(rest, t, p, X)
        assert np.abs(E).sum() > 0
        fd = _fd(rest, t, p, X, range(len(X)), 1e-6)
        assert np.linalg.norm(F - fd) / np.linalg.norm(F) < 1e-7


def test_forces_are_energy_gradient_rbc_mesh():
    rng = np.random.default_rng(6)
    rest, t = I.rbc_mesh()
    X = rest + 0.05 * rng.normal(size=rest.shape)
    F, _, _ = O.membrane(rest, t, PARAMS, X)
    idx = rng.choice(len(X), 12, replace=False)
    fd = _fd(rest, t, PARAMS, X, idx, 1e-5)
    assert np.linalg.norm(F[idx] - fd) / np.linalg.norm(F[idx]) < 1e-7


def test_rest_state_and_rigid_motion():
    rest, t = I.rbc_mesh()
    F, E, _ = O.membrane(rest, t, PARAMS, rest)
    assert np.abs(F).max() <= 1e-14 * PARAMS[:4].max()
    assert np.abs(E).max() == 0.0
    rng = np.random.default_rng(7)
    X = rest + 0.05 * rng.normal(size=rest.shape)
    R = I.random_rotation(rng)
    F1, E1, _ = O.membrane(rest, t, PARAMS, X)
    F2, E2, _ = O.membrane(rest, t, PARAMS, X @ R.T + np.array([3.0, -1.0, 2.0]))
    assert np.allclose(E1, E2, rtol=1e-11, atol=0)
    assert np.abs(F2 - F1 @ R.T).max() < 1e-10 * np.abs(F1).max()
    assert np.abs(F1.sum(0)).max() < 1e-11 * np.abs(F1).max()
    assert np.abs(np.cross(X, F1).sum(0)).max() < 1e-10 * np.abs(F1).max() * np.abs(X).max()


def test_local_area_closed_form_under_uniform_scaling():
    """X = s * rest: every triangle area is s^2 A_t0, so the local term is
    1/2 k_local (s^2 - 1)^2 sum_t A_t0 = 1/2 k_local (s^2 - 1)^2 A0, and
    the bending energy is zero (dihedral angles are scale invariant)."""
    rest, t = I.rbc_mesh()
    p = np.array([0.0, 80.0, 0.0, 0.0, 1e-3, 0.015, 3.0, 0.7, 0.6])
    for s in (0.9, 1.1, 1.25):
        _, E, AV = O.membrane(rest, t, p, s * rest)
        A0 = AV[2]
        assert abs(E[2] - 0.5 * 0.7 * (s * s - 1) ** 2 * A0) < 1e-12 * E[2]
        assert abs(E[1]) < 1e-20


def test_bending_harmonic_limit_and_bound():
    """theta_m -> infinity recovers the harmonic bending forces; for finite
    theta_m the bending energy is at least the harmonic one and the two
    agree to second order for small deformations."""
    rng = np.random.default_rng(8)
    rest, t = I.rbc_mesh()
    X = rest + 0.03 * rng.normal(size=rest.shape)
    harm = np.array([0.0, 80.0, 0.0, 0.0, 1e-3, 0.015, 3.0, 0.0, 0.0])
    big = harm.copy()
    big[8] = 1e4
    Fh, Eh, _ = O.membrane(rest, t, harm, X)
    Fb, Eb, _ = O.membrane(rest, t, big, X)
    assert np.linalg.norm(Fb - Fh) / np.linalg.norm(Fh) < 1e-7
    nl = harm.copy()
    nl[8] = 0.5
    _, En, _ = O.membrane(rest, t, nl, X)
    assert En[1] > Eh[1]
    Xs = rest + 1e-4 * (X - rest)
    _, Ehs, _ = O.membrane(rest, t, harm, Xs)
    _, Ens, _ = O.membrane(rest, t, nl, Xs)
    assert abs(Ens[1] / Ehs[1] - 1) < 1e-6


def test_defaults_leave_the_model_unchanged():
    """k_local = 0 and theta_m = 0 give the four-term model bit for bit."""
    rng = np.random.default_rng(9)
    rest, t = I.rbc_mesh()
    X = rest + 0.05 * rng.normal(size=rest.shape)
    F7, E7, _ = O.membrane(rest, t, PARAMS[:7], X)
    p9 = PARAMS.copy()
    p9[7:] = 0.0
    F9, E9, _ = O.membrane(rest, t, p9, X)
    assert np.array_equal(F7, F9) and np.array_equal(E7, E9)
