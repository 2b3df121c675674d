"""Pins of the oracle's time-scale separation and vertex integrators
(Sec. 2.6: cells integrated by Euler or Adams-Bashforth; the membrane model
evaluated every N fluid steps and held in between).

Closed form used below: in a fully periodic box at rest with a uniform body
force g and no membrane force, every node stays identical, so streaming is
the identity, the density stays 1, and the Guo-forced BGK collision adds
exactly g to the momentum per step.  The velocity that includes F/2, read
after the streaming of the step with index n (0-based), is therefore
U^n = (n + 3/2) g everywhere, and the 4-point kernel interpolates a uniform
field exactly.  Euler moves a vertex by sum_n U^n; Adams-Bashforth moves it
by U^0 on the first step, then by 3/2 U^n - 1/2 U^{n-1} = (n + 2) g, the
velocity at mid-step n + 1/2 (the two-step formula is exact for a velocity
linear in time).
"""
import numpy as np
import pytest

import oracle as O
from paper_2305_02752_gb300 import inputs as I

G = np.array([2e-4, -1e-4, 5e-5])
PARAMS = np.array([15.0, 80.0, 5.0, 20.0, 1e-3, 0.015, 3.0])
FREE = np.array([0.0, 0.0, 0.0, 0.0, 1e-3, 0.015, 3.0])  # all four moduli zero


def _accelerating_box(params):
    n = 10
    s = O.OracleSim(n, n, n, 0.9, (1, 1, 1), None, None, G)
    s.set_velocity(None)
    v, t = I.icosphere(1)
    s.add_mesh(v * 2.5, t, params)
    s.add_cells(0, np.array([[4.3, 5.1, 4.7]]), np.eye(3)[None])
    return s


def _euler_sum(n0, n1):
    """sum of U^n for n0 <= n < n1 (in units of g)."""
    return sum(n + 1.5 for n in range(n0, n1))


def _ab2_sum(n0, n1):
    """Adams-Bashforth displacement over steps n0 <= n < n1 started at n0."""
    return (n0 + 1.5) + sum(1.5 * (n + 1.5) - 0.5 * (n + 0.5) for n in range(n0 + 1, n1))


@pytest.mark.parametrize('integrator', ['euler', 'ab2'])
def test_uniform_acceleration_closed_form(integrator):
    """A force-free cell in a uniformly accelerated periodic fluid: every
    vertex moves by the closed-form displacement of the chosen integrator."""
    s = _accelerating_box(FREE)
    X0 = s.get()['X']
    s.set_time_scales(1, integrator)
    K = 6
    s.step(K)
    out = s.get()
    assert np.abs(out['Fv']).max() == 0.0
    assert np.abs(out['u'] - (K + 0.5) * G).max() < 1e-15
    k = _euler_sum(0, K) if integrator == 'euler' else _ab2_sum(0, K)
    assert k == (24.0 if integrator == 'euler' else 26.5)
    assert np.abs(out['X'] - (X0 + k * G)).max() < 1e-14


def test_ab2_restarts_with_euler_after_a_change():
    """Switching to Adams-Bashforth after three Euler steps: the first step
    after the switch has no previous velocity and is an Euler step."""
    s = _accelerating_box(FREE)
    X0 = s.get()['X']
    s.step(3)
    s.set_time_scales(1, 'ab2')
    s.step(4)
    k = _euler_sum(0, 3) + _ab2_sum(3, 7)
    assert k == 7.5 + 4.5 + 6.0 + 7.0 + 8.0
    assert np.abs(s.get()['X'] - (X0 + k * G)).max() < 1e-14


@pytest.mark.parametrize('integrator', ['euler', 'ab2'])
def test_forces_held_between_evaluations(integrator):
    """Time-scale separation N = 4 on a deformed cell: after each step the
    membrane forces are those of the positions at the last evaluation step
    (n = 0, 4, 8, ...), held unchanged, and they differ from the forces at
    the current positions on the steps in between."""
    s = _accelerating_box(PARAMS)
    v, t = I.icosphere(1)
    rest = v * 2.5
    X = s.get()['X']
    X = X.mean(0) + (X - X.mean(0)) * np.array([1.15, 1.0, 0.9])  # stretched: non-zero forces
    s.set_vertices(X)
    N = 4
    s.set_time_scales(N, integrator)
    held = None
    for n in range(11):
        Xn = s.get()['X']
        Fn = O.membrane(rest, t, PARAMS, Xn)[0]
        if n % N == 0:
            held = Fn
        s.step(1)
        Fv = s.get()['Fv']
        assert np.array_equal(Fv, held), n
        if n % N:
            assert np.abs(Fn - held).max() > 1e-3 * np.abs(held).max(), n


def test_force_every_one_is_the_default_step():
    """N = 1 with Euler is the default coupled step, bit for bit, and
    Adams-Bashforth changes the trajectory of a deforming cell."""
    def run(ts):
        s = _accelerating_box(PARAMS)
        X = s.get()['X']
        s.set_vertices(X.mean(0) + (X - X.mean(0)) * np.array([1.1, 1.0, 0.95]))
        if ts:
            s.set_time_scales(*ts)
        s.step(5)
        return s.get()

    a, b, c = run(None), run((1, 'euler')), run((1, 'ab2'))
    for k in ('X', 'u', 'Fv', 'rho'):
        assert np.array_equal(a[k], b[k]), k
    assert np.abs(a['X'] - c['X']).max() > 1e-6


def test_time_scale_arguments():
    s = _accelerating_box(FREE)
    with pytest.raises(ValueError):
        s.set_time_scales(0, 'euler')
    with pytest.raises(KeyError):
        s.set_time_scales(2, 'rk4')


# ---------------------------------------------------------------------------
# adaptive separation (Sec. 2.6: the separation may also be adaptive; the
# criterion of the cited work is not available, so it is the build's own:
# re-evaluate when the largest vertex displacement since the last evaluation
# exceeds a tolerance delta, or when force_every steps have passed)
# ---------------------------------------------------------------------------
def _stretched_box():
    s = _accelerating_box(PARAMS)
    X = s.get()['X']
    s.set_vertices(X.mean(0) + (X - X.mean(0)) * np.array([1.15, 1.0, 0.9]))
    return s


@pytest.mark.parametrize('integrator', ['euler', 'ab2'])
def test_adaptive_zero_tolerance_is_every_step(integrator):
    """delta = 0: every step in which anything moved re-evaluates, which is
    the default schedule (N = 1) bit for bit."""
    a = _stretched_box()
    a.set_time_scales(1, integrator)
    a.step(7)
    b = _stretched_box()
    b.set_time_scales(10 ** 9, integrator)
    b.set_force_tolerance(0.0)
    b.step(7)
    assert b.force_evaluations == 7
    ra, rb = a.get(), b.get()
    for k in ('X', 'u', 'Fv', 'rho'):
        assert np.array_equal(ra[k], rb[k]), k


def test_adaptive_infinite_tolerance():
    """delta = inf: with no bound on the interval the forces of the first
    step are held for the whole run (one evaluation); with the bound N = 4
    the schedule is the constant separation N = 4, bit for bit."""
    v, t = I.icosphere(1)
    rest = v * 2.5
    s = _stretched_box()
    s.set_time_scales(10 ** 9, 'euler')
    s.set_force_tolerance(np.inf)
    F0 = O.membrane(rest, t, PARAMS, s.get()['X'])[0]
    for n in range(9):
        s.step(1)
        assert np.array_equal(s.get()['Fv'], F0), n
    assert s.force_evaluations == 1
    a = _stretched_box()
    a.set_time_scales(4, 'ab2')
    a.step(11)
    b = _stretched_box()
    b.set_time_scales(4, 'ab2')
    b.set_force_tolerance(np.inf)
    b.step(11)
    assert b.force_evaluations == 3
    ra, rb = a.get(), b.get()
    for k in ('X', 'u', 'Fv'):
        assert np.array_equal(ra[k], rb[k]), k


@pytest.mark.parametrize('delta,N', [(0.05, 10 ** 9), (0.07, 4)])
def test_adaptive_schedule_follows_the_criterion(delta, N):
    """A cell stretched and carried by the accelerating fluid, so that the
    displacement per step grows: after each step the forces are those of the
    positions at the start of the step exactly when the criterion, evaluated
    here from the positions alone, calls for an evaluation (the first step,
    N steps since the last one, or a vertex more than delta from its
    position then), and the held ones otherwise; the evaluations are
    irregular in time."""
    v, t = I.icosphere(1)
    rest = v * 2.5
    s = _stretched_box()
    s.set_time_scales(N, 'euler')
    s.set_force_tolerance(delta)
    held, Xe, ne, steps = None, None, None, []
    for n in range(24):
        Xn = s.get()['X']
        evaluate = Xe is None or n - ne >= N or np.linalg.norm(Xn - Xe, axis=1).max() > delta
        if evaluate:
            held, Xe, ne = O.membrane(rest, t, PARAMS, Xn)[0], Xn, n
            steps.append(n)
        s.step(1)
        assert np.array_equal(s.get()['Fv'], held), n
    assert s.force_evaluations == len(steps)
    gaps = np.diff(steps)
    assert len(steps) >= 4 and len(set(gaps.tolist())) > 1, steps
