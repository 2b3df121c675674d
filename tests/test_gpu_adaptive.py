"""Adaptive time-scale separation (Sec. 2.6: the separation may be adaptive;
the criterion is the library's own: the membrane forces are evaluated again
when a vertex has moved more than a tolerance since the last evaluation, or
when force_every steps have passed) on the CUDA path, against the oracle
with the same settings.  The decision is taken on the device every step.

* FP64, a red cell in shear whose displacement per step grows as it starts
  to tank-tread, so that the evaluations come at irregular intervals:
  relative L2 <= 1e-12 (u, X, forces), both integrators.
* FP32, a small channel suspension, 200 steps: velocity <= 1e-5.
* Limits, bit for bit on the GPU: tolerance 0 is the default schedule;
  infinite tolerance with force_every = 4 is the constant separation N = 4.
* Arguments and the states that refuse it; checkpoint and resume with the
  adaptive decision words in the saved state.
"""
import numpy as np
import pytest

import oracle as O
from paper_2305_02752_gb300 import hemo
from paper_2305_02752_gb300 import inputs as I
from tests.helpers import assert_close, forces_close, small_cell_shear

pytestmark = pytest.mark.gpu

F64_TOL = 1e-12
F32_TOL = 1e-5


def run_both(cfg, precision, steps, delta, force_every, integrator):
    sim = hemo.Simulation.from_config(cfg, precision)
    ref = O.from_config(cfg)
    sim.set_time_scales(force_every, integrator)
    ref.set_time_scales(force_every, integrator)
    sim.set_force_tolerance(delta)
    ref.set_force_tolerance(delta)
    sim.step(steps)
    ref.step(steps)
    got = sim.get_fields()
    got['evaluations'] = sim.force_evaluations
    sim.close()
    return got, ref.get(), ref.force_evaluations


@pytest.mark.parametrize('integrator', ['euler', 'ab2'])
@pytest.mark.parametrize('delta,force_every', [(0.0031, 10 ** 9), (0.0017, 7)])
def test_shear_cell_f64(delta, force_every, integrator):
    cfg = small_cell_shear(steps=40)
    got, exp, nevals = run_both(cfg, 'f64', 40, delta, force_every, integrator)
    assert 3 <= nevals <= 30, nevals  # held steps and evaluations both occur
    assert got['evaluations'] == nevals  # the device decided the same steps
    for k in ('u', 'X'):
        assert_close(got[k], exp[k], F64_TOL, k)
    assert forces_close(got['Fv'], exp['Fv'], cfg)


def test_channel_f32_200_steps():
    cfg = I.channel(nx=32, ny=32, nz=64, ncell=6, seed=3, steps=200, pack_iter=50, exact_iter=50)
    got, exp, nevals = run_both(cfg, 'f32', 200, 0.053, 10, 'ab2')
    assert 40 <= nevals <= 120, nevals
    assert abs(got['evaluations'] - nevals) <= 2  # (FP32 displacements decide near the threshold)
    assert_close(got['u'], exp['u'], F32_TOL, 'u')
    assert_close(got['X'], exp['X'], F32_TOL, 'X')


def _fields(cfg, precision, steps, setup):
    sim = hemo.Simulation.from_config(cfg, precision)
    setup(sim)
    sim.step(steps)
    out = sim.get_fields(hemo.HEMO_U | hemo.HEMO_VERTS | hemo.HEMO_FORCES)
    sim.close()
    return out


@pytest.mark.parametrize('precision', ['f64', 'f32'])
def test_zero_tolerance_is_the_default_schedule(precision):
    cfg = small_cell_shear(steps=12)
    a = _fields(cfg, precision, 12, lambda s: None)

    def adaptive(s):
        s.set_time_scales(10 ** 9, 'euler')
        s.set_force_tolerance(0.0)
    b = _fields(cfg, precision, 12, adaptive)
    for k in a:
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize('precision', ['f64', 'f32'])
def test_infinite_tolerance_is_the_constant_schedule(precision):
    cfg = small_cell_shear(steps=14)
    a = _fields(cfg, precision, 14, lambda s: s.set_time_scales(4, 'ab2'))

    def adaptive(s):
        s.set_time_scales(4, 'ab2')
        s.set_force_tolerance(np.inf)
    b = _fields(cfg, precision, 14, adaptive)
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_arguments_and_refusals():
    cfg = small_cell_shear(steps=4)
    sim = hemo.Simulation.from_config(cfg, 'f64')
    with pytest.raises(hemo.HemoError) as e:
        sim.set_force_tolerance(float('nan'))
    assert e.value.code == hemo.HEMO_ERR_ARG
    sim.set_force_tolerance(0.01)
    sim.step(2)
    with pytest.raises(hemo.HemoError) as e:
        sim.record(100)
    assert e.value.code == hemo.HEMO_ERR_STATE
    sim.set_force_tolerance(-1.0)  # back to the constant schedule
    sim.record(100)
    with pytest.raises(hemo.HemoError) as e:
        sim.set_force_tolerance(0.01)
    assert e.value.code == hemo.HEMO_ERR_STATE
    sim.close()
    box = I.shear_cell(n=24, ncell=1, seed=9, steps=4)
    box.mask, box.periodic, box.wall_velocity = None, (1, 1, 1), np.zeros((2, 3))
    le = hemo.Simulation.from_config(box, 'f64')
    le.set_lees_edwards(0.01)
    with pytest.raises(hemo.HemoError) as e:
        le.set_force_tolerance(0.01)
    assert e.value.code == hemo.HEMO_ERR_STATE
    le.close()


def test_resume_with_adaptive_separation_bitwise():
    cfg = small_cell_shear(steps=30)

    def setup(s):
        s.set_time_scales(6, 'ab2')
        s.set_force_tolerance(0.0023)
    a = hemo.Simulation.from_config(cfg, 'f64')
    setup(a)
    a.step(30)
    ref = a.get_fields(hemo.HEMO_U | hemo.HEMO_VERTS | hemo.HEMO_FORCES)
    a.close()
    b = hemo.Simulation.from_config(cfg, 'f64')
    setup(b)
    b.step(17)
    state = b.save_state()
    b.close()
    c = hemo.Simulation.from_config(cfg, 'f64')
    c.load_state(state)
    c.step(13)
    got = c.get_fields(hemo.HEMO_U | hemo.HEMO_VERTS | hemo.HEMO_FORCES)
    c.close()
    for k in ref:
        assert np.array_equal(got[k], ref[k]), k


def test_evaluation_count_across_schedules():
    """Constant schedules are counted on the host, the adaptive one on the
    device; the total over a switch of schedule and across a checkpoint
    equals the oracle's."""
    cfg = small_cell_shear(steps=24)
    sim = hemo.Simulation.from_config(cfg, 'f64')
    ref = O.from_config(cfg)
    for s in (sim, ref):
        s.set_time_scales(3, 'euler')
        s.step(10)  # steps 0, 3, 6, 9
    assert sim.force_evaluations == ref.force_evaluations == 4
    for s in (sim, ref):
        s.set_force_tolerance(0.0021)
        s.step(7)
    state = sim.save_state()
    sim.close()
    sim = hemo.Simulation.from_config(cfg, 'f64')
    sim.load_state(state)
    assert sim.force_evaluations == ref.force_evaluations
    for s in (sim, ref):
        s.set_force_tolerance(-1.0)
        s.set_time_scales(2, 'euler')
        s.step(5)
    assert sim.force_evaluations == ref.force_evaluations
    sim.close()
