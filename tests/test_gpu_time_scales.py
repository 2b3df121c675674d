"""Time-scale separation (membrane forces every N steps, held in between)
and the Adams-Bashforth vertex integrator (Sec. 2.6) on the CUDA path,
against the oracle with the same settings and seeded inputs.  Tolerances as
for the default step: FP64 relative L2 <= 1e-12, FP32 velocity relative L2
<= 1e-5 after 200 steps."""
import numpy as np
import pytest

import oracle as O
from paper_2305_02752_gb300 import hemo
from paper_2305_02752_gb300 import inputs as I
from tests.helpers import assert_close, forces_close, rel_l2, small_cell_shear

pytestmark = pytest.mark.gpu

F64_TOL = 1e-12
F32_TOL = 1e-5


def run_both(cfg, precision, steps, force_every, integrator, switch_at=0):
    """Both sides take `switch_at` default steps, then the setting, then the
    remaining steps."""
    sim = hemo.Simulation.from_config(cfg, precision)
    ref = O.from_config(cfg)
    if switch_at:
        sim.step(switch_at)
        ref.step(switch_at)
    sim.set_time_scales(force_every, integrator)
    ref.set_time_scales(force_every, integrator)
    sim.step(steps - switch_at)
    ref.step(steps - switch_at)
    got = sim.get_fields()
    sim.close()
    return got, ref.get()


@pytest.mark.parametrize('force_every,integrator,steps', [
    (3, 'ab2', 20), (3, 'ab2', 22), (4, 'ab2', 21), (1, 'ab2', 20), (5, 'euler', 21)])
def test_coupled_small_f64(force_every, integrator, steps):
    """Single cell in shear; both step parities at the end, hold lengths that
    do and do not divide the step count."""
    cfg = small_cell_shear(steps=steps)
    got, exp = run_both(cfg, 'f64', steps, force_every, integrator)
    for k in ('u', 'X', 'rho'):
        assert_close(got[k], exp[k], F64_TOL, k)
    assert forces_close(got['Fv'], exp['Fv'], cfg)
    assert_close(got['cellstats'], exp['cellstats'], F64_TOL)


def test_switch_after_odd_step_count_f64():
    """The setting made after 7 default steps: the hold schedule and the
    Euler start of Adams-Bashforth count from there."""
    cfg = small_cell_shear(n=24, steps=26, center=[0.3, 23.6, 11.5])
    got, exp = run_both(cfg, 'f64', 26, 4, 'ab2', switch_at=7)
    for k in ('u', 'X'):
        assert_close(got[k], exp[k], F64_TOL, k)
    assert forces_close(got['Fv'], exp['Fv'], cfg)


def test_c0_f64_500_steps_ab2_every_4():
    """Single red cell (642 vertices) in a 32^3 shear box, forces every 4
    steps, Adams-Bashforth, 500 steps."""
    cfg = I.shear_cell()
    got, exp = run_both(cfg, 'f64', 500, 4, 'ab2')
    for k in ('u', 'X', 'rho'):
        assert_close(got[k], exp[k], F64_TOL, k)
    assert forces_close(got['Fv'], exp['Fv'], cfg)


def test_channel_f32_200_steps_ab2_every_4():
    """Small channel suspension (red cells and platelets), FP32."""
    cfg = I.channel(nx=32, ny=32, nz=64, ncell=10, seed=3, platelet_ratio=0.5, pack_iter=100, exact_iter=0)
    got, exp = run_both(cfg, 'f32', 200, 4, 'ab2')
    assert_close(got['u'], exp['u'], F32_TOL)
    assert_close(got['X'], exp['X'], F32_TOL)


@pytest.mark.parametrize('precision', ['f32', 'bf16'])
def test_forces_held_bit_for_bit(precision):
    """With N = 3 the forces read after steps 1, 2, 3 of a hold are the same
    bits, and the next evaluation changes them."""
    cfg = small_cell_shear(steps=12)
    sim = hemo.Simulation.from_config(cfg, precision)
    sim.step(2)
    sim.set_time_scales(3, 'euler')
    F = []
    for _ in range(6):
        sim.step(1)
        F.append(sim.get_fields(hemo.HEMO_FORCES)['Fv'])
    sim.close()
    assert np.array_equal(F[0], F[1]) and np.array_equal(F[1], F[2])
    assert np.array_equal(F[3], F[4]) and np.array_equal(F[4], F[5])
    assert not np.array_equal(F[2], F[3])


def test_record_needs_default_time_scales():
    cfg = small_cell_shear(steps=4)
    sim = hemo.Simulation.from_config(cfg, 'f64')
    sim.set_time_scales(2, 'euler')
    with pytest.raises(hemo.HemoError) as e:
        sim.record(2)
    assert e.value.code == hemo.HEMO_ERR_STATE
    sim.set_time_scales(1, 'euler')
    sim.record(2)
    with pytest.raises(hemo.HemoError) as e:
        sim.set_time_scales(1, 'ab2')
    assert e.value.code == hemo.HEMO_ERR_STATE
    with pytest.raises(hemo.HemoError) as e:
        sim.set_time_scales(0, 'euler')
    assert e.value.code == hemo.HEMO_ERR_ARG
    sim.close()
