"""Checkpoint and resume (hemo_save_state / hemo_load_state, Sec. 2.6: a run
is paused, its state kept and the run continued) and the failure path of the
staged collision's bounded waits.

* Resume: a run of k + m steps against k steps, save, a new simulation built
  from the same configuration, load, m more steps.  Populations, density,
  velocity, vertices and membrane forces agree bit for bit: FP64 with one
  cell in shear (k odd, so the populations are saved in the swapped in-place
  layout), with forces held over 3 steps and Adams-Bashforth (the held
  forces, the centroid split and the previous velocity are part of the
  state), and BF16 storage with its row reference (per-node and staged
  collision); a state is refused by a simulation of another size or
  precision.
* Stalled wait: with HEMO_OPT_TEST_STALLED_WAIT the staged collision, and
  the FP32 interpolation before its tensor copy, wait on a barrier that
  nothing completes; the wait runs out after 2 ms, the step reports
  HEMO_ERR_CUDA through the device status, and the GPU context stays usable
  (a new simulation steps normally afterwards).
"""
import numpy as np
import pytest

from paper_2305_02752_gb300 import hemo
from paper_2305_02752_gb300 import inputs as I
from tests.helpers import small_cell_shear

pytestmark = pytest.mark.gpu


def _fields(sim):
    out = sim.get_fields(hemo.HEMO_RHO | hemo.HEMO_U | hemo.HEMO_VERTS | hemo.HEMO_FORCES)
    out['f'] = sim.populations()
    return out


def _resume_case(cfg, prec, k, m, setup=None, options=0):
    a = hemo.Simulation.from_config(cfg, prec, options=options)
    if setup:
        setup(a)
    a.step(k + m)
    ref = _fields(a)
    a.close()
    b = hemo.Simulation.from_config(cfg, prec, options=options)
    if setup:
        setup(b)
    b.step(k)
    state = b.save_state()
    b.close()
    c = hemo.Simulation.from_config(cfg, prec, options=options)
    c.load_state(state)
    c.step(m)
    got = _fields(c)
    c.close()
    for key in ref:
        assert np.array_equal(got[key], ref[key]), key


def test_resume_f64_bitwise():
    _resume_case(small_cell_shear(n=16, steps=20), 'f64', 7, 6)


def test_resume_held_forces_ab2_bitwise():
    """Forces every 3 steps, Adams-Bashforth; saved between two force
    evaluations (k = 5), so the resumed run starts on a held step."""
    _resume_case(small_cell_shear(n=16, steps=20), 'f64', 5, 8, setup=lambda s: s.set_time_scales(3, 'ab2'))


@pytest.mark.parametrize('prec', ['f32', 'bf16'])
def test_resume_reduced_precision_bitwise(prec):
    cfg = I.channel(nx=32, ny=24, nz=40, ncell=3, seed=12, pack_iter=20, exact_iter=20)
    _resume_case(cfg, prec, 9, 4)


def test_resume_staged_collision_bitwise():
    """BF16 storage through the staged collision (forced on these short
    rows), saved after an odd step."""
    cfg = I.channel(nx=32, ny=24, nz=40, ncell=3, seed=12, pack_iter=20, exact_iter=20)
    _resume_case(cfg, 'bf16', 9, 4, options=hemo.HEMO_OPT_STAGED_COLLISION)


def test_state_of_another_simulation_is_refused():
    a = hemo.Simulation.from_config(small_cell_shear(n=16, steps=2), 'f64')
    a.step(2)
    state = a.save_state()
    a.close()
    b = hemo.Simulation.from_config(small_cell_shear(n=16, steps=2), 'f32')
    with pytest.raises(hemo.HemoError) as e:
        b.load_state(state)
    assert e.value.code == hemo.HEMO_ERR_ARG
    b.close()
    c = hemo.Simulation.from_config(small_cell_shear(n=18, steps=2), 'f64')
    with pytest.raises(hemo.HemoError) as e:
        c.load_state(state)
    assert e.value.code == hemo.HEMO_ERR_ARG
    with pytest.raises(hemo.HemoError) as e:
        c.load_state(state[:100])
    assert e.value.code == hemo.HEMO_ERR_ARG
    c.close()


def test_stalled_wait_reports_and_context_survives():
    cfg = I.channel(nx=64, ny=20, nz=8, ncell=0, pack_iter=1)
    opts = hemo.HEMO_OPT_STAGED_COLLISION | hemo.HEMO_OPT_TEST_STALLED_WAIT
    sim = hemo.Simulation.from_config(cfg, 'f16', options=opts)
    assert sim.lattice_plan()[0] > 0  # the staged kernel runs on every step
    sim.step(1)   # the staged kernel's wait runs out
    with pytest.raises(hemo.HemoError) as e:
        sim.sync()
    assert e.value.code == hemo.HEMO_ERR_CUDA
    assert 'timed out' in str(e.value)
    sim.close()
    # the context is still usable
    ok = hemo.Simulation.from_config(cfg, 'f16', options=hemo.HEMO_OPT_STAGED_COLLISION)
    ok.step(3)
    ok.sync()
    u = ok.get_fields(hemo.HEMO_U)['u']
    ok.close()
    assert np.isfinite(u).all()


def test_interpolation_stalled_wait_reports_and_context_survives():
    cfg = I.channel(nx=32, ny=32, nz=64, ncell=6, seed=3, steps=4, pack_iter=20, exact_iter=10)
    sim = hemo.Simulation.from_config(cfg, 'f32', options=hemo.HEMO_OPT_TEST_STALLED_WAIT)
    sim.step(1)   # the interpolation's first wait runs out in the bins staged by tensor copy
    with pytest.raises(hemo.HemoError) as e:
        sim.sync()
    assert e.value.code == hemo.HEMO_ERR_CUDA
    assert 'timed out' in str(e.value)
    sim.close()
    ok = hemo.Simulation.from_config(cfg, 'f32')
    ok.step(3)
    ok.sync()
    assert np.isfinite(ok.get_fields(hemo.HEMO_VERTS)['X']).all()
    ok.close()
