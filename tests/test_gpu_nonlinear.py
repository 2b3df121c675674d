"""The optional large-deformation terms (nonlinear bending with a maximum
deviation theta_m, local per-triangle area) on the CUDA path against the
oracle with the same parameters: FP64 relative L2 <= 1e-12, FP32 velocity
and vertex relative L2 <= 1e-5 after 200 steps."""
import dataclasses

import numpy as np
import pytest

import oracle as O
from paper_2305_02752_gb300 import hemo
from paper_2305_02752_gb300 import inputs as I
from tests.helpers import assert_close, forces_close, rel_l2, run_both, small_cell_shear

pytestmark = pytest.mark.gpu

F64_TOL = 1e-12
F32_TOL = 1e-5


def _with_terms(cfg, k_local=0.05, theta_m=0.5):
    cfg.meshes = [dataclasses.replace(mt, k_local=k_local, theta_m=theta_m) for mt in cfg.meshes]
    return cfg


@pytest.mark.parametrize('steps', [20, 21])
def test_single_cell_f64(steps):
    cfg = _with_terms(small_cell_shear(steps=steps))
    got, exp = run_both(cfg, 'f64', steps)
    for k in ('u', 'X', 'rho'):
        assert_close(got[k], exp[k], F64_TOL, k)
    assert forces_close(got['Fv'], exp['Fv'], cfg)
    # the terms matter at this tolerance
    ref = O.from_config(small_cell_shear(steps=steps))
    ref.step(steps)
    assert rel_l2(ref.get()['Fv'], exp['Fv']) > 1e-6


@pytest.mark.parametrize('which', ['bend', 'local'])
def test_each_term_alone_f64(which):
    cfg = small_cell_shear(steps=15)
    cfg = _with_terms(cfg, k_local=0.05 if which == 'local' else 0.0, theta_m=0.5 if which == 'bend' else 0.0)
    got, exp = run_both(cfg, 'f64', 15)
    for k in ('u', 'X'):
        assert_close(got[k], exp[k], F64_TOL, k)
    assert forces_close(got['Fv'], exp['Fv'], cfg)


def test_channel_f32_200_steps():
    cfg = _with_terms(I.channel(nx=32, ny=32, nz=64, ncell=10, seed=3, platelet_ratio=0.5, pack_iter=100, exact_iter=0))
    got, exp = run_both(cfg, 'f32', 200)
    assert_close(got['u'], exp['u'], F32_TOL)
    assert_close(got['X'], exp['X'], F32_TOL)


def test_record_refuses_the_optional_terms():
    sim = hemo.Simulation.from_config(_with_terms(small_cell_shear(steps=4)), 'f64')
    with pytest.raises(hemo.HemoError) as e:
        sim.record(2)
    assert e.value.code == hemo.HEMO_ERR_STATE
    sim.close()


def test_bad_parameters_are_rejected():
    cfg = _with_terms(small_cell_shear(steps=2), k_local=-1.0)
    with pytest.raises(hemo.HemoError) as e:
        hemo.Simulation.from_config(cfg, 'f32')
    assert e.value.code == hemo.HEMO_ERR_ARG
