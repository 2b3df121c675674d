"""Lees-Edwards boundary (Sec. 2.5) on the CUDA path against the oracle with
the same image velocity: the lattice alone (populations, density, velocity)
and coupled runs with cells across the plane and crossing it, FP64 relative
L2 <= 1e-12, FP32 velocity and vertices <= 1e-5 after 200 steps."""
import dataclasses

import numpy as np
import pytest

import oracle as O
from paper_2305_02752_gb300 import hemo
from paper_2305_02752_gb300 import inputs as I
from tests.helpers import assert_close, direction_map, forces_close, rel_l2, small_cell_shear

pytestmark = pytest.mark.gpu

F64_TOL = 1e-12
F32_TOL = 1e-5


def _le_config(n=24, center=(11.3, 12.1, 23.2), steps=20, seed=5, uz=0.0):
    cfg = small_cell_shear(n=n, steps=steps, seed=seed, center=list(center))
    rng = np.random.default_rng(seed)
    u0 = 0.004 * rng.normal(size=(n, n, n, 3))
    u0[..., 2] += uz
    return dataclasses.replace(cfg, mask=None, periodic=(1, 1, 1), wall_velocity=np.zeros((2, 3)),
                               init_velocity=u0)


def _run_both(cfg, precision, steps, U):
    sim = hemo.Simulation.from_config(cfg, precision)
    sim.set_lees_edwards(U)
    sim.step(steps)
    got = sim.get_fields()
    got['f'] = sim.populations()
    sim.close()
    ref = O.from_config(cfg)
    ref.set_lees_edwards(U)
    ref.step(steps)
    exp = ref.get()
    exp['f'] = ref.populations()
    return got, exp


@pytest.mark.parametrize('steps', [1, 2, 13])
def test_lattice_only_f64(steps):
    cfg = dataclasses.replace(_le_config(n=12, seed=2), cell_type=np.zeros(0, np.int64), centers=np.zeros((0, 3)),
                              rotations=np.zeros((0, 3, 3)))
    got, exp = _run_both(cfg, 'f64', steps, 0.037)
    perm = direction_map()
    assert_close(got['f'][..., :], exp['f'][..., perm], F64_TOL)
    for k in ('u', 'rho'):
        assert_close(got[k], exp[k], F64_TOL, k)


@pytest.mark.parametrize('center,uz', [((11.3, 12.1, 23.2), 0.0), ((5.6, 20.4, 0.4), 0.0), ((11.3, 12.1, 23.5), 0.02)])
def test_coupled_f64(center, uz):
    """A red cell across the top plane, across the bottom plane, and one
    carried upwards through the plane (its centroid crosses)."""
    steps = 30
    cfg = _le_config(center=center, uz=uz, steps=steps)
    got, exp = _run_both(cfg, 'f64', steps, 0.02)
    for k in ('u', 'X', 'rho'):
        assert_close(got[k], exp[k], F64_TOL, k)
    assert forces_close(got['Fv'], exp['Fv'], cfg)
    if uz:
        assert exp['cellstats'][0, 2] < 2.0  # the centroid went through z = nz


def test_coupled_f32_200_steps():
    cfg = _le_config(center=(11.3, 12.1, 23.2), steps=200)
    got, exp = _run_both(cfg, 'f32', 200, 0.02)
    assert_close(got['u'], exp['u'], F32_TOL)
    assert_close(got['X'], exp['X'], F32_TOL)


def test_arguments_and_state():
    with_walls = small_cell_shear(steps=2)
    sim = hemo.Simulation.from_config(with_walls, 'f32')
    with pytest.raises(hemo.HemoError) as e:
        sim.set_lees_edwards(0.01)
    assert e.value.code == hemo.HEMO_ERR_ARG
    sim.close()
    sim = hemo.Simulation.from_config(_le_config(steps=2), 'f64')
    with pytest.raises(hemo.HemoError) as e:
        sim.set_lees_edwards(0.5)
    assert e.value.code == hemo.HEMO_ERR_ARG
    sim.set_lees_edwards(0.01)
    with pytest.raises(hemo.HemoError) as e:
        sim.set_time_scales(2, 'euler')
    assert e.value.code == hemo.HEMO_ERR_STATE
    with pytest.raises(hemo.HemoError) as e:
        sim.record(2)
    assert e.value.code == hemo.HEMO_ERR_STATE
    sim.step(1)
    sim.close()


def test_with_large_deformation_terms_f64():
    """Lees-Edwards with the large-deformation terms on, a cell across the
    plane: FP64 against the oracle with the same settings.  The internal
    viscosity is refused with the boundary (its rays would cross the
    displaced plane)."""
    steps = 20
    cfg = _le_config(center=(11.3, 12.1, 23.2), steps=steps)
    cfg.meshes = [dataclasses.replace(mt, k_local=0.05, theta_m=0.5) for mt in cfg.meshes]
    sim = hemo.Simulation.from_config(cfg, 'f64')
    sim.set_lees_edwards(0.02)
    with pytest.raises(hemo.HemoError) as e:
        sim.set_viscosity_ratio(5.0)
    assert e.value.code == hemo.HEMO_ERR_STATE
    sim.step(steps)
    got = sim.get_fields()
    sim.close()
    ref = O.from_config(cfg)
    ref.set_lees_edwards(0.02)
    ref.step(steps)
    exp = ref.get()
    for k in ('u', 'X', 'rho'):
        assert_close(got[k], exp[k], F64_TOL, k)


@pytest.mark.parametrize('prec', ['f16', 'bf16'])
def test_16bit_storage_against_fp32(prec):
    """The two-array streaming with 16-bit deviations stays within the
    precision form's error of the FP32 run (1e-3 FP16, 1e-2 BF16 after 100
    steps)."""
    cfg = _le_config(center=(11.3, 12.1, 23.2), steps=100)
    out = {}
    for p in ('f32', prec):
        sim = hemo.Simulation.from_config(cfg, p)
        sim.set_lees_edwards(0.02)
        sim.step(100)
        out[p] = sim.get_fields(hemo.HEMO_U)['u'].astype(np.float64)
        sim.close()
    assert_close(out[prec], out['f32'], (1e-3 if prec == 'f16' else 1e-2))
