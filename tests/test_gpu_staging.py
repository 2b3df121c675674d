"""The staged collision (tiles of wall-free rows copied through shared
memory by bulk copies) against the per-node kernel on the same inputs:
identical populations, density and velocity after an odd number of steps
(both step parities), for the storage types that use it, on lattices with
walls on one axis, with periodic wrap of the shifted rows in y and z, and
with ragged tiles.  With cells the membrane forces are summed by
floating-point atomics in a varying order, so that case is compared to a
tolerance instead."""
import numpy as np
import pytest

from paper_2305_02752_gb300 import hemo
from paper_2305_02752_gb300 import inputs as I
from tests.helpers import rel_l2, small_cell_shear

pytestmark = pytest.mark.gpu


def _no_cells(cfg):
    cfg.cell_type = np.zeros(0, np.int64)
    cfg.centers = np.zeros((0, 3))
    cfg.rotations = np.zeros((0, 3, 3))
    return cfg


def _perturbed(cfg, seed):
    rng = np.random.default_rng(seed)
    u0 = np.zeros((cfg.nz, cfg.ny, cfg.nx, 3)) if cfg.init_velocity is None else cfg.init_velocity
    cfg.init_velocity = u0 + 0.004 * rng.standard_normal(u0.shape)
    if cfg.mask is not None:
        cfg.init_velocity[cfg.mask != 0] = 0.0
    return cfg


def shear_case():
    """Walls at z = 0 and z = 23 moving along x; x and y periodic (the rows
    shifted in y wrap around)."""
    return _perturbed(_no_cells(small_cell_shear(n=24, steps=7, seed=3)), 1)


def channel_case():
    """Walls at y = 0 and y = 39; x and z periodic; Poiseuille start."""
    return _perturbed(_no_cells(I.channel(nx=32, ny=40, nz=24, ncell=0, pack_iter=1)), 2)


def box_case():
    """No walls at all: every row is staged, shifts wrap in y and z."""
    cfg = _perturbed(_no_cells(I.channel(nx=48, ny=20, nz=18, ncell=0, pack_iter=1)), 3)
    cfg.mask = None
    cfg.periodic = (1, 1, 1)
    return cfg


CASES = {'shear': shear_case, 'channel': channel_case, 'box': box_case}


def run(cfg, prec, steps, options):
    sim = hemo.Simulation.from_config(cfg, prec, options=options)
    plan = sim.lattice_plan()
    sim.step(steps)
    out = sim.get_fields(hemo.HEMO_RHO | hemo.HEMO_U | hemo.HEMO_VERTS)
    out['f'] = sim.populations()
    sim.close()
    return plan, out


@pytest.mark.parametrize('prec', ['f32', 'f16', 'bf16'])
@pytest.mark.parametrize('case', sorted(CASES))
def test_staged_matches_per_node(case, prec):
    cfg = CASES[case]()
    plan, a = run(cfg, prec, 7, 0)
    plan0, b = run(cfg, prec, 7, hemo.HEMO_OPT_NO_STAGING)
    assert plan[0] > 0 and plan0 == (0, 0, 0, 0)
    if case == 'box':
        assert plan[1] == 0
    for k in ('f', 'rho', 'u'):
        assert np.array_equal(a[k], b[k]), k


def test_staged_with_cells_close_to_per_node():
    cfg = small_cell_shear(n=24, steps=9, seed=5)
    _, a = run(cfg, 'f32', 9, 0)
    _, b = run(cfg, 'f32', 9, hemo.HEMO_OPT_NO_STAGING)
    assert rel_l2(a['u'], b['u']) < 1e-6
    assert rel_l2(a['X'], b['X']) < 1e-6


@pytest.mark.parametrize('prec,stages', [('f32', 2), ('f16', 4)])
def test_channel_plan(prec, stages):
    """64x64x256 channel: rows y = 2..61 of each z-plane are wall-free (60
    rows, 15 tiles of 4 rows = 256 nodes), rows 1 and 62 go to the per-node
    kernel, rows 0 and 63 are walls.  A CTA's ring holds at most 54 KiB
    (88 B per node in FP32, 50 B with 16-bit storage)."""
    cfg = _no_cells(I.channel(ncell=0, pack_iter=1))
    sim = hemo.Simulation.from_config(cfg, prec)
    plan = sim.lattice_plan()
    sim.close()
    assert plan == (15 * 256, 2 * 256, 4, stages)


def test_no_staging_for_f64_or_unaligned_rows():
    cfg = _no_cells(I.channel(nx=30, ny=20, nz=8, ncell=0, pack_iter=1))  # 30 * 4 B is not a multiple of 16
    for prec in ('f64', 'f32'):
        sim = hemo.Simulation.from_config(cfg, prec)
        assert sim.lattice_plan() == (0, 0, 0, 0)
        sim.close()
