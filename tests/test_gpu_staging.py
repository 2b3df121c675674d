"""The staged collision (tiles of wall-free rows copied through shared
memory by bulk copies; HEMO_OPT_STAGED_COLLISION) against the per-node
kernel (the default) on the same inputs:
identical populations, density and velocity after an odd number of steps
(both step parities staged), for the storage types that use it (16-bit), on
lattices with walls on one axis, with periodic wrap of the shifted rows in
y and z, with ragged tiles, with long rows, and with cells."""
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


def wide_case():
    """Rows of 264 nodes: three rows per tile, the last tile of each plane
    ragged (13 interior rows); walls at y = 0 and 16, x and z periodic."""
    return _perturbed(_no_cells(I.channel(nx=264, ny=17, nz=10, ncell=0, pack_iter=1)), 4)


CASES = {'shear': shear_case, 'channel': channel_case, 'box': box_case, 'wide': wide_case}


def run(cfg, prec, steps, options):
    sim = hemo.Simulation.from_config(cfg, prec, options=options)
    plan = sim.lattice_plan()
    sim.step(steps)
    out = sim.get_fields(hemo.HEMO_RHO | hemo.HEMO_U | hemo.HEMO_VERTS)
    out['f'] = sim.populations()
    sim.close()
    return plan, out


@pytest.mark.parametrize('prec', ['f16', 'bf16'])
@pytest.mark.parametrize('case', sorted(CASES))
def test_staged_matches_per_node(case, prec):
    cfg = CASES[case]()
    plan, a = run(cfg, prec, 7, hemo.HEMO_OPT_STAGED_COLLISION)
    plan0, b = run(cfg, prec, 7, 0)
    assert plan[0] > 0 and plan0 == (0, 0, 0, 0)
    if case == 'box':
        assert plan[1] == 0
    for k in ('f', 'rho', 'u'):
        assert np.array_equal(a[k], b[k]), k


def test_staged_with_cells_matches_per_node():
    """With cells: the membrane forces are gathered in a fixed order and the
    spreading is fixed-point, so the coupled step is reproducible and the
    two collision paths agree bit for bit."""
    cfg = small_cell_shear(n=24, steps=9, seed=5)
    _, a = run(cfg, 'f16', 9, hemo.HEMO_OPT_STAGED_COLLISION)
    _, b = run(cfg, 'f16', 9, 0)
    for k in ('f', 'u', 'X'):
        assert np.array_equal(a[k], b[k]), k


def test_staged_with_internal_viscosity_matches_per_node():
    """Cells with an internal viscosity ratio: the staged collision relaxes
    the inside nodes with their own rate, as the per-node kernel does (the
    same bits after an odd number of steps)."""
    cfg = small_cell_shear(n=24, steps=9, seed=7)

    def run_visc(opts):
        sim = hemo.Simulation.from_config(cfg, 'f16', options=opts)
        sim.set_viscosity_ratio(5.0)
        plan = sim.lattice_plan()
        sim.step(9)
        out = sim.get_fields(hemo.HEMO_U | hemo.HEMO_VERTS)
        out['f'] = sim.populations()
        sim.close()
        return plan, out
    plan, a = run_visc(hemo.HEMO_OPT_STAGED_COLLISION)
    plan0, b = run_visc(hemo.HEMO_OPT_UNSTAGED_COLLISION)
    assert plan[0] > 0 and plan0 == (0, 0, 0, 0)
    for k in ('f', 'u', 'X'):
        assert np.array_equal(a[k], b[k]), k


def test_channel_plan():
    """64x64x256 channel, 16-bit storage: rows y = 2..61 of each z-plane are
    wall-free (60 rows: tiles of 16, 16, 16 and 12 rows, a stage holding
    1024 nodes), rows 1 and 62 go to the per-node kernel, rows 0 and 63 are
    walls.  The ring of the one CTA per SM takes four stages of 1024 nodes at
    50 B (19 two-byte populations and three FP32 force components)."""
    cfg = _no_cells(I.channel(ncell=0, pack_iter=1))
    for prec in ('f16', 'bf16'):
        sim = hemo.Simulation.from_config(cfg, prec, options=hemo.HEMO_OPT_STAGED_COLLISION)
        plan = sim.lattice_plan()
        sim.close()
        assert plan == (4 * 256, 2 * 256, 16, 4)
        sim = hemo.Simulation.from_config(cfg, prec)  # default: per-node kernel only
        assert sim.lattice_plan() == (0, 0, 0, 0)
        sim.close()


def test_wide_plan():
    """Rows of 1000 nodes (the pipe's length): one row per tile, staged by
    default (rows of at least 512 nodes) and on request alike, not with
    HEMO_OPT_UNSTAGED_COLLISION; rows of 1032 nodes are longer than a stage
    holds and are not staged."""
    cfg = _no_cells(I.channel(nx=1000, ny=12, nz=4, ncell=0, pack_iter=1))
    for opts in (0, hemo.HEMO_OPT_STAGED_COLLISION):
        sim = hemo.Simulation.from_config(cfg, 'bf16', options=opts)
        plan = sim.lattice_plan()
        sim.close()
        assert plan == (8 * 4, 2 * 4, 1, 4)
    for opts in (hemo.HEMO_OPT_UNSTAGED_COLLISION, hemo.HEMO_OPT_UNSTAGED_COLLISION | hemo.HEMO_OPT_STAGED_COLLISION):
        sim = hemo.Simulation.from_config(cfg, 'bf16', options=opts)
        assert sim.lattice_plan() == (0, 0, 0, 0)
        sim.close()
    cfg = _no_cells(I.channel(nx=1032, ny=12, nz=4, ncell=0, pack_iter=1))
    sim = hemo.Simulation.from_config(cfg, 'bf16', options=hemo.HEMO_OPT_STAGED_COLLISION)
    assert sim.lattice_plan() == (0, 0, 0, 0)
    sim.close()


@pytest.mark.parametrize('prec', ['f16', 'bf16'])
def test_default_staging_matches_per_node(prec):
    """Rows of 520 nodes are staged by default: the same bits as the
    per-node kernel (HEMO_OPT_UNSTAGED_COLLISION) after an odd number of
    steps."""
    cfg = _perturbed(_no_cells(I.channel(nx=520, ny=14, nz=6, ncell=0, pack_iter=1)), 5)
    plan, a = run(cfg, prec, 7, 0)
    plan0, b = run(cfg, prec, 7, hemo.HEMO_OPT_UNSTAGED_COLLISION)
    assert plan[0] > 0 and plan0 == (0, 0, 0, 0)
    for k in ('f', 'rho', 'u'):
        assert np.array_equal(a[k], b[k]), k


def test_no_staging_for_4_and_8_byte_storage_or_unaligned_rows():
    cfg = _no_cells(I.channel(nx=64, ny=20, nz=8, ncell=0, pack_iter=1))
    for prec in ('f64', 'f32'):
        sim = hemo.Simulation.from_config(cfg, prec, options=hemo.HEMO_OPT_STAGED_COLLISION)
        assert sim.lattice_plan() == (0, 0, 0, 0)
        sim.close()
    cfg = _no_cells(I.channel(nx=60, ny=20, nz=8, ncell=0, pack_iter=1))  # 60 * 2 B is not a multiple of 16
    sim = hemo.Simulation.from_config(cfg, 'f16', options=hemo.HEMO_OPT_STAGED_COLLISION)
    assert sim.lattice_plan() == (0, 0, 0, 0)
    sim.close()
