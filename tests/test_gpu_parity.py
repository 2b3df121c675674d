"""CUDA path (through the C ABI) against the CPU oracle on the same seeded
inputs.  Integer work is compared bit-exactly; FP64 results to relative L2
1e-12 (the FP64 path differs from the oracle only in summation order and in
the split of positions into FP64 centroid + FP64 offset); FP32 results to
1e-5 velocity relative L2 (FP32 rounding, ~1e-7 per operation, accumulated
over a few hundred steps)."""
import numpy as np
import pytest

import oracle as O
from paper_2305_02752_gb300 import hemo
from paper_2305_02752_gb300 import inputs as I
from tests.helpers import assert_close, direction_map, forces_close, rel_l2, run_both, small_cell_shear

pytestmark = pytest.mark.gpu

F64_TOL = 1e-12
F32_TOL = 1e-5


def _lbm_box(nx, ny, nz, per, seed, walls=True, g=(2e-6, -1e-6, 0.0)):
    rng = np.random.default_rng(seed)
    mask = None
    if walls:
        mask = I.plate_mask(nx, ny, nz, axis=2, lo_id=I.WALL_A, hi_id=I.WALL_B)
    u0 = 0.02 * rng.normal(size=(nz, ny, nx, 3))
    wv = np.array([[-0.01, 0.002, 0], [0.01, 0, -0.003]])
    return mask, u0, wv, np.array(g)


@pytest.mark.parametrize('steps', [1, 2, 7, 8])
@pytest.mark.parametrize('dims', [(16, 12, 10), (5, 3, 9), (1, 1, 12)])
def test_lattice_only_f64(steps, dims):
    """Collide + stream with force, moving walls and periodic edges, both
    in-place parities, ragged and degenerate sizes."""
    nx, ny, nz = dims
    mask, u0, wv, g = _lbm_box(nx, ny, nz, (1, 1, 0), 3)
    sim = hemo.Simulation(nx, ny, nz, 0.8, 'f64', (1, 1, 0), mask, wv, g)
    sim.set_velocity(u0)
    sim.step(steps)
    got = sim.get_fields(hemo.HEMO_RHO | hemo.HEMO_U)
    fg = sim.populations()
    sim.close()
    ref = O.OracleSim(nx, ny, nz, 0.8, (1, 1, 0), mask, wv, g)
    ref.set_velocity(u0)
    ref.step(steps)
    exp = ref.get()
    fo = ref.populations()[..., direction_map()]
    fluid = mask == 0
    assert_close(fg[fluid], fo[fluid], F64_TOL)
    assert_close(got['rho'][fluid], exp['rho'][fluid], F64_TOL)
    assert_close(got['u'], exp['u'], F64_TOL)


def test_fully_periodic_no_walls_f64():
    rng = np.random.default_rng(1)
    n = 9
    u0 = 0.03 * rng.normal(size=(n, n, n, 3))
    sim = hemo.Simulation(n, n, n, 0.7, 'f64', (1, 1, 1), None, None, [1e-5, 0, 2e-5])
    sim.set_velocity(u0)
    sim.step(11)
    got = sim.get_fields(hemo.HEMO_U | hemo.HEMO_RHO)
    ref = O.OracleSim(n, n, n, 0.7, (1, 1, 1), None, None, np.array([1e-5, 0, 2e-5]))
    ref.set_velocity(u0)
    ref.step(11)
    exp = ref.get()
    assert_close(got['u'], exp['u'], F64_TOL)
    assert_close(got['rho'], exp['rho'], F64_TOL)


def test_wall_links_bit_exact():
    """Integer neighbour work: the library's wall links against the oracle's,
    mapped by velocity vector, plus the wall ids by brute force."""
    rng = np.random.default_rng(5)
    nx, ny, nz = 11, 9, 7
    mask = (rng.random((nz, ny, nx)) < 0.2).astype(np.uint8) * rng.integers(1, 4, size=(nz, ny, nx)).astype(np.uint8)
    per = (1, 0, 1)
    sim = hemo.Simulation(nx, ny, nz, 1.0, 'f32', per, mask)
    lk = sim.links()
    sim.close()
    ref = O.OracleSim(nx, ny, nz, 1.0, per, mask)
    lo = ref.wall_links()
    dm = direction_map()
    cg, _ = hemo.velocity_set()
    for i in range(19):
        code = (lk >> np.uint64(2 * i)) & np.uint64(3)
        assert np.array_equal(code != 0, ((lo >> np.uint32(dm[i])) & np.uint32(1)) == 1), i
        # wall id by brute force
        z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing='ij')
        xx, yy, zz = (x + cg[i, 0]) % nx, y + cg[i, 1], (z + cg[i, 2]) % nz
        outside = (yy < 0) | (yy >= ny)
        nb = np.where(outside, 1, mask[zz, np.clip(yy, 0, ny - 1), xx])
        expect = np.where(mask == 0, nb, 0).astype(np.uint64)
        assert np.array_equal(code, expect), i


@pytest.mark.parametrize('sub', [0, 2, 3])
def test_edge_tables_bit_exact(sub):
    v, t = I.icosphere(sub)
    mt = I.MeshType('m', I.evans_fung(v, 10.0), t, 1, 1, 1, 1, 1e-7, 0.015, 3.0)
    sim = hemo.Simulation(16, 16, 16, 1.0, 'f32')
    sim.add_cells(mt, np.zeros((0, 3)), np.zeros((0, 3, 3)))
    eg = sim.edges(0)
    sim.close()
    assert np.array_equal(eg, O.build_edges(len(v), t))


def test_bins_bit_exact():
    """Vertex binning (key, stable permutation, block starts) against the
    oracle on identical positions, including positions exactly on lattice
    planes and wrapped across periodic edges."""
    cfg = I.channel(nx=40, ny=32, nz=48, ncell=6, seed=11, platelet_ratio=0.5, pack_iter=50, exact_iter=0)
    sim = hemo.Simulation.from_config(cfg, 'f32')
    rng = np.random.default_rng(2)
    X = I.cell_vertices(cfg)
    X[:, 0] += rng.normal(size=len(X)) * 30
    X[:, 2] += rng.normal(size=len(X)) * 30
    X[::5] = np.floor(X[::5])
    sim.set_vertices(X)
    Xg = sim.get_fields(hemo.HEMO_VERTS)['X']
    key, perm, start = sim.bins()
    sim.close()
    ref = O.from_config(cfg)
    k2, p2, s2 = ref.bins(Xg, 8)
    assert np.array_equal(key, k2)
    assert np.array_equal(perm, p2)
    assert np.array_equal(start, s2)


@pytest.mark.parametrize('steps', [1, 20, 21])
def test_coupled_small_f64(steps):
    """Single cell in shear: membrane forces, spreading, LBM, interpolation
    and Euler move, FP64 against the oracle."""
    cfg = small_cell_shear(steps=steps)
    got, exp = run_both(cfg, 'f64', steps)
    for k in ('u', 'X', 'rho'):
        assert_close(got[k], exp[k], F64_TOL, k)
    assert forces_close(got['Fv'], exp['Fv'], cfg)
    assert_close(got['cellstats'], exp['cellstats'], F64_TOL)


def test_coupled_cell_across_periodic_edge_f64():
    """A cell straddling the periodic x and y edges (stencils and bins wrap)."""
    cfg = small_cell_shear(n=24, steps=15, center=[0.3, 23.6, 11.5])
    got, exp = run_both(cfg, 'f64', 15)
    for k in ('u', 'X'):
        assert_close(got[k], exp[k], F64_TOL, k)
    assert forces_close(got['Fv'], exp['Fv'], cfg)


def test_coupled_c0_f64_500_steps():
    """Config: single red cell (642 vertices) in a 32^3 shear box, FP64, 500
    steps; relative L2 <= 1e-12 against the oracle."""
    cfg = I.shear_cell()
    got, exp = run_both(cfg, 'f64', 500)
    for k in ('u', 'X', 'rho'):
        assert_close(got[k], exp[k], F64_TOL, k)
    assert forces_close(got['Fv'], exp['Fv'], cfg)
    assert_close(got['cellstats'], exp['cellstats'], F64_TOL)


def test_coupled_channel_f32_200_steps():
    """Small channel suspension with red cells and platelets, FP32 storage
    and arithmetic: velocity relative L2 <= 1e-5 after 200 steps."""
    cfg = I.channel(nx=32, ny=32, nz=64, ncell=10, seed=3, platelet_ratio=0.5, pack_iter=100, exact_iter=0)
    got, exp = run_both(cfg, 'f32', 200)
    assert_close(got['u'], exp['u'], F32_TOL)
    assert_close(got['X'], exp['X'], F32_TOL)


def test_mass_conservation_f64():
    cfg = small_cell_shear(n=20, steps=40)
    sim = hemo.Simulation.from_config(cfg, 'f64')
    m0 = sim.populations().sum()
    sim.step(41)
    m1 = sim.populations().sum()
    sim.close()
    assert abs(m1 - m0) / m0 < 1e-13


def test_numeric_status_is_reported():
    """A body force that accelerates the fluid past |u| = 0.3 raises the
    device status; the host reads HEMO_ERR_NUMERIC (no trap)."""
    sim = hemo.Simulation(8, 8, 8, 1.0, 'f32', (1, 1, 1), None, None, [0.05, 0, 0])
    sim.step(10)
    with pytest.raises(hemo.HemoError) as e:
        sim.sync()
    assert e.value.code == hemo.HEMO_ERR_NUMERIC
    with pytest.raises(hemo.HemoError):
        sim.step(1)
    sim.close()


def test_domain_status_is_reported():
    """A vertex beyond a non-periodic edge raises HEMO_ERR_DOMAIN."""
    cfg = small_cell_shear(n=16, steps=1)
    cfg.periodic = (1, 0, 0)
    cfg.mask = None
    cfg.centers = np.array([[8.0, 1.0, 8.0]])
    sim = hemo.Simulation.from_config(cfg, 'f64')
    sim.step(1)
    with pytest.raises(hemo.HemoError) as e:
        sim.sync()
    assert e.value.code == hemo.HEMO_ERR_DOMAIN
    sim.close()


def test_state_errors():
    sim = hemo.Simulation(8, 8, 8, 1.0, 'f32')
    sim.step(1)
    with pytest.raises(hemo.HemoError) as e:
        sim.set_velocity(None)
    assert e.value.code == hemo.HEMO_ERR_STATE
    sim.close()
