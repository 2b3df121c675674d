"""The allocation-free binning entry point against the simulation's own.

hemo_bin_vertices_noalloc serves callers that cannot let a library allocate
device memory (inside another framework's memory budget, in latency-critical
loops, or holding positions in their own buffers without a simulation).  Its
scratch is a fixed array in the library's device image that every call
reuses, so this test makes two calls in a row, with different positions, and
compares each against hemo_get_bins bit for bit (the tolerance of every
integer comparison here).  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2305_02752_gb300 import hemo
from paper_2305_02752_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_noalloc_bins_match_simulation_bins_twice():
    import torch
    cfg = I.channel(nx=40, ny=32, nz=48, ncell=6, seed=11, platelet_ratio=0.5, pack_iter=50, exact_iter=0)
    sim = hemo.Simulation.from_config(cfg, 'f64')
    _, nv, _, nbins = sim.sizes()
    key = torch.empty(nv, dtype=torch.int32, device='cuda')
    perm = torch.empty(nv, dtype=torch.int32, device='cuda')
    start = torch.empty(nbins + 1, dtype=torch.int32, device='cuda')
    rng = np.random.default_rng(4)
    for call in range(2):
        X = I.cell_vertices(cfg)
        X[:, 0] += rng.normal(size=nv) * 25
        X[:, 2] += rng.normal(size=nv) * 25
        X[call::7] = np.floor(X[call::7])        # positions exactly on lattice planes
        sim.set_vertices(X)
        Xg = sim.get_fields(hemo.HEMO_VERTS)['X']  # the exact FP64 positions the simulation bins
        k_ref, p_ref, s_ref = sim.bins()
        verts = torch.from_numpy(Xg).cuda()
        hemo.bin_vertices_noalloc(verts, (cfg.nx, cfg.ny, cfg.nz), cfg.periodic, key, perm, start)
        torch.cuda.synchronize()
        assert np.array_equal(key.cpu().numpy(), k_ref), call
        assert np.array_equal(perm.cpu().numpy(), p_ref), call
        assert np.array_equal(start.cpu().numpy(), s_ref), call
    sim.close()


def _small_sphere_cells(nx, ny, nz, per, centers):
    v, t = I.icosphere(1)
    mt = I.MeshType('s', v * 1.5, t, 1.0, 1.0, 1.0, 1.0, 1e-7, 0.015, 3.0)
    sim = hemo.Simulation(nx, ny, nz, 1.0, 'f32', per)
    sim.add_cells(mt, np.asarray(centers, float), np.repeat(np.eye(3)[None], len(centers), 0))
    return sim


def _noalloc_bins(X, dims, per, nbins):
    import torch
    nv = len(X)
    key = torch.full((nv,), -7, dtype=torch.int32, device='cuda')
    perm = torch.full((nv,), -7, dtype=torch.int32, device='cuda')
    start = torch.full((nbins + 1,), -7, dtype=torch.int32, device='cuda')
    hemo.bin_vertices_noalloc(torch.from_numpy(np.ascontiguousarray(X, np.float64).reshape(nv, 3)).cuda(),
                              dims, per, key, perm, start)
    torch.cuda.synchronize()
    return key.cpu().numpy(), perm.cpu().numpy(), start.cpu().numpy()


def test_noalloc_odd_non_periodic_lattice():
    """A 13 x 21 x 9 lattice without periodic axes (2 x 3 x 2 blocks, none
    of the sizes a multiple of 8), FP32 simulation: vertices inside, on
    lattice planes, and at the last node of each axis, against hemo_get_bins
    bit for bit; then vertices beyond the edges, which both clamp to the edge
    block (the simulation also reports the domain error)."""
    dims, per = (13, 21, 9), (0, 0, 0)
    centers = [[3.0, 4.0, 3.0], [9.5, 17.2, 5.5], [6.0, 10.0, 4.5], [10.2, 3.3, 6.1]]
    sim = _small_sphere_cells(*dims, per, centers)
    _, nv, _, nbins = sim.sizes()
    assert nbins == 2 * 3 * 2
    X = sim.get_fields(hemo.HEMO_VERTS)['X']
    X[::5] = np.floor(X[::5])
    X[1] = [12.0, 20.0, 8.0]
    X[2] = [7.999999999, 15.9999999, 1.0]  # (not 0: the FP32 offset could round below the edge)
    sim.set_vertices(X)
    Xg = sim.get_fields(hemo.HEMO_VERTS)['X']
    k_ref, p_ref, s_ref = sim.bins()
    sim.close()
    k, p, s = _noalloc_bins(Xg, dims, per, nbins)
    assert np.array_equal(k, k_ref) and np.array_equal(p, p_ref) and np.array_equal(s, s_ref)
    # beyond the edges: the simulation flags the domain error but still bins
    sim = _small_sphere_cells(*dims, per, centers)
    Xo = Xg.copy()
    Xo[0] = [-3.5, 25.0, 9.5]
    Xo[3] = [14.0, -0.5, -2.0]
    sim.set_vertices(Xo)
    Xg2 = sim.get_fields(hemo.HEMO_VERTS)['X']
    _, nv2, _, _ = sim.sizes()
    key = np.zeros(nv2, np.int32)
    perm = np.zeros(nv2, np.int32)
    start = np.zeros(nbins + 1, np.int32)
    with pytest.raises(hemo.HemoError) as e:
        hemo.check(hemo.lib().hemo_get_bins(sim.handle, key.ctypes.data, perm.ctypes.data, start.ctypes.data))
    assert e.value.code == hemo.HEMO_ERR_DOMAIN
    sim.close()
    k, p, s = _noalloc_bins(Xg2, dims, per, nbins)
    assert np.array_equal(k, key) and np.array_equal(p, perm) and np.array_equal(s, start)
    assert k[0] == 0 + 2 * (2 + 3 * 1) and k[3] == 1


def test_noalloc_without_vertices():
    """nv = 0: only the clearing and the scan run; every block starts at 0,
    as in a simulation without cells."""
    import torch
    dims, per = (40, 24, 17), (1, 0, 1)
    sim = hemo.Simulation(*dims, 1.0, 'f32', per)
    _, nv, _, nbins = sim.sizes()
    assert nv == 0
    _, _, s_ref = sim.bins()
    sim.close()
    start = torch.full((nbins + 1,), -7, dtype=torch.int32, device='cuda')
    empty = torch.zeros(0, dtype=torch.int32, device='cuda')
    hemo.bin_vertices_noalloc(torch.zeros((0, 3), dtype=torch.float64, device='cuda'), dims, per, empty, empty, start)
    torch.cuda.synchronize()
    assert np.array_equal(start.cpu().numpy(), s_ref)
    assert not start.cpu().numpy().any()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    verts = torch.zeros((4, 3), dtype=torch.float64, device='cuda')
    out = torch.zeros(8, dtype=torch.int32, device='cuda')
    start = torch.zeros(128 ** 3 + 1, dtype=torch.int32, device='cuda')  # large enough for the binding's check
    with pytest.raises(hemo.HemoError) as e:
        hemo.bin_vertices_noalloc(verts, (1024, 1024, 1024), (1, 1, 1), out, out, start)
    assert e.value.code == hemo.HEMO_ERR_ARG
    assert 'blocks' in str(e.value)
