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


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    verts = torch.zeros((4, 3), dtype=torch.float64, device='cuda')
    out = torch.zeros(8, dtype=torch.int32, device='cuda')
    with pytest.raises(hemo.HemoError) as e:
        hemo.bin_vertices_noalloc(verts, (1024, 1024, 1024), (1, 1, 1), out, out, out)
    assert e.value.code == hemo.HEMO_ERR_ARG
    assert 'blocks' in str(e.value)
