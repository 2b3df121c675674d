"""The lattice kernels' 64-bit index variants (HEMO_OPT_WIDE_INDEX), which
by default run only on lattices of more than about 226 M nodes, against the
32-bit variants on small ones: the same bits.

* Every storage type (FP64, FP32, FP16, BF16) with cells and moving walls,
  after even and odd step counts (both AA layouts): populations, density,
  velocity, vertices.
* The 16-bit two-nodes-per-thread kernels (both passes), the staged
  collision, and the internal viscosity's per-node relaxation rate.
"""
import numpy as np
import pytest

from paper_2305_02752_gb300 import hemo
from paper_2305_02752_gb300 import inputs as I
from tests.helpers import small_cell_shear

pytestmark = pytest.mark.gpu

W = hemo.HEMO_OPT_WIDE_INDEX


def _run(cfg, prec, steps, options, setup=None):
    sim = hemo.Simulation.from_config(cfg, prec, options=options)
    if setup is not None:
        setup(sim)
    sim.step(steps)
    out = sim.get_fields(hemo.HEMO_RHO | hemo.HEMO_U | hemo.HEMO_VERTS)
    out['f'] = sim.populations()
    sim.close()
    return out


def _same(a, b):
    for k in a:
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize('steps', [5, 6])
@pytest.mark.parametrize('prec', ['f64', 'f32', 'f16', 'bf16'])
def test_wide_index_same_bits(prec, steps):
    cfg = small_cell_shear(n=24, steps=steps, seed=11)
    _same(_run(cfg, prec, steps, 0), _run(cfg, prec, steps, W))


@pytest.mark.parametrize('opt', [hemo.HEMO_OPT_PAIR_COLLISION, hemo.HEMO_OPT_STAGED_COLLISION])
def test_wide_index_16bit_variants(opt):
    cfg = I.channel(nx=32, ny=32, nz=64, ncell=4, seed=7, steps=9, pack_iter=20, exact_iter=10)
    _same(_run(cfg, 'bf16', 9, opt), _run(cfg, 'bf16', 9, opt | W))


@pytest.mark.parametrize('prec', ['f64', 'f32'])
def test_wide_index_internal_viscosity(prec):
    cfg = I.channel(nx=32, ny=32, nz=64, ncell=4, seed=8, steps=7, pack_iter=20, exact_iter=10)

    def visc(s):
        s.set_viscosity_ratio(5.0)
    _same(_run(cfg, prec, 7, 0, visc), _run(cfg, prec, 7, W, visc))
