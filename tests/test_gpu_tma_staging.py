"""Staging of the FP32 interpolation's lattice neighbourhood: one tensor copy
per bin (the default where nx is a multiple of 4 and the neighbourhood does
not wrap around a periodic edge) against node-by-node copies
(HEMO_OPT_NODE_STAGING).  The staged values, and so every result, are the
same bits.

* A suspension in a channel (periodic x: the bins at the x edges wrap and
  take the node-by-node path, the others the tensor copy), FP32 and BF16
  storage, both integrators.
* A cell next to the walls of a box that is periodic along no axis (the
  tensor copy reads zeros beyond the lattice, as the node-by-node path
  writes them), and one across the periodic edges of a periodic box.
"""
import numpy as np
import pytest

from paper_2305_02752_gb300 import hemo
from paper_2305_02752_gb300 import inputs as I
from tests.helpers import small_cell_shear

pytestmark = pytest.mark.gpu

NS = hemo.HEMO_OPT_NODE_STAGING


def _run(cfg, prec, steps, options, setup=None):
    sim = hemo.Simulation.from_config(cfg, prec, options=options)
    if setup is not None:
        setup(sim)
    sim.step(steps)
    out = sim.get_fields(hemo.HEMO_U | hemo.HEMO_VERTS | hemo.HEMO_FORCES)
    sim.close()
    return out


def _same(a, b):
    for k in a:
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize('integrator', ['euler', 'ab2'])
@pytest.mark.parametrize('prec', ['f32', 'bf16'])
def test_channel_tensor_copy_same_bits(prec, integrator):
    cfg = I.channel(nx=32, ny=32, nz=64, ncell=6, seed=3, steps=12, pack_iter=30, exact_iter=20)

    def setup(s):
        s.set_time_scales(1 if integrator == 'euler' else 2, integrator)
    _same(_run(cfg, prec, 12, 0, setup), _run(cfg, prec, 12, NS, setup))


def test_non_periodic_box_edges():
    cfg = small_cell_shear(n=24, steps=6, seed=4, center=[4.6, 19.2, 4.9])
    cfg.periodic = (0, 0, 0)
    _same(_run(cfg, 'f32', 6, 0), _run(cfg, 'f32', 6, NS))


def test_periodic_edges():
    cfg = small_cell_shear(n=24, steps=6, seed=6, center=[0.3, 23.6, 11.5])
    _same(_run(cfg, 'f32', 6, 0), _run(cfg, 'f32', 6, NS))
