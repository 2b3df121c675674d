"""Full-size configurations: parity of the FP32 path with the oracle on the
64x64x256 channel with 440 red cells, the precision forms on the
128x128x512 vessel at 40 % haematocrit (velocity relative L2 against the
FP64 run after 200 steps: FP32 <= 1e-5, FP16 <= 1e-3), and invariants on the
1000x208x208 pipe with 19,600 red cells (mass conservation, finite fields,
no domain error)."""
import numpy as np
import pytest

import oracle as O
from paper_2305_02752_gb300 import hemo
from paper_2305_02752_gb300 import inputs as I
from tests.helpers import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module')
def channel_cfg():
    return I.channel()


@pytest.fixture(scope='module')
def vessel_runs():
    cfg = I.channel(nx=128, ny=128, nz=512, ncell=4460, seed=20230502, steps=200, platelet_ratio=0.1,
                    name='vessel', pack_iter=60, exact_iter=0)
    out = {}
    for prec in ('f64', 'f32', 'f16', 'bf16'):
        sim = hemo.Simulation.from_config(cfg, prec)
        sim.step(200)
        out[prec] = sim.get_fields(hemo.HEMO_U | hemo.HEMO_VERTS)
        sim.close()
    return cfg, out


def test_channel_full_size_f32_matches_oracle(channel_cfg):
    """64x64x256 channel, 440 cells (282,480 vertices), the launch
    configuration the benchmark times: 5 steps against the oracle."""
    got = {}
    sim = hemo.Simulation.from_config(channel_cfg, 'f32')
    sim.step(5)
    got = sim.get_fields()
    sim.close()
    ref = O.from_config(channel_cfg)
    ref.step(5)
    exp = ref.get()
    assert rel_l2(got['u'], exp['u']) < 1e-5
    assert rel_l2(got['X'], exp['X']) < 1e-5
    assert rel_l2(got['cellstats'][:, :5], exp['cellstats'][:, :5]) < 1e-5


@pytest.mark.parametrize('prec,tol', [('f32', 1e-5), ('f16', 1e-3)])
def test_vessel_precision_forms(vessel_runs, prec, tol):
    cfg, out = vessel_runs
    ref = out['f64']
    assert rel_l2(out[prec]['u'], ref['u']) < tol
    assert rel_l2(out[prec]['X'], ref['X']) < tol


def test_vessel_bf16_error_is_reported(vessel_runs):
    """BF16 deviations carry 8 significant bits; their velocity error after
    200 steps is measured against the FP64 run (it exceeds the 1e-3 target,
    which FP16 meets) and must stay below 1e-2."""
    cfg, out = vessel_runs
    err = rel_l2(out['bf16']['u'], out['f64']['u'])
    assert err < 1e-2


def test_pipe_full_size_invariants():
    cfg = I.pipe(pack_iter=3)  # placement relaxation shortened: overlaps do not affect the invariants
    sim = hemo.Simulation.from_config(cfg, 'f32')
    m0 = sim.get_fields(hemo.HEMO_RHO)['rho'].astype(np.float64).sum()
    sim.step(10)
    f = sim.get_fields(hemo.HEMO_RHO | hemo.HEMO_U | hemo.HEMO_VERTS)
    sim.sync()
    sim.close()
    assert np.isfinite(f['u']).all() and np.isfinite(f['X']).all()
    m1 = f['rho'].astype(np.float64).sum()
    assert abs(m1 - m0) / m0 < 1e-6
    assert cfg.n_vertices == 19600 * 642
