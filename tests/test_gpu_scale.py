"""Full-size configurations against the oracle, in the launch configurations
the benchmark times.

* Channel 64x64x256 with 440 red cells (282,480 vertices), FP32: 200 steps
  against the oracle (velocity relative L2 <= 1e-5).
* Vessel 128x128x512 at 40 % haematocrit (4460 red cells + 446 platelets):
  the FP64 GPU run against the oracle after 20 steps (<= 1e-12), which
  anchors the 200-step comparison of the storage forms against that FP64 run
  (FP32 <= 1e-5, FP16 and BF16 <= 1e-3).
* Pipe 1000x208x208 with 19,600 red cells (12.6 M vertices): FP32 and FP16
  against the oracle after 3 steps, and mass conservation.

The oracle runs on all host cores (its results do not depend on the thread
count).  Every comparison checks the relative L2 error and the largest
per-element error (tests.helpers.assert_close).
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_2305_02752_gb300 import hemo
from paper_2305_02752_gb300 import inputs as I
from tests.helpers import assert_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module', autouse=True)
def oracle_threads():
    O.set_threads(os.cpu_count() or 1)
    yield
    O.set_threads(1)


def _gpu(cfg, prec, steps, what=hemo.HEMO_RHO | hemo.HEMO_U | hemo.HEMO_VERTS | hemo.HEMO_CELLSTATS):
    sim = hemo.Simulation.from_config(cfg, prec)
    sim.step(steps)
    out = sim.get_fields(what)
    sim.close()
    return out


def _oracle(cfg, steps):
    ref = O.from_config(cfg)
    ref.step(steps)
    out = ref.get()
    ref.close()
    return out


def test_channel_full_size_f32_200_steps_matches_oracle():
    """64x64x256 channel, 440 cells, FP32, 200 steps (the step count at which
    the FP32 tolerance is stated)."""
    cfg = I.channel()
    got = _gpu(cfg, 'f32', 200)
    exp = _oracle(cfg, 200)
    assert_close(got['u'], exp['u'], 1e-5, 'u')
    assert_close(got['X'], exp['X'], 1e-5, 'X')
    assert_close(got['cellstats'][:, :5], exp['cellstats'][:, :5], 1e-5, 'cellstats')


@pytest.fixture(scope='module')
def vessel_cfg():
    return I.channel(nx=128, ny=128, nz=512, ncell=4460, seed=20230502, steps=200, platelet_ratio=0.1,
                     name='vessel', pack_iter=60, exact_iter=0)


def test_vessel_f64_matches_oracle(vessel_cfg):
    """The FP64 path on the 40 % haematocrit vessel (red cells and
    platelets) against the oracle after 20 steps."""
    got = _gpu(vessel_cfg, 'f64', 20)
    exp = _oracle(vessel_cfg, 20)
    assert_close(got['u'], exp['u'], 1e-12, 'u')
    assert_close(got['rho'], exp['rho'], 1e-12, 'rho')
    assert_close(got['X'], exp['X'], 1e-12, 'X')
    assert_close(got['cellstats'], exp['cellstats'], 1e-12, 'cellstats')


@pytest.fixture(scope='module')
def vessel_runs(vessel_cfg):
    out = {}
    for prec in ('f64', 'f32', 'f16', 'bf16'):
        out[prec] = _gpu(vessel_cfg, prec, 200, hemo.HEMO_U | hemo.HEMO_VERTS)
    return out


@pytest.mark.parametrize('prec,tol', [('f32', 1e-5), ('f16', 1e-3), ('bf16', 1e-3)])
def test_vessel_precision_forms(vessel_runs, prec, tol):
    """Storage forms after 200 steps against the FP64 run of the same seed
    (anchored to the oracle by test_vessel_f64_matches_oracle)."""
    ref = vessel_runs['f64']
    assert_close(vessel_runs[prec]['u'], ref['u'], tol, 'u')
    assert_close(vessel_runs[prec]['X'], ref['X'], tol, 'X')


@pytest.fixture(scope='module')
def pipe_cfg():
    return I.pipe()


@pytest.fixture(scope='module')
def pipe_oracle(pipe_cfg):
    return _oracle(pipe_cfg, 3)


@pytest.mark.parametrize('prec,tol', [('f32', 1e-5), ('f16', 1e-3)])
def test_pipe_full_size_matches_oracle(pipe_cfg, pipe_oracle, prec, tol):
    """1000x208x208 pipe, 19,600 red cells (12.6 M vertices), the benchmark's
    workload: 3 steps against the oracle; the density is conserved to the
    storage precision."""
    sim = hemo.Simulation.from_config(pipe_cfg, prec)
    m0 = sim.get_fields(hemo.HEMO_RHO)['rho'].astype(np.float64).sum()
    sim.step(3)
    got = sim.get_fields(hemo.HEMO_RHO | hemo.HEMO_U | hemo.HEMO_VERTS)
    sim.close()
    exp = pipe_oracle
    assert pipe_cfg.n_vertices == 19600 * 642
    assert_close(got['u'], exp['u'], tol, 'u')
    assert_close(got['X'], exp['X'], tol, 'X')
    m1 = got['rho'].astype(np.float64).sum()
    assert abs(m1 - m0) / m0 < (1e-6 if prec == 'f32' else 1e-4)
