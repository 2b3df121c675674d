"""The bounds-checked build (libhemo_checked.so, loaded when
HEMO_BOUNDS_CHECK=1): the data-driven indices of the vertex, bin and
membrane kernels are tested on the device and a failed test is reported
through the status word.  On valid inputs no test fails, and the checked
build computes the same bits as the default one (the tests do not touch the
arithmetic): a suspension channel in FP32 and BF16 storage, a red cell in
shear in FP64 with the adaptive separation and Adams-Bashforth."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2305_02752_gb300 import hemo

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RUN = r'''
import json, sys
import numpy as np
sys.path.insert(0, {root!r})
from paper_2305_02752_gb300 import hemo
from paper_2305_02752_gb300 import inputs as I
from tests.helpers import small_cell_shear
case, prec, out = sys.argv[1], sys.argv[2], sys.argv[3]
if case == 'channel':
    cfg = I.channel(nx=32, ny=32, nz=64, ncell=6, seed=3, steps=12, pack_iter=30, exact_iter=20)
    steps, setup = 12, None
else:
    cfg = small_cell_shear(steps=16)
    steps = 16
    def setup(s):
        s.set_time_scales(5, 'ab2')
        s.set_force_tolerance(0.0023)
sim = hemo.Simulation.from_config(cfg, prec)
if setup:
    setup(sim)
sim.step(steps)
f = sim.get_fields(hemo.HEMO_U | hemo.HEMO_VERTS | hemo.HEMO_FORCES)
sim.close()
np.savez(out, lib=np.array(hemo.LIB_PATH), **f)
'''


def _run(case, prec, checked, tmp_path):
    out = str(tmp_path / f'{case}_{prec}_{int(checked)}.npz')
    env = dict(os.environ)
    env['HEMO_BOUNDS_CHECK'] = '1' if checked else '0'
    subprocess.run([sys.executable, '-c', RUN.format(root=ROOT), case, prec, out], check=True, env=env, cwd=ROOT)
    d = dict(np.load(out))
    assert str(d.pop('lib')).endswith('libhemo_checked.so' if checked else 'libhemo.so')
    return d


@pytest.mark.parametrize('case,prec', [('channel', 'f32'), ('channel', 'bf16'), ('shear', 'f64')])
def test_checked_build_same_bits(case, prec, tmp_path):
    a = _run(case, prec, False, tmp_path)
    b = _run(case, prec, True, tmp_path)  # raises (non-zero exit) if a check failed
    for k in a:
        assert np.array_equal(a[k], b[k]), k
