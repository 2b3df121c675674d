"""Write tests/golden/oracle_shear16.txt: a regression snapshot of the CPU
oracle on a tiny sheared cell (16^3 box, plates at z = 0 and 15 moving at
-/+0.01, one 162-vertex biconcave cell of diameter 8, 20 steps).

The paper prints no worked example for the coupled step, so this file is not
a pin: it records the oracle's own output so that an unintended change of the
oracle's arithmetic is noticed.  It calls only `oracle` and the seeded input
generators.  Run:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2305_02752_gb300 import inputs as I  # noqa: E402


def golden_config():
    cfg = I.shear_cell(n=16, ncell=1, seed=42, steps=20)
    v, t = I.icosphere(2)
    cfg.meshes[0].rest = I.evans_fung(v, 8.0)
    cfg.meshes[0].tri = t
    cfg.centers = np.array([[8.0, 8.0, 7.5]])
    return cfg


def compute():
    cfg = golden_config()
    s = O.from_config(cfg)
    s.step(cfg.steps)
    out = s.get()
    rows = []
    rows.append(('mass', out['rho'].sum()))
    for z, y, x in ((1, 1, 1), (7, 8, 3), (14, 2, 9), (8, 8, 8)):
        for d in range(3):
            rows.append((f'u[{z},{y},{x}][{d}]', out['u'][z, y, x, d]))
    for v in (0, 17, 161):
        for d in range(3):
            rows.append((f'X[{v}][{d}]', out['X'][v, d]))
            rows.append((f'Fv[{v}][{d}]', out['Fv'][v, d]))
    for k, name in enumerate(('cx', 'cy', 'cz', 'area', 'volume', 'DI')):
        rows.append((name, out['cellstats'][0, k]))
    return rows


if __name__ == '__main__':
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), 'oracle_shear16.txt')
    with open(path, 'w') as f:
        f.write('# oracle regression snapshot written by tests/golden/make_golden.py (not a paper value)\n')
        for k, v in compute():
            f.write(f'{k} {v:.17e}\n')
    print('wrote', path)
