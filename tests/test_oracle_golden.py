"""The oracle still reproduces its committed regression snapshot."""
import os

import numpy as np

from tests.golden.make_golden import compute

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_matches_snapshot():
    ref = {}
    with open(os.path.join(HERE, 'golden', 'oracle_shear16.txt')) as f:
        for line in f:
            if line.startswith('#'):
                continue
            k, v = line.split()
            ref[k] = float(v)
    got = dict(compute())
    assert set(got) == set(ref)
    for k, v in got.items():
        assert abs(v - ref[k]) <= 1e-12 * max(1.0, abs(ref[k])), k
