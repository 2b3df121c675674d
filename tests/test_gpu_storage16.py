"""16-bit population storage: the two-nodes-per-thread kernels against the
one-node kernels, and the per-row reference equilibrium.

* Two-node kernels (by default the velocity pass for 16-bit storage with nx
  even; the collision too with HEMO_OPT_PAIR_COLLISION) and the per-node
  kernels (HEMO_OPT_NODE_COLLISION) give the same bits:
  populations, density and velocity after even and odd step counts, with
  walls on y or z, fully periodic boxes whose rows are not a multiple of the
  64-node warp chunk (ragged last chunks, a row of two nodes), and cells.
* The stored values carry the departure from the row's reference: after
  hemo_set_velocity with a profile of rows, the decoded populations equal
  the oracle's equilibrium to within the 16-bit rounding of f - w - K (K
  the oracle's storage reference of the row's mean x-velocity), far below
  the rounding of f - w itself.
"""
import numpy as np
import pytest

import oracle as O
from paper_2305_02752_gb300 import hemo
from paper_2305_02752_gb300 import inputs as I
from tests.helpers import direction_map, small_cell_shear

pytestmark = pytest.mark.gpu


def _box(nx, ny, nz, seed, walls_axis=None, profile=True):
    rng = np.random.default_rng(seed)
    mask = None if walls_axis is None else I.plate_mask(nx, ny, nz, axis=walls_axis)
    per = [1, 1, 1]
    if walls_axis is not None:
        per[walls_axis] = 0
    u0 = 0.004 * rng.standard_normal((nz, ny, nx, 3))
    if profile:  # a row profile along x, varying with y and z
        y = np.arange(ny)[None, :, None]
        z = np.arange(nz)[:, None, None]
        u0[..., 0] += 0.02 * np.sin(0.3 * y + 0.2 * z)
    if mask is not None:
        u0[mask != 0] = 0.0
    g = np.array([2e-6, -1e-6, 5e-7])
    return dict(nx=nx, ny=ny, nz=nz, per=tuple(per), mask=mask, u0=u0, g=g)


def _run(case, prec, steps, options, cells=None):
    if cells is not None:
        sim = hemo.Simulation.from_config(cells, prec, options=options)
    else:
        sim = hemo.Simulation(case['nx'], case['ny'], case['nz'], 0.8, prec, case['per'], case['mask'], None,
                              case['g'], options=options)
        sim.set_velocity(case['u0'])
    sim.step(steps)
    out = sim.get_fields(hemo.HEMO_RHO | hemo.HEMO_U | hemo.HEMO_VERTS)
    out['f'] = sim.populations()
    sim.close()
    return out


BOXES = {
    'walls_y': lambda: _box(64, 20, 12, 1, walls_axis=1),
    'walls_z': lambda: _box(70, 9, 14, 2, walls_axis=2),
    'periodic_ragged': lambda: _box(100, 10, 6, 3),      # chunks of 64 + 36 nodes
    'periodic_short_rows': lambda: _box(2, 12, 10, 4),   # one lane per row
    'periodic_66': lambda: _box(66, 7, 5, 5),            # a last chunk of one lane
}


@pytest.mark.parametrize('steps', [1, 2, 7, 8])
@pytest.mark.parametrize('prec', ['f16', 'bf16'])
@pytest.mark.parametrize('case', sorted(BOXES))
def test_pair_kernels_match_node_kernels(case, prec, steps):
    """Default (pair velocity pass), both passes by pairs, both per node."""
    c = BOXES[case]()
    a = _run(c, prec, steps, 0)
    b = _run(c, prec, steps, hemo.HEMO_OPT_NODE_COLLISION)
    p = _run(c, prec, steps, hemo.HEMO_OPT_PAIR_COLLISION)
    for k in ('f', 'rho', 'u'):
        assert np.array_equal(a[k], b[k]), k
        assert np.array_equal(p[k], b[k]), k


@pytest.mark.parametrize('prec', ['f16', 'bf16'])
def test_pair_kernels_with_cells(prec):
    cfg = small_cell_shear(n=24, steps=9, seed=5)
    a = _run(None, prec, 9, 0, cells=cfg)
    b = _run(None, prec, 9, hemo.HEMO_OPT_NODE_COLLISION, cells=cfg)
    p = _run(None, prec, 9, hemo.HEMO_OPT_PAIR_COLLISION, cells=cfg)
    for k in ('f', 'u', 'X'):
        assert np.array_equal(a[k], b[k]), k
        assert np.array_equal(p[k], b[k]), k


def test_odd_row_length_uses_node_kernels():
    """nx odd: no pair words; both options take the per-node kernels."""
    c = _box(33, 8, 6, 6)
    a = _run(c, 'bf16', 3, 0)
    b = _run(c, 'bf16', 3, hemo.HEMO_OPT_NODE_COLLISION)
    assert np.array_equal(a['f'], b['f'])


@pytest.mark.parametrize('prec,eps,floor', [('f16', 2.0 ** -11, 2.0 ** -25 + 4e-9), ('bf16', 2.0 ** -8, 4e-9)])
def test_reference_reconstruction(prec, eps, floor):
    """Rows of a pure x-profile U(y, z): each population decodes to the
    oracle's equilibrium of (U, 0, 0) within the 16-bit rounding (half an
    ulp: 2^-11 FP16, 2^-8 BF16, relative) of f - w - K(U), plus an absolute
    floor for the FP32 rounding of the reference and, for FP16, half its
    subnormal spacing.  On the directions with c_x != 0, where K carries the
    flow, that error is below 5 % of the rounding f - w itself would get."""
    nx, ny, nz = 16, 12, 10
    y = np.arange(ny)[None, :, None]
    z = np.arange(nz)[:, None, None]
    U = 0.02 * np.sin(0.4 * y + 0.25 * z) + 0.005
    u0 = np.zeros((nz, ny, nx, 3))
    u0[..., 0] = U
    sim = hemo.Simulation(nx, ny, nz, 1.0, prec, (1, 1, 1))
    sim.set_velocity(u0)
    f = sim.populations()  # library order
    sim.close()
    dm = direction_map()   # oracle index of each library direction
    cg, _ = hemo.velocity_set()
    xdir = cg[:, 0] != 0
    _, w, _ = O.d3q19()
    worst_ratio = 0.0
    for zz in range(nz):
        for yy in range(ny):
            Ur = float(U[zz, yy, 0])
            feq = O.equilibrium(1.0, [Ur, 0.0, 0.0])[dm]
            K = O.storage_reference(Ur)[dm]
            err = np.abs(f[zz, yy, :, :] - feq[None, :])
            bound = eps * np.abs(feq - w[dm] - K) + floor
            assert (err <= bound[None, :]).all(), (zz, yy, err.max(), bound)
            plain = eps * np.abs(feq - w[dm]) + floor
            worst_ratio = max(worst_ratio, (err / plain[None, :])[:, xdir].max())
    assert worst_ratio < 0.05
