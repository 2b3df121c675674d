"""Pin of the oracle's whole coupled step: equivariance under the symmetries
of the cubic lattice and under integer translations of a periodic box.

D3Q19 (Sec. 2.2), the BGK collision with Guo forcing, halfway bounce-back,
the 4-point Peskin kernel (a product of even 1-D kernels, Sec. 2.3) and the
membrane energies (functions of lengths, angles, areas and volumes) are all
unchanged by the 48 axis permutations and reflections that map the lattice
onto itself.  So one step commutes with such a map T: running the
transformed configuration gives the transformed result.  The velocity turns
with T's matrix, densities move with the nodes, vertex positions map by T
and forces turn with it; a reflection also mirrors each rest shape, which
reverses its triangles' winding so that they stay counter-clockwise seen
from outside.  A wrong index, a dropped or sign-flipped term, or a swapped
pair of axes anywhere in the step breaks this for some T, while it holds
to rounding (the transformed run sums the same terms in another order).
"""
import dataclasses

import numpy as np
import pytest

import oracle as O
from paper_2305_02752_gb300 import inputs as I
from tests.helpers import forces_close, rel_l2, small_cell_shear

MIRROR = np.diag([1.0, 1.0, -1.0])  # fixed reflection used to keep rotations proper


def _map(perm, sign, n):
    """T(p) = A p + b with (A p)_k = sign_k p_perm[k]; b puts the image of
    the lattice {0..n-1}^3 back on itself."""
    A = np.zeros((3, 3))
    for k in range(3):
        A[k, perm[k]] = sign[k]
    b = np.where(np.array(sign) < 0, n - 1.0, 0.0)
    return A, b


def _nodes_back(A, b, n):
    """For every node p' of the transformed grid ([z, y, x] order) the index
    arrays of its preimage p = A^T (p' - b)."""
    g = np.arange(n)
    z, y, x = np.meshgrid(g, g, g, indexing='ij')
    pp = np.stack([x, y, z], -1).astype(float)
    p = np.rint((pp - b) @ A).astype(int)  # (p' - b) A = A^T (p' - b) row-wise
    return p[..., 2], p[..., 1], p[..., 0]


def _field(a, A, b, n, vector):
    z, y, x = _nodes_back(A, b, n)
    out = a[z, y, x]
    return out @ A.T if vector else out


def _transform(cfg, A, b):
    n = cfg.nx
    assert cfg.nx == cfg.ny == cfg.nz
    perm = np.abs(A).argmax(axis=1)
    proper = np.linalg.det(A) > 0
    meshes = []
    for mt in cfg.meshes:
        if proper:
            meshes.append(mt)
        else:
            meshes.append(dataclasses.replace(mt, rest=mt.rest @ MIRROR.T, tri=mt.tri[:, [0, 2, 1]].copy()))
    rots = np.einsum('ij,njk->nik', A, cfg.rotations)
    if not proper:
        rots = np.einsum('nij,jk->nik', rots, MIRROR)
    return dataclasses.replace(
        cfg,
        periodic=tuple(int(cfg.periodic[perm[k]]) for k in range(3)),
        mask=None if cfg.mask is None else _field(cfg.mask, A, b, n, False),
        wall_velocity=cfg.wall_velocity @ A.T,
        body_force=A @ cfg.body_force,
        init_velocity=None if cfg.init_velocity is None else _field(cfg.init_velocity, A, b, n, True),
        meshes=meshes,
        centers=cfg.centers @ A.T + b,
        rotations=rots,
    )


def _run(cfg, steps):
    s = O.from_config(cfg)
    s.step(steps)
    out = s.get()
    s.close()
    return out


def _periodic_close(got, exp, n, periodic, tol):
    d = got - exp
    for k in range(3):
        if periodic[k]:
            d[:, k] -= n * np.round(d[:, k] / n)
    return np.linalg.norm(d) / np.linalg.norm(exp) < tol


TRANSFORMS = {
    'reflect_x': ((0, 1, 2), (-1, 1, 1)),
    'reflect_z': ((0, 1, 2), (1, 1, -1)),
    'rotate_z_90': ((1, 0, 2), (-1, 1, 1)),
    'cycle_xyz': ((2, 0, 1), (1, 1, 1)),
    'inversion': ((0, 1, 2), (-1, -1, -1)),
    'rotoreflection': ((2, 0, 1), (-1, 1, -1)),
}


def _periodic_case():
    """Fully periodic cube: a red cell off-centre across two periodic edges,
    a random velocity field and a body force along no axis."""
    n = 20
    cfg = small_cell_shear(n=n, seed=3, steps=10, center=[18.6, 1.3, 9.7])
    rng = np.random.default_rng(12)
    cfg.rotations = I.random_rotation(rng)[None]
    return dataclasses.replace(cfg, mask=None, periodic=(1, 1, 1), wall_velocity=np.zeros((2, 3)),
                               body_force=np.array([1e-5, -2e-6, 3e-6]),
                               init_velocity=0.004 * rng.normal(size=(n, n, n, 3)))


def _walls_case():
    """Moving plates at z = 0 and z = n - 1 (ids 2 and 3), a tilted cell."""
    cfg = small_cell_shear(n=20, seed=4, steps=10, center=[7.4, 11.9, 9.2])
    rng = np.random.default_rng(13)
    cfg.rotations = I.random_rotation(rng)[None]
    u0 = 0.003 * rng.normal(size=(20, 20, 20, 3))
    u0[cfg.mask != 0] = 0.0
    return dataclasses.replace(cfg, wall_velocity=np.array([[-0.01, 0.004, 0.0], [0.01, 0.0, 0.0]]),
                               init_velocity=u0)


def _check(cfg, name, steps):
    A, b = _map(*TRANSFORMS[name], cfg.nx)
    ref = _run(cfg, steps)
    got = _run(_transform(cfg, A, b), steps)
    n = cfg.nx
    assert rel_l2(got['u'], _field(ref['u'], A, b, n, True)) < 1e-12
    assert rel_l2(got['rho'], _field(ref['rho'], A, b, n, False)) < 1e-14
    tper = tuple(int(cfg.periodic[k]) for k in np.abs(A).argmax(axis=1))
    assert _periodic_close(got['X'], ref['X'] @ A.T + b, n, tper, 1e-13)
    assert forces_close(got['Fv'], ref['Fv'] @ A.T, cfg)
    # area, volume and deformation index are invariant
    np.testing.assert_allclose(got['cellstats'][:, 3:6], ref['cellstats'][:, 3:6], rtol=1e-12)
    return ref


@pytest.mark.parametrize('name', sorted(TRANSFORMS))
def test_periodic_box(name):
    ref = _check(_periodic_case(), name, 10)
    assert np.abs(ref['Fv']).max() > 0  # the cell is deformed: forces take part


@pytest.mark.parametrize('name', ['reflect_x', 'reflect_z', 'rotate_z_90', 'inversion'])
def test_moving_walls(name):
    _check(_walls_case(), name, 10)


@pytest.mark.parametrize('name', ['reflect_x', 'cycle_xyz'])
def test_large_deformation_terms(name):
    cfg = _periodic_case()
    cfg.meshes = [dataclasses.replace(mt, k_local=0.05, theta_m=0.5) for mt in cfg.meshes]
    _check(cfg, name, 6)


def test_a_planted_axis_swap_is_caught():
    """The pin is not vacuous: a configuration transformed with the wrong
    field map (velocities not turned with T) gives a different run."""
    cfg = _periodic_case()
    A, b = _map(*TRANSFORMS['rotate_z_90'], cfg.nx)
    bad = _transform(cfg, A, b)
    bad.init_velocity = _field(cfg.init_velocity, A, b, cfg.nx, False)  # positions moved, vectors not turned
    ref = _run(cfg, 4)
    got = _run(bad, 4)
    assert rel_l2(got['u'], _field(ref['u'], A, b, cfg.nx, True)) > 1e-3


def test_periodic_translation():
    """An integer translation of everything on the periodic box translates
    the result (the wrap of stencils and streaming across every edge)."""
    cfg = _periodic_case()
    n, shift = cfg.nx, np.array([7, -5, 13])
    moved = dataclasses.replace(cfg, centers=cfg.centers + shift,
                                init_velocity=np.roll(cfg.init_velocity, shift=tuple(shift[::-1]), axis=(0, 1, 2)))
    ref, got = _run(cfg, 8), _run(moved, 8)
    roll = lambda a: np.roll(a, shift=tuple(shift[::-1]), axis=(0, 1, 2))  # noqa: E731
    assert rel_l2(got['u'], roll(ref['u'])) < 1e-13
    assert rel_l2(got['rho'], roll(ref['rho'])) < 1e-15
    assert _periodic_close(got['X'], ref['X'] + shift, n, (1, 1, 1), 1e-13)
    assert forces_close(got['Fv'], ref['Fv'], cfg)


# Lees-Edwards along z (Sec. 2.5): a reflection of x or of z turns the image
# above the box into one displaced and moving the other way, i.e. the same
# boundary with -U; reflecting y, or both x and z, keeps U.
LE_TRANSFORMS = {
    'reflect_x': (((0, 1, 2), (-1, 1, 1)), -1.0),
    'reflect_y': (((0, 1, 2), (1, -1, 1)), 1.0),
    'reflect_z': (((0, 1, 2), (1, 1, -1)), -1.0),
    'rotate_y_180': (((0, 1, 2), (-1, 1, -1)), 1.0),
}


@pytest.mark.parametrize('name', sorted(LE_TRANSFORMS))
def test_lees_edwards(name):
    """A red cell across the bottom plane in a sheared periodic box."""
    cfg = dataclasses.replace(_periodic_case(), centers=np.array([[9.3, 10.6, 1.2]]))
    (perm, sign), flip = LE_TRANSFORMS[name]
    A, b = _map(perm, sign, cfg.nx)
    U = 0.03

    def run(c, u_le):
        s = O.from_config(c)
        s.set_lees_edwards(u_le)
        s.step(9)
        out = s.get()
        s.close()
        return out

    ref, got = run(cfg, U), run(_transform(cfg, A, b), flip * U)
    n = cfg.nx
    assert rel_l2(got['u'], _field(ref['u'], A, b, n, True)) < 1e-12
    assert rel_l2(got['rho'], _field(ref['rho'], A, b, n, False)) < 1e-14
    # positions: the images differ by the plane's displacement, so compare x
    # modulo the box only where no plane was crossed (this cell's centroid
    # stays inside the box)
    assert _periodic_close(got['X'], ref['X'] @ A.T + b, n, (1, 1, 0), 1e-13)
    assert forces_close(got['Fv'], ref['Fv'] @ A.T, cfg)


@pytest.mark.parametrize('name', ['reflect_x', 'reflect_z', 'rotate_z_90', 'cycle_xyz'])
def test_internal_viscosity(name):
    """Viscosity ratio 5 inside the cell: the inside/outside indicator and
    the per-node relaxation move with the configuration (its tie rules only
    matter for nodes exactly on the membrane, which these positions avoid)."""
    cfg = _periodic_case()
    A, b = _map(*TRANSFORMS[name], cfg.nx)

    def run(c):
        s = O.from_config(c)
        s.set_viscosity_ratio(5.0)
        ins0 = s.inside().copy()
        s.step(8)
        out = s.get()
        out['inside0'] = ins0
        s.close()
        return out

    ref, got = run(cfg), run(_transform(cfg, A, b))
    n = cfg.nx
    assert ref['inside0'].sum() > 50
    assert np.array_equal(got['inside0'], _field(ref['inside0'], A, b, n, False))
    assert rel_l2(got['u'], _field(ref['u'], A, b, n, True)) < 1e-12
    assert _periodic_close(got['X'], ref['X'] @ A.T + b, n, (1, 1, 1), 1e-13)
