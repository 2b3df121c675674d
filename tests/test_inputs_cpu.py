"""The seeded input generators (shared by the CUDA path and the oracle; they
hold none of the method's arithmetic): meshes, rotations, masks, profiles,
the force-bias packer and the configurations, checked against definitions
that do not reuse their code.

Shape pins: Sec. 1 gives an undeformed red cell 6-8 um across and 2-3 um
thick; the Evans-Fung profile (2T(r) the thickness at radius r,
T = D sqrt(1 - 4 r^2/D^2) (a0 + a1 r^2/D^2 + a2 r^4/D^4)) integrated as a
surface of revolution gives the continuum area and volume that the meshes
must approach at second order, near the published means of 135 um^2 and
94 um^3."""
import numpy as np
import pytest
from scipy.integrate import quad

from paper_2305_02752_gb300 import inputs as I


def _mesh_area_volume(x, t):
    a, b, c = x[t[:, 0]], x[t[:, 1]], x[t[:, 2]]
    area = 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1).sum()
    vol = np.einsum('ij,ij->i', a, np.cross(b, c)).sum() / 6.0
    return area, vol


def _edges(t):
    e = np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]])
    return e


@pytest.mark.parametrize('s', range(5))
def test_icosphere_topology(s):
    v, t = I.icosphere(s)
    nt = 20 * 4 ** s
    assert t.shape == (nt, 3) and len(v) == 10 * 4 ** s + 2
    np.testing.assert_allclose(np.linalg.norm(v, axis=1), 1.0, atol=1e-15)
    e = _edges(t)
    # every directed edge appears once and its reverse once: closed, oriented, manifold
    fwd = {tuple(x) for x in e}
    assert len(fwd) == len(e)
    assert all((b, a) in fwd for a, b in fwd)
    assert len(v) - len(e) // 2 + nt == 2  # Euler characteristic of a sphere
    # outward: every triangle's normal points away from the centre
    a, b, c = v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]
    assert (np.einsum('ij,ij->i', np.cross(b - a, c - a), a + b + c) > 0).all()


def _evans_fung_continuum(D):
    def T(r):
        x = (r / D) ** 2
        return D * np.sqrt(max(0.0, 1.0 - 4.0 * x)) * (I.EF_A0 + I.EF_A1 * x + I.EF_A2 * x * x)

    vol = quad(lambda r: 2.0 * T(r) * 2.0 * np.pi * r, 0.0, D / 2)[0]

    def ring(th):  # r = (D/2) sin(th) removes the rim's infinite slope
        r, dr = 0.5 * D * np.sin(th), 0.5 * D * np.cos(th)
        h = 1e-7
        dz = (T(0.5 * D * np.sin(th + h)) - T(0.5 * D * np.sin(th - h))) / (2 * h)
        return 2.0 * np.pi * r * np.hypot(dr, dz)

    area = 2.0 * quad(ring, 0.0, np.pi / 2, limit=200)[0]
    return area, vol


def test_red_cell_shape():
    D = I.RBC_DIAMETER_UM
    A, V = _evans_fung_continuum(D)
    assert abs(A / 135.0 - 1) < 0.02 and abs(V / 94.0 - 1) < 0.02
    errs, um = [], []
    for s in (3, 4, 5):
        v, t = I.icosphere(s)
        x = I.evans_fung(v, D)
        a, vol = _mesh_area_volume(x, t)
        um.append((a, vol))
        errs.append((a / A - 1, vol / V - 1))
        assert np.ptp(x[:, 0]) == pytest.approx(D, rel=1e-12)
        assert 2.0 < np.ptp(x[:, 2]) < 3.0 and 6.0 < D < 8.0  # Sec. 1
    errs = np.abs(np.array(errs))
    assert (errs[0] < 0.01).all()
    ratio = errs[:-1] / errs[1:]
    assert ((ratio > 3.5) & (ratio < 4.5)).all()  # second order in the edge length
    # the default mesh is the 3-split one in lattice units (dx = 0.5 um)
    x, t = I.rbc_mesh()
    a, vol = _mesh_area_volume(x, t)
    assert a * I.DX_UM ** 2 == pytest.approx(um[0][0], rel=1e-12)
    assert vol * I.DX_UM ** 3 == pytest.approx(um[0][1], rel=1e-12)


def test_platelet_shape():
    x, t = I.platelet_mesh()
    a, c = I.PLATELET_SEMI_AXES_UM[0] / I.DX_UM, I.PLATELET_SEMI_AXES_UM[2] / I.DX_UM
    np.testing.assert_allclose(np.ptp(x, axis=0), [2 * a, 2 * a, 2 * c], rtol=1e-12)
    exact = 4.0 / 3.0 * np.pi * a * a * c
    errs = [abs(_mesh_area_volume(I.spheroid(I.icosphere(s)[0], a, c), I.icosphere(s)[1])[1] / exact - 1)
            for s in (2, 3, 4)]
    assert _mesh_area_volume(x, t)[1] == pytest.approx(exact * (1 - errs[0]), rel=1e-12)
    assert errs[0] < 0.04 and 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


def test_random_rotation_is_uniform():
    rng = np.random.default_rng(11)
    R = np.stack([I.random_rotation(rng) for _ in range(20000)])
    np.testing.assert_allclose(np.einsum('nij,nkj->nik', R, R), np.broadcast_to(np.eye(3), R.shape), atol=1e-13)
    np.testing.assert_allclose(np.linalg.det(R), 1.0, atol=1e-13)
    # Haar measure on SO(3): E[R] = 0 and E[R_ij^2] = 1/3
    assert np.abs(R.mean(axis=0)).max() < 0.02
    assert np.abs((R ** 2).mean(axis=0) - 1 / 3).max() < 0.02


def test_masks_and_profiles():
    m = I.plate_mask(5, 6, 7, axis=1, lo_id=I.WALL_A, hi_id=I.WALL_B)
    assert m.shape == (7, 6, 5)
    assert (m[:, 0, :] == I.WALL_A).all() and (m[:, 5, :] == I.WALL_B).all() and (m[:, 1:5, :] == 0).all()
    u = I.channel_profile(4, 16, 3, 1, 0.5, 14.5, 0.02)
    y = np.arange(16)
    assert np.allclose(u[..., 1:], 0) and np.allclose(u[0, :, 0, 0], u[2, :, 3, 0])
    assert u[0, :, 0, 0].max() == pytest.approx(0.02 * (1 - 0.5 ** 2 / 7 ** 2))  # no node on the centreline 7.5
    assert (u[0, [0, 15], 0, 0] == 0).all() and np.allclose(u[0, y, 0, 0], u[0, 15 - y, 0, 0])
    # the pipe: fluid nodes inside the radius, pi r^2 per cross-section
    cyl = I.cylinder_mask(3, 208, 208, 100.0, 103.5, 103.5)
    nfl = int((cyl[:, :, 0] == 0).sum())
    assert abs(nfl / (np.pi * 100.0 ** 2) - 1) < 1e-3
    assert (cyl == 0).sum() == 3 * nfl


def _overlap_pairs(centers, rots, axes, periodic, span, samples):
    """Pairs whose bounding ellipsoids overlap, by brute force over all pairs
    and dense surface samples (minimum-image distances on periodic axes)."""
    n = len(centers)
    out = 0
    per = np.asarray(periodic, bool)
    for i in range(n):
        for j in range(i + 1, n):
            d = centers[j] - centers[i]
            d = np.where(per, d - span * np.round(d / span), d)
            if np.linalg.norm(d) > axes[i].max() + axes[j].max():
                continue
            pj = d + (samples * axes[j]) @ rots[j].T  # surface of j relative to centre i
            loc = pj @ rots[i]
            if (np.sum((loc / axes[i]) ** 2, axis=1) < 1).any():
                out += 1
    return out


def test_contact_function():
    """Perram-Wertheim F against closed forms and brute force: equal spheres
    (F = d^2 / (2 r)^2), ellipsoids aligned along a shared axis (touching at
    d = a + b), F quadratic in the centre distance, and for random pairs the
    pair scaled to distance d / sqrt(F) touching (no dense surface sample of
    one strictly inside the other, some within 1 %)."""
    eye = np.broadcast_to(np.eye(3), (3, 3, 3))
    d = np.array([[1.5, 0, 0], [0, 2.0, 0], [0, 0, 2.5]])
    F = I.contact_function(d, eye, np.ones((3, 3)), eye, np.ones((3, 3)))
    np.testing.assert_allclose(F, np.array([1.5, 2.0, 2.5]) ** 2 / 4, rtol=1e-9)
    a, b = np.array([[4.0, 1.0, 2.0]]), np.array([[3.0, 2.0, 0.5]])
    for ax in range(3):
        r = np.zeros((1, 3))
        r[0, ax] = 1.0
        F = I.contact_function(r, eye[:1], a, eye[:1], b)
        assert F[0] == pytest.approx(1.0 / (a[0, ax] + b[0, ax]) ** 2, rel=1e-9)
    rng = np.random.default_rng(2)
    n = 12
    Ra = np.stack([I.random_rotation(rng) for _ in range(n)])
    Rb = np.stack([I.random_rotation(rng) for _ in range(n)])
    aa, ab = 1 + 4 * rng.random((n, 3)), 1 + 4 * rng.random((n, 3))
    r = rng.normal(size=(n, 3))
    F = I.contact_function(r, Ra, aa, Rb, ab)
    np.testing.assert_allclose(I.contact_function(2.5 * r, Ra, aa, Rb, ab), 6.25 * F, rtol=1e-9)
    sv, _ = I.icosphere(5)
    for k in range(n):
        rt = r[k] / np.sqrt(F[k])
        surf_b = rt + (sv * ab[k]) @ Rb[k].T
        rad = np.sum(((surf_b @ Ra[k]) / aa[k]) ** 2, axis=1)
        assert rad.min() > 1 - 1e-6 and rad.min() < 1.01


def test_packer():
    kinds = [0] * 40
    lo, hi, per = np.array([0.0, 2.5, 0.0]), np.array([48.0, 45.5, 48.0]), (1, 0, 1)
    bounds = {0: I.RBC_BOUND}
    c0, r0, _ = I.pack_cells(np.random.default_rng(8), lo, hi, per, kinds, bounds, max_iter=0)
    c1, r1, proxy = I.pack_cells(np.random.default_rng(8), lo, hi, per, kinds, bounds)
    c2, r2, resid = I.pack_cells(np.random.default_rng(8), lo, hi, per, kinds, bounds, exact_iter=200)
    c3, r3, _ = I.pack_cells(np.random.default_rng(8), lo, hi, per, kinds, bounds, exact_iter=200)
    assert np.array_equal(c2, c3) and np.array_equal(r2, r3)  # seeded
    assert np.array_equal(r0, r1) and np.array_equal(r0, r2)  # only the centres move
    axes = np.tile(np.array(I.RBC_BOUND), (40, 1))
    samples, _ = I.icosphere(3)
    span = hi - lo
    before = _overlap_pairs(c0, r0, axes, per, span, samples)
    proxy_left = _overlap_pairs(c1, r1, axes, per, span, samples)
    assert proxy == 0 and before >= 20 and proxy_left < before  # the sample proxy misses shallow overlaps
    assert resid == 0 and _overlap_pairs(c2, r2, axes, per, span, samples) == 0
    # inside the box: wrapped on periodic axes, whole bounding ellipsoid on the others
    ext = np.sqrt(np.einsum('njk,nk->nj', r2 ** 2, axes ** 2))
    assert ((c2[:, [0, 2]] >= 0) & (c2[:, [0, 2]] < 48)).all()
    assert (c2[:, 1] - ext[:, 1] >= 2.5 - 1e-9).all() and (c2[:, 1] + ext[:, 1] <= 45.5 + 1e-9).all()


def test_packer_cylinder():
    """With the cylinder constraint every bounding ellipsoid lies inside the
    cylinder about the x axis (dense surface samples within the radius), in
    both phases, and a moderately dense pipe is packed free of overlap."""
    kinds = [0] * 14
    cy = cz = 20.0
    radius = 18.0
    lo, hi, per = np.array([0.0, cy - radius, cz - radius]), np.array([60.0, cy + radius, cz + radius]), (1, 0, 0)
    axes = np.tile(np.array(I.RBC_BOUND), (14, 1))
    samples, _ = I.icosphere(4)
    for exact in (0, 400):
        c, r, resid = I.pack_cells(np.random.default_rng(5), lo, hi, per, kinds, {0: I.RBC_BOUND},
                                   max_iter=100, exact_iter=exact, cylinder=(cy, cz, radius))
        surf = c[:, None, :] + np.einsum('pk,nk,njk->npj', samples, axes, r)
        rad = np.hypot(surf[..., 1] - cy, surf[..., 2] - cz)
        assert rad.max() <= radius + 1e-9, exact
        if exact:
            assert resid == 0
            assert _overlap_pairs(c, r, axes, per, hi - lo, samples) == 0


def test_pipe_placement_inside_the_wall():
    """The pipe workload (1000 x 208 x 208, 19,600 red cells): every cell's
    bounding ellipsoid lies at least 3 nodes inside the voxelised wall."""
    cy = (208 - 1) / 2.0
    c, r, _ = I.pipe_placement(np.random.default_rng(20230504), 1000, cy, cy, 97.0, 19600, 1, 0)
    assert len(c) == 19600
    axes = np.tile(np.array(I.RBC_BOUND), (len(c), 1))
    samples, _ = I.icosphere(2)
    surf = c[:, None, :] + np.einsum('pk,nk,njk->npj', samples, axes, r)
    assert np.hypot(surf[..., 1] - cy, surf[..., 2] - cy).max() <= 97.0 + 1e-9


def _red_cell_overlaps(cfg):
    """Pairs of red cells with a vertex of one inside the other's biconcave
    body (|z| < T(r) in its frame, the Evans-Fung profile)."""
    D = I.RBC_DIAMETER_UM / I.DX_UM

    def T(r):
        x = (r / D) ** 2
        return D * np.sqrt(np.clip(1.0 - 4.0 * x, 0.0, None)) * (I.EF_A0 + I.EF_A1 * x + I.EF_A2 * x * x)

    rest = cfg.meshes[0].rest
    C, R = cfg.centers, cfg.rotations
    span = np.array([cfg.nx, cfg.ny, cfg.nz], float)
    per = np.array(cfg.periodic, bool)
    bad = 0
    for i in range(len(C)):
        d = C - C[i]
        d = np.where(per, d - span * np.round(d / span), d)
        for j in np.where((np.linalg.norm(d, axis=1) < 2 * D) & (np.arange(len(C)) > i))[0]:
            loc = (d[j] + rest @ R[j].T) @ R[i]
            r = np.hypot(loc[:, 0], loc[:, 1])
            bad += bool(((r < D / 2) & (np.abs(loc[:, 2]) < T(r))).any())
    return bad


@pytest.fixture(scope='module')
def channel():
    return I.channel()


def test_channel_configuration(channel):
    cfg = channel
    assert (cfg.nx, cfg.ny, cfg.nz) == (64, 64, 256) and cfg.periodic == (1, 0, 1)
    assert len(cfg.centers) == 440 and cfg.n_vertices == 440 * 642
    assert cfg.n_fluid == 64 * 62 * 256
    X = I.cell_vertices(cfg)
    assert X.shape == (cfg.n_vertices, 3)
    # every vertex starts in the fluid between the walls at y = 0 and y = 63
    assert X[:, 1].min() > 1.0 and X[:, 1].max() < 62.0
    # placed without overlap: bounding ellipsoids (dense samples) and the cells themselves
    assert cfg.note.endswith(': 0')
    assert _overlap_pairs(cfg.centers, cfg.rotations, np.tile(np.array(I.RBC_BOUND), (440, 1)), cfg.periodic,
                          np.array([64.0, 64.0, 256.0]), I.icosphere(2)[0]) == 0
    assert _red_cell_overlaps(cfg) == 0
    # haematocrit of the seeded suspension: cell volume over fluid volume
    _, v = _mesh_area_volume(cfg.meshes[0].rest, cfg.meshes[0].tri)
    assert 0.28 < 440 * v / cfg.n_fluid < 0.34  # about 30 %
    again = I.channel()
    assert np.array_equal(cfg.centers, again.centers) and np.array_equal(cfg.rotations, again.rotations)


def test_kbt_scaling():
    """dt = nu_LU dx^2 / nu, so the lattice energy unit rho dx^5 / dt^2 goes as
    dx / (tau - 1/2)^2 and kBT in lattice units as (tau - 1/2)^2 / dx."""
    k = I.kbt_lattice(1.0)
    assert I.kbt_lattice(1.5) / k == pytest.approx(4.0, rel=1e-12)
    assert I.kbt_lattice(1.0, 0.25) / k == pytest.approx(2.0, rel=1e-12)
    assert k == pytest.approx(1.917e-7, rel=1e-3)


def test_locality_order_renumbers_the_same_surface():
    """The renumbering is a bijection of the vertices that keeps every
    triangle (with its orientation) and brings neighbouring vertices to
    nearby ids."""
    v, t = I.icosphere(3)
    v2, t2 = I.locality_order(v, t)
    assert v2.shape == v.shape and t2.shape == t.shape
    # recover the permutation from the positions
    key = {tuple(np.round(p, 12)): k for k, p in enumerate(v)}
    old = np.array([key[tuple(np.round(p, 12))] for p in v2])
    assert sorted(old) == list(range(len(v)))
    # triangle k of the renumbered mesh is triangle k of the original
    assert np.array_equal(old[t2], t)
    gap = lambda tt: np.median(np.abs(np.concatenate([tt[:, 0] - tt[:, 1], tt[:, 1] - tt[:, 2], tt[:, 2] - tt[:, 0]])))
    assert gap(t2) < gap(t) / 10
    a0, v0 = _mesh_area_volume(v, t)
    a1, v1 = _mesh_area_volume(v2, t2)
    assert abs(a1 - a0) < 1e-12 * a0 and abs(v1 - v0) < 1e-12 * v0
