"""Pins of the CPU oracle against what the paper and the mathematics fix.

The paper prints no worked example with numbers for the coupled step, so the
oracle is pinned by exact identities, closed-form flows, conservation laws,
invariances and brute force.  Each test names the passage it pins.
"""
import fractions
import math

import numpy as np
import pytest

import oracle as O
from paper_2305_02752_gb300 import inputs as I


# ---------------------------------------------------------------------------
# Sec. 2.2: D3Q19 tables and the equilibrium
# ---------------------------------------------------------------------------
def test_d3q19_exact_moments():
    """Lattice isotropy fixed by c_s^2 = 1/3 (Sec. 2.2): sum w = 1,
    sum w c_a = 0, sum w c_a c_b = delta/3, fourth moment = (dd+dd+dd)/9,
    checked in exact rational arithmetic."""
    c, w, opp = O.d3q19()
    wf = [fractions.Fraction(x).limit_denominator(1000) for x in w]
    assert all(abs(float(a) - b) < 1e-16 for a, b in zip(wf, w))
    assert sum(wf) == 1
    assert sorted(wf).count(fractions.Fraction(1, 36)) == 12
    assert sorted(wf).count(fractions.Fraction(1, 18)) == 6
    for a in range(3):
        assert sum(wf[i] * c[i, a] for i in range(19)) == 0
        for b in range(3):
            assert sum(wf[i] * c[i, a] * c[i, b] for i in range(19)) == (fractions.Fraction(1, 3) if a == b else 0)
            for g in range(3):
                assert sum(wf[i] * c[i, a] * c[i, b] * c[i, g] for i in range(19)) == 0
                for d in range(3):
                    m4 = sum(wf[i] * c[i, a] * c[i, b] * c[i, g] * c[i, d] for i in range(19))
                    ex = fractions.Fraction(int(a == b and g == d) + int(a == g and b == d) + int(a == d and b == g), 9)
                    assert m4 == ex
    for i in range(19):
        assert np.all(c[opp[i]] == -c[i])
    assert len({tuple(x) for x in c}) == 19


@pytest.mark.parametrize('seed', range(4))
def test_equilibrium_moments(seed):
    """The equilibrium of Sec. 2.2 reproduces rho and rho u exactly and the
    momentum flux rho/3 I + rho u u."""
    rng = np.random.default_rng(seed)
    rho = 0.8 + 0.4 * rng.random()
    u = 0.1 * rng.normal(size=3)
    feq = O.equilibrium(rho, u)
    c, _, _ = O.d3q19()
    assert abs(feq.sum() - rho) < 1e-15
    assert np.abs(feq @ c - rho * u).max() < 1e-15
    pi = np.einsum('i,ia,ib->ab', feq, c, c)
    assert np.abs(pi - (rho / 3.0 * np.eye(3) + rho * np.outer(u, u))).max() < 1e-14


# ---------------------------------------------------------------------------
# Sec. 2.2 + 2.5: closed-form flows
# ---------------------------------------------------------------------------
def test_couette_exact():
    """Plates moving at -/+0.01 (Sec. 2.5 shear): the steady LBM profile is
    the linear Couette profile between the effective walls at z = 0.5 and
    z = 30.5, to round-off."""
    n = 32
    mask = I.plate_mask(1, 1, n, axis=2, lo_id=I.WALL_A, hi_id=I.WALL_B)
    s = O.OracleSim(1, 1, n, 1.0, (1, 1, 0), mask, np.array([[-0.01, 0, 0], [0.01, 0, 0]]))
    s.set_velocity(None)
    s.step(30000)
    u = s.get()['u'][:, 0, 0, :]
    z = np.arange(n)
    ex = -0.01 + 0.02 * (z - 0.5) / (n - 2)
    assert np.abs(u[1:-1, 0] - ex[1:-1]).max() < 1e-10
    assert np.abs(u[1:-1, 1:]).max() < 1e-14


def _poiseuille(H, steps_factor=8.0, tau=1.0):
    ny = H + 2
    mask = I.plate_mask(1, ny, 1, axis=1)
    nu = (tau - 0.5) / 3
    g = 8 * nu * 0.02 / H ** 2
    s = O.OracleSim(1, ny, 1, tau, (1, 0, 1), mask, None, np.array([g, 0, 0]))
    s.set_velocity(None)
    s.step(int(steps_factor * H * H / nu))
    u = s.get()['u'][0, :, 0, 0]
    y = np.arange(ny)
    ex = g / (2 * nu) * (y - 0.5) * (ny - 1.5 - y)
    return np.abs(u[1:-1] - ex[1:-1]).max() / ex.max()


def test_poiseuille_profile_and_convergence():
    """Body-force channel with halfway bounce-back: parabolic profile within
    1 %, error falling as H^-2."""
    errs = [_poiseuille(H) for H in (14, 30, 62)]
    assert max(errs) < 0.01
    assert 3.5 < errs[0] / errs[1] < 5.5
    assert 3.5 < errs[1] / errs[2] < 5.5


def test_poiseuille_magic_tau():
    """At tau = 1/2 + sqrt(3/16) halfway bounce-back places the wall exactly
    and the Poiseuille profile is reproduced to round-off."""
    assert _poiseuille(14, steps_factor=20.0, tau=0.5 + math.sqrt(3.0 / 16.0)) < 1e-9


def test_startup_transient():
    """Flow started from rest by a body force between resting plates follows
    the Fourier-series solution of the diffusion equation, to O(dx^2)."""
    H = 30
    ny = H + 2
    nu = 1.0 / 6.0
    g = 1e-6
    mask = I.plate_mask(1, ny, 1, axis=1)
    s = O.OracleSim(1, ny, 1, 1.0, (1, 0, 1), mask, None, np.array([g, 0, 0]))
    s.set_velocity(None)
    t = int(0.05 * H * H / nu)
    s.step(t)
    u = s.get()['u'][0, 1:-1, 0, 0]
    y = np.arange(1, ny - 1) - 0.5
    ex = g / (2 * nu) * y * (H - y)
    for k in range(1, 400, 2):
        ex -= 4 * g * H * H / (nu * math.pi ** 3 * k ** 3) * np.sin(k * math.pi * y / H) * math.exp(-nu * (k * math.pi / H) ** 2 * (t + 0.5))
    assert np.abs(u - ex).max() / np.abs(ex).max() < 2e-3


# ---------------------------------------------------------------------------
# conservation
# ---------------------------------------------------------------------------
def _small_shear_with_cell(n=24, seed=5):
    cfg = I.shear_cell(n=n, ncell=1, seed=seed, steps=50)
    mt = cfg.meshes[0]
    # a smaller cell so that it fits the small box with room for the stencil
    mt.rest = I.evans_fung(I.icosphere(2)[0], 8.0)
    mt.tri = I.icosphere(2)[1]
    return cfg


def test_mass_conservation_walls_and_cells():
    """sum f is conserved by BGK + forcing + halfway bounce-back, including
    moving walls and immersed cells (relative 1e-13)."""
    cfg = _small_shear_with_cell()
    s = O.from_config(cfg)
    m0 = s.populations().sum()
    s.step(60)
    m1 = s.populations().sum()
    assert abs(m1 - m0) / m0 < 1e-13


def test_momentum_balance_periodic():
    """Fully periodic box: total momentum grows by exactly sum_x F(x) per step
    (body force plus spread membrane forces; the latter sum to zero)."""
    n = 16
    g = np.array([1e-5, -2e-5, 3e-6])
    s = O.OracleSim(n, n, n, 0.8, (1, 1, 1), None, None, g)
    rng = np.random.default_rng(3)
    u0 = 0.01 * rng.normal(size=(n, n, n, 3))
    s.set_velocity(u0)
    v, t = I.icosphere(1)
    X = v * 3.0
    s.add_mesh(X, t, np.array([15.0, 80.0, 5.0, 20.0, 1e-3, 0.015, 3.0]))
    s.add_cells(0, np.array([[8.0, 8.3, 7.6]]), (I.random_rotation(rng) @ np.diag([1.2, 1.0, 0.8]))[None])
    c, _, _ = O.d3q19()
    p0 = np.einsum('zyxi,ia->a', s.populations(), c)
    s.step(5)
    out = s.get()
    p1 = np.einsum('zyxi,ia->a', s.populations(), c)
    # membrane forces of the last step sum to zero (rigid invariance)
    assert np.abs(out['Fv'].sum(0)).max() < 1e-15 * 1e3
    expected = 5 * n ** 3 * g
    assert np.abs((p1 - p0) - expected).max() < 1e-12


# ---------------------------------------------------------------------------
# Sec. 2.3 coupling kernel
# ---------------------------------------------------------------------------
def test_peskin_kernel_identities():
    """Peskin 4-point kernel: partition of unity, zero first moment, even/odd
    sums 1/2, sum of squares 3/8, and its closed-form values."""
    rng = np.random.default_rng(0)
    for r in rng.random(50) * 4 - 2:
        j = np.arange(-6, 7)
        p = O.phi(r - j)
        assert abs(p.sum() - 1) < 1e-15
        assert abs(((r - j) * p).sum()) < 1e-15
        assert abs(p[j % 2 == 0].sum() - 0.5) < 1e-15
        assert abs((p ** 2).sum() - 3.0 / 8.0) < 1e-15
    assert O.phi(np.array([0.0]))[0] == 0.5
    assert abs(O.phi(np.array([1.0]))[0] - 0.25) < 1e-16
    assert O.phi(np.array([2.0]))[0] == 0.0
    assert O.phi(np.array([2.5]))[0] == 0.0
    assert abs(O.phi(np.array([0.5]))[0] - (2 + math.sqrt(2)) / 8) < 1e-16
    assert abs(O.phi(np.array([1.5]))[0] - (2 - math.sqrt(2)) / 8) < 1e-16


def test_spread_interpolate_adjoint_and_conservation():
    """<S F_v, u> = <F_v, I u>, sum_x S F_v = sum_v F_v away from walls, and a
    uniform velocity is interpolated exactly."""
    rng = np.random.default_rng(7)
    nx, ny, nz = 12, 10, 14
    s = O.OracleSim(nx, ny, nz, 1.0, (1, 1, 1))
    X = rng.random((40, 3)) * [nx, ny, nz] + rng.normal(size=(40, 3)) * 3   # wraps too
    Fv = rng.normal(size=(40, 3))
    u = rng.normal(size=(nz, ny, nx, 3))
    SF = s.spread(X, Fv)
    Iu = s.interpolate(X, u)
    assert abs((SF * u).sum() - (Fv * Iu).sum()) < 1e-12
    assert np.abs(SF.sum(axis=(0, 1, 2)) - Fv.sum(0)).max() < 1e-12
    U = s.interpolate(X, np.broadcast_to(np.array([0.3, -0.2, 0.1]), u.shape))
    assert np.abs(U - [0.3, -0.2, 0.1]).max() < 1e-15


# ---------------------------------------------------------------------------
# Sec. 2.3 membrane forces
# ---------------------------------------------------------------------------
PARAMS_FD = np.array([15.0, 80.0, 5.0, 20.0, 1e-3, 0.015, 3.0])


def _fd_forces(rest, tri, params, X, idx, h):
    fd = np.zeros((len(idx), 3))
    for a, i in enumerate(idx):
        for k in range(3):
            Xp = X.copy(); Xp[i, k] += h
            Xm = X.copy(); Xm[i, k] -= h
            fd[a, k] = -(O.membrane(rest, tri, params, Xp)[1].sum() - O.membrane(rest, tri, params, Xm)[1].sum()) / (2 * h)
    return fd


@pytest.mark.parametrize('term', [None, 0, 1, 2, 3])
def test_membrane_forces_are_energy_gradient_icosahedron(term):
    """F_total = F_link + F_bend + F_area + F_volume (Sec. 2.3) is minus the
    gradient of the stated energies: central differences on a randomly
    perturbed 12-vertex icosahedron, each term alone and all together."""
    rng = np.random.default_rng(11 if term is None else term)
    v, t = I.icosphere(0)
    rest = v * 3.0
    p = PARAMS_FD.copy()
    if term is not None:
        for j in range(4):
            if j != term:
                p[j] = 0.0
    X = rest + 0.15 * rng.normal(size=rest.shape)
    F, _, _ = O.membrane(rest, t, p, X)
    fd = _fd_forces(rest, t, p, X, range(len(X)), 1e-6)
    assert np.linalg.norm(F - fd) / np.linalg.norm(F) < 1e-7


def test_membrane_forces_gradient_rbc_mesh():
    """Same check on the 642-vertex red-cell mesh (sampled vertices)."""
    rng = np.random.default_rng(2)
    rest, t = I.rbc_mesh()
    X = rest + 0.05 * rng.normal(size=rest.shape)
    p = PARAMS_FD.copy()
    F, _, _ = O.membrane(rest, t, p, X)
    idx = rng.choice(len(X), 12, replace=False)
    fd = _fd_forces(rest, t, p, X, idx, 1e-5)
    assert np.linalg.norm(F[idx] - fd) / np.linalg.norm(F[idx]) < 1e-7


def test_membrane_rest_state_has_no_force():
    for rest, t in (I.rbc_mesh(), I.platelet_mesh(), (I.icosphere(0)[0] * 2, I.icosphere(0)[1])):
        F, E, AV = O.membrane(rest, t, PARAMS_FD, rest)
        assert np.abs(F).max() <= 1e-14 * PARAMS_FD[:4].max()
        assert np.abs(E).max() == 0.0


def test_membrane_rigid_motion_invariance():
    """Net force and torque vanish and forces rotate with the body."""
    rng = np.random.default_rng(4)
    rest, t = I.rbc_mesh()
    X = rest + 0.1 * rng.normal(size=rest.shape)
    F, E, _ = O.membrane(rest, t, PARAMS_FD, X)
    scale = np.abs(F).max()
    assert np.abs(F.sum(0)).max() < 1e-12 * scale * len(X)
    assert np.abs(np.cross(X, F).sum(0)).max() < 1e-11 * scale * len(X)
    R = I.random_rotation(rng)
    shift = np.array([13.1, -4.2, 7.7])
    F2, E2, _ = O.membrane(rest, t, PARAMS_FD, X @ R.T + shift)
    assert np.abs(F2 - F @ R.T).max() < 1e-10 * scale
    assert np.allclose(E2, E, rtol=1e-10)


def test_area_volume_converge_on_sphere():
    """Area and volume of the icosphere tend to 4 pi and 4 pi / 3 at O(h^2)."""
    errA, errV = [], []
    for k in range(1, 5):
        v, t = I.icosphere(k)
        _, _, AV = O.membrane(v, t, PARAMS_FD, v)
        errA.append(abs(AV[0] - 4 * math.pi))
        errV.append(abs(AV[1] - 4 * math.pi / 3))
    for e in (errA, errV):
        for a, b in zip(e, e[1:]):
            assert 3.0 < a / b < 5.0
    # volume of a closed mesh does not depend on the reference point
    v, t = I.icosphere(2)
    _, _, AV1 = O.membrane(v, t, PARAMS_FD, v)
    _, _, AV2 = O.membrane(v, t, PARAMS_FD, v + 100.0)
    assert abs(AV1[1] - AV2[1]) < 1e-11


def test_red_cell_shape_numbers():
    """Evans-Fung red cell at dx = 0.5 um: about 135 um^2 and 94 um^3."""
    rest, t = I.rbc_mesh()
    _, _, AV = O.membrane(rest, t, PARAMS_FD, rest)
    assert 125 < AV[0] * 0.25 < 140
    assert 88 < AV[1] * 0.125 < 96


# ---------------------------------------------------------------------------
# mesh integers
# ---------------------------------------------------------------------------
@pytest.mark.parametrize('k,counts', [(0, (12, 30, 20)), (2, (162, 480, 320)), (3, (642, 1920, 1280))])
def test_mesh_counts_and_edge_table(k, counts):
    v, t = I.icosphere(k)
    E = O.build_edges(len(v), t)
    assert (len(v), len(E), len(t)) == counts
    assert len(v) - len(E) + len(t) == 2
    # brute force: every edge lies on exactly two triangles, (v0,v1,a) and
    # (v1,v0,b) as cyclic orientations
    cyc = set()
    for tri in t:
        for r in range(3):
            cyc.add(tuple(np.roll(tri, r)))
    seen = set()
    for v0, v1, a, b in E:
        assert (v0, v1, a) in cyc and (v1, v0, b) in cyc
        key = (min(v0, v1), max(v0, v1))
        assert key not in seen
        seen.add(key)
    owners = {}
    for tri in t:
        for r in range(3):
            key = (min(tri[r], tri[(r + 1) % 3]), max(tri[r], tri[(r + 1) % 3]))
            owners[key] = owners.get(key, 0) + 1
    assert set(owners.values()) == {2} and set(owners) == seen
    # discovery order: edge ids follow first appearance in the triangle list
    first = []
    for tri in t:
        for r in range(3):
            key = (min(tri[r], tri[(r + 1) % 3]), max(tri[r], tri[(r + 1) % 3]))
            if key not in first:
                first.append(key)
            if len(first) > 40:
                break
        if len(first) > 40:
            break
    got = [(min(e[0], e[1]), max(e[0], e[1])) for e in E[:len(first)]]
    assert got == first


def test_deformation_index():
    v, t = I.icosphere(3)
    assert abs(O.deformation_index(v * 5.0)) < 1e-12
    for s in (1.3, 2.0):
        assert abs(O.deformation_index(v * [s, 1, 1]) - (s - 1) / (s + 1)) < 1e-12


def test_deformation_loss_closed_form():
    """The loss of the differentiation form (mean Taylor deformation index
    plus mean squared centroid drift) in closed form: a round cell
    (icosphere, DI = 0) and a cell stretched by diag(s, 1, 1)
    (DI = (s - 1)/(s + 1)), each moved rigidly after placement: cell c by a
    rotation about its centroid and a translation d_c.  DI is invariant
    under the rigid motion and the centroid moves by d_c from where the
    cells were placed, so loss = ((s - 1)/(s + 1) + |d_0|^2 + |d_1|^2) / 2.
    A wrong sign, a missing 1/ncell or the wrong reference centroid fails."""
    v, t = I.icosphere(3)
    s = 1.6
    params = [1.0, 1.0, 1.0, 1.0, 1e-7, 0.015, 3.0]
    sim = O.OracleSim(64, 64, 64, 1.0, (1, 1, 1))
    sim.add_mesh(v * 5.0, t, params)
    sim.add_mesh(v * [5.0 * s, 5.0, 5.0], t, params)
    centers = np.array([[20.0, 30.0, 31.0], [40.0, 22.0, 35.0]])
    sim.add_cells(0, centers[:1], np.eye(3)[None])
    sim.add_cells(1, centers[1:], np.eye(3)[None])
    X0 = np.concatenate([v * 5.0 + centers[0], v * [5.0 * s, 5.0, 5.0] + centers[1]])
    di1 = (s - 1) / (s + 1)
    assert abs(sim.loss() - di1 / 2) < 1e-12  # no drift at placement
    rng = np.random.default_rng(3)
    d = np.array([[1.5, -0.75, 2.0], [-3.0, 0.5, 0.25]])
    nv = len(v)
    X = X0.copy()
    for c in range(2):
        R = I.random_rotation(rng)
        Xc = X0[c * nv:(c + 1) * nv]
        X[c * nv:(c + 1) * nv] = (Xc - centers[c]) @ R.T + centers[c] + d[c]
    sim.set_vertices(X)
    expect = (di1 + (d ** 2).sum()) / 2
    assert abs(sim.loss() - expect) < 1e-12 * max(1.0, expect)
    # only the drift changes with a further translation of one cell
    X[:nv] += [0.0, 0.0, 1.0]
    sim.set_vertices(X)
    expect2 = (di1 + (d ** 2).sum() - d[0, 2] ** 2 + (d[0, 2] + 1.0) ** 2) / 2
    assert abs(sim.loss() - expect2) < 1e-12 * max(1.0, expect2)


def test_storage_reference_closed_forms():
    """Reference of the 16-bit storage form for a row velocity (U, 0, 0):
    zero at U = 0 and on every direction with c_x = 0; its mass is U^2 and
    its x-momentum U (sum_i K_i = 3 U^2 sum_{c_x != 0} w_i = U^2 and
    sum_i K_i c_x = 3 U sum w_i c_x^2 = U), no y or z momentum; and the
    equilibrium of (U, 0, 0) minus w minus K leaves exactly -1.5 w_i U^2 on
    the directions with c_x = 0 and nothing on the others."""
    c, w, _ = O.d3q19()
    assert not O.storage_reference(0.0).any()
    for U in (0.02, -0.013, 0.1):
        K = O.storage_reference(U)
        assert (K[c[:, 0] == 0] == 0).all()
        assert abs(K.sum() - U * U) < 1e-16
        assert abs((K * c[:, 0]).sum() - U) < 1e-16
        assert abs((K * c[:, 1]).sum()) < 1e-16 and abs((K * c[:, 2]).sum()) < 1e-16
        rest = O.equilibrium(1.0, [U, 0.0, 0.0]) - w - K
        np.testing.assert_allclose(rest[c[:, 0] != 0], 0.0, atol=1e-17)
        np.testing.assert_allclose(rest[c[:, 0] == 0], -1.5 * w[c[:, 0] == 0] * U * U, rtol=1e-12)


# ---------------------------------------------------------------------------
# integer work: binning, wall links (brute force)
# ---------------------------------------------------------------------------
def test_bins_match_stable_argsort():
    rng = np.random.default_rng(9)
    nx, ny, nz = 40, 24, 33
    s = O.OracleSim(nx, ny, nz, 1.0, (1, 0, 1))
    X = rng.random((3000, 3)) * [nx, ny, nz] + rng.normal(size=(3000, 3)) * [20, 0, 20]
    X[:, 1] = np.clip(X[:, 1], 0, ny - 1e-9)
    X[::7] = np.floor(X[::7])     # exactly on node planes
    B = 8
    key, perm, start = s.bins(X, B)
    fl = np.floor(X).astype(np.int64)
    fl[:, 0] %= nx
    fl[:, 2] %= nz
    nb = [(nx + B - 1) // B, (ny + B - 1) // B, (nz + B - 1) // B]
    k2 = fl[:, 0] // B + nb[0] * (fl[:, 1] // B + nb[1] * (fl[:, 2] // B))
    assert np.array_equal(key, k2)
    assert np.array_equal(perm, np.argsort(k2, kind='stable'))
    assert np.array_equal(start, np.concatenate([[0], np.cumsum(np.bincount(k2, minlength=np.prod(nb)))]))


def test_wall_links_brute_force():
    rng = np.random.default_rng(1)
    nx, ny, nz = 7, 6, 5
    mask = (rng.random((nz, ny, nx)) < 0.25).astype(np.uint8)
    s = O.OracleSim(nx, ny, nz, 1.0, (1, 0, 1), mask)
    links = s.wall_links()
    c, _, _ = O.d3q19()
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                b = 0
                if not mask[z, y, x]:
                    for i in range(19):
                        xx, yy, zz = (x + c[i, 0]) % nx, y + c[i, 1], (z + c[i, 2]) % nz
                        if yy < 0 or yy >= ny or mask[zz, yy, xx]:
                            b |= 1 << i
                assert links[z, y, x] == b


def test_thread_count_does_not_change_results():
    """The oracle's loops over independent nodes, cells and vertices may run
    on several threads: the coupled state is the same bits with 1 and 4."""
    from tests.helpers import small_cell_shear
    cfg = small_cell_shear(n=16, steps=6)
    out = []
    for nt in (1, 4):
        O.set_threads(nt)
        try:
            s = O.from_config(cfg)
            s.step(6)
            out.append((s.get(), s.populations()))
            s.close()
        finally:
            O.set_threads(1)
    (a, fa), (b, fb) = out
    assert np.array_equal(fa, fb)
    for k in ('u', 'X', 'Fv', 'rho'):
        assert np.array_equal(a[k], b[k]), k
