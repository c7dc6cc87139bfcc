"""Pins of the oracle's element matrices against closed forms and invariants.

Beam: Euler-Bernoulli cantilever closed forms (tip PL^3/3EI in both planes,
PL/EA, TL/GJ, ML^2/2EI), symmetry, exactly six rigid-body null modes, the
vertical-member axis rule.  Quad (MITC-4 flat facet, Sec. 2.2.1): symmetry, six
null modes on flat / distorted / warped elements, membrane and bending patch
tests on a distorted patch, the cubic dependence on thickness, FD of dk/dz.
"""
import numpy as np
import pytest

import meshgen

E, G, IY, IZ, J, A = 2.1e11, 8.0e10, 3.0e-6, 1.2e-6, 2.5e-6, 2.0e-3


def _rot(seed):
    q, r = np.linalg.qr(np.random.default_rng(seed).normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def _cantilever(orc, ex, L=2.5):
    """12x12 beam along unit vector ex; returns (K free end 6x6, R local axes)."""
    xi = np.array([0.3, -0.2, 0.1])
    xj = xi + L * ex
    K = orc.beam_ke(xi, xj, [E, G, IY, IZ, J, A])
    return K[6:, 6:]


@pytest.mark.parametrize("direction", [(1, 0, 0), (0.3, 0.8, -0.2), (-0.5, 0.1, 0.7)])
def test_beam_cantilever_closed_forms(orc, direction):
    L = 2.5
    ex = np.asarray(direction, float)
    ex /= np.linalg.norm(ex)
    ey = np.cross([0, 0, 1.0], ex)
    ey /= np.linalg.norm(ey)
    ez = np.cross(ex, ey)
    Kf = _cantilever(orc, ex, L)

    def tip(force=None, moment=None):
        f = np.zeros(6)
        if force is not None:
            f[:3] = force
        if moment is not None:
            f[3:] = moment
        return np.linalg.solve(Kf, f)

    P = 1234.0
    u = tip(force=P * ez)  # bending in local x-z -> Iy
    assert np.dot(u[:3], ez) == pytest.approx(P * L ** 3 / (3 * E * IY), rel=1e-12)
    u = tip(force=P * ey)  # bending in local x-y -> Iz
    assert np.dot(u[:3], ey) == pytest.approx(P * L ** 3 / (3 * E * IZ), rel=1e-12)
    assert np.dot(u[3:], ez) == pytest.approx(P * L ** 2 / (2 * E * IZ), rel=1e-12)
    u = tip(force=P * ex)
    assert np.dot(u[:3], ex) == pytest.approx(P * L / (E * A), rel=1e-12)
    u = tip(moment=P * ex)
    assert np.dot(u[3:], ex) == pytest.approx(P * L / (G * J), rel=1e-12)
    u = tip(moment=P * ey)  # end moment about local y: w = M L^2 / 2EIy
    assert abs(np.dot(u[:3], ez)) == pytest.approx(P * L ** 2 / (2 * E * IY), rel=1e-12)
    assert np.dot(u[3:], ey) == pytest.approx(P * L / (E * IY), rel=1e-12)


def test_beam_multi_element_cantilever_exact(orc):
    """Euler-Bernoulli elements are exact for point loads: 5 elements give PL^3/3EI."""
    n, L, P = 5, 4.0, -700.0
    model = meshgen.empty_model(n + 1)
    model["xyz"][:, 0] = np.linspace(0, L, n + 1)
    model["beam_conn"] = np.stack([np.arange(n), np.arange(1, n + 1)], 1).astype(np.int32)
    model["beam_props"] = np.tile([E, G, IY, IZ, J, A], (n, 1))
    model["fixed"][0] = 1
    model["nodal_load"][n, 2] = P
    u, C = orc.solve(model)
    assert u[6 * n + 2] == pytest.approx(P * L ** 3 / (3 * E * IY), rel=1e-11)
    assert C == pytest.approx(P * u[6 * n + 2], rel=1e-14)


def test_beam_vertical_member_axis_rule(orc):
    """Within 1e-8 of vertical, local y = global Y: a Y load bends about Iz."""
    L, P = 3.0, 500.0
    K = orc.beam_ke([0, 0, 0], [0, 0, L], [E, G, IY, IZ, J, A])[6:, 6:]
    f = np.zeros(6)
    f[1] = P
    u = np.linalg.solve(K, f)
    assert u[1] == pytest.approx(P * L ** 3 / (3 * E * IZ), rel=1e-12)
    f = np.zeros(6)
    f[0] = P
    u = np.linalg.solve(K, f)
    assert u[0] == pytest.approx(P * L ** 3 / (3 * E * IY), rel=1e-12)


def test_beam_symmetry_and_null_space(orc):
    K = orc.beam_ke([0.1, 0.2, 0.3], [1.1, 0.7, 1.5], [E, G, IY, IZ, J, A])
    assert np.abs(K - K.T).max() <= 1e-14 * np.abs(K).max()
    ev = np.sort(np.abs(np.linalg.eigvalsh(K))) / np.abs(K).max()
    assert np.all(ev[:6] < 1e-12) and ev[6] > 1e-6
    # the null space is exactly the rigid motions
    X = np.array([[0.1, 0.2, 0.3], [1.1, 0.7, 1.5]])
    for rigid in _rigid_modes(X):
        assert np.linalg.norm(K @ rigid) <= 1e-9 * np.abs(K).max() * np.linalg.norm(rigid)


def _rigid_modes(X):
    """6 rigid-body displacement fields of the nodes X [n,3] (node-major 6 dofs)."""
    modes = []
    for k in range(3):
        m = np.zeros((X.shape[0], 6))
        m[:, k] = 1.0
        modes.append(m.ravel())
    for k in range(3):
        w = np.zeros(3)
        w[k] = 1.0
        m = np.zeros((X.shape[0], 6))
        m[:, :3] = np.cross(w, X)
        m[:, 3:] = w
        modes.append(m.ravel())
    return modes


QUADS = {
    "square": np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0]], float),
    "distorted": np.array([[0, 0, 0], [1.3, 0.1, 0], [1.1, 0.9, 0], [-0.2, 1.2, 0]], float),
    "warped": np.array([[0, 0, 0.05], [1.2, 0.1, -0.08], [1.1, 1.0, 0.12], [0.1, 0.9, -0.02]], float),
    "tilted": np.array([[0, 0, 0], [1, 0, 0.5], [1.2, 1, 1.1], [0.1, 1.1, 0.4]], float),
}
QPROPS = np.array([0.12, 3.0e10, 0.2, 1.0, 1.0])


@pytest.mark.parametrize("name", sorted(QUADS))
def test_quad_symmetry_and_rigid_modes(orc, name):
    X = QUADS[name]
    K = orc.quad_ke(X, QPROPS)
    scale = np.abs(K).max()
    assert np.abs(K - K.T).max() <= 1e-13 * scale
    ev = np.sort(np.abs(np.linalg.eigvalsh(K))) / scale
    assert np.all(ev[:6] < 1e-12), ev[:8]
    assert ev[6] > 1e-7, ev[:8]
    for rigid in _rigid_modes(X):
        assert np.linalg.norm(K @ rigid) <= 1e-10 * scale * np.linalg.norm(rigid)


def _patch_solve(orc, model, field):
    """Prescribe `field` (node-major 6-vector per node) on boundary nodes of a
    3x3 patch and solve the interior node (index 4) with no load."""
    K = orc.assemble_dense(model)
    interior = np.arange(24, 30)
    boundary = np.setdiff1d(np.arange(54), interior)
    ub = field[boundary]
    ui = np.linalg.solve(K[np.ix_(interior, interior)], -K[np.ix_(interior, boundary)] @ ub)
    return ui


@pytest.mark.parametrize("distort", [0.0, 0.3])
def test_quad_membrane_patch(orc, distort):
    model = meshgen.patch_mesh(distort=distort, seed=3)
    X = model["xyz"]
    a = np.array([1e-3, 2e-3, -1.5e-3])
    b = np.array([-2e-3, 0.5e-3, 3e-3])
    field = np.zeros((9, 6))
    field[:, 0] = a[0] + a[1] * X[:, 0] + a[2] * X[:, 1]
    field[:, 1] = b[0] + b[1] * X[:, 0] + b[2] * X[:, 1]
    field[:, 5] = 0.5 * (b[1] - a[2])  # rz equal to the in-plane rotation
    ui = _patch_solve(orc, model, field.ravel())
    np.testing.assert_allclose(ui, field[4], rtol=0, atol=1e-12)


@pytest.mark.parametrize("distort", [0.0, 0.3])
def test_quad_bending_patch(orc, distort):
    """Constant curvature w = (a x^2 + 2 b x y + c y^2)/2 with zero shear
    (beta = -grad w, ry = beta_x, rx = -beta_y) is reproduced exactly."""
    model = meshgen.patch_mesh(distort=distort, seed=5)
    X = model["xyz"]
    a, b, c = 2e-3, -1e-3, 1.5e-3
    x, y = X[:, 0], X[:, 1]
    field = np.zeros((9, 6))
    field[:, 2] = 0.5 * (a * x ** 2 + 2 * b * x * y + c * y ** 2)
    beta_x = -(a * x + b * y)
    beta_y = -(b * x + c * y)
    field[:, 4] = beta_x
    field[:, 3] = -beta_y
    ui = _patch_solve(orc, model, field.ravel())
    np.testing.assert_allclose(ui, field[4], rtol=0, atol=1e-12)


@pytest.mark.parametrize("name", ["distorted", "warped"])
def test_quad_thickness_is_cubic(orc, name):
    """Membrane, shear and drilling scale with t, bending with t^3: K(t) = A t + B t^3.
    Fit A, B from two thicknesses, check a third and the dual-number dK/dt."""
    X = QUADS[name]

    def K_of(t):
        p = QPROPS.copy()
        p[0] = t
        return orc.quad_ke(X, p)

    t1, t2, t3 = 0.05, 0.2, 0.13
    K1, K2 = K_of(t1), K_of(t2)
    # K1 = A t1 + B t1^3, K2 = A t2 + B t2^3
    det = t1 * t2 ** 3 - t2 * t1 ** 3
    Bc = (t1 * K2 - t2 * K1) / det
    Ac = (K1 - Bc * t1 ** 3) / t1
    scale = np.abs(K2).max()
    np.testing.assert_allclose(K_of(t3), Ac * t3 + Bc * t3 ** 3, rtol=0, atol=1e-12 * scale)
    p = QPROPS.copy()
    p[0] = t3
    dK = orc.quad_dke(X, p, 12)
    np.testing.assert_allclose(dK, Ac + 3 * Bc * t3 ** 2, rtol=0, atol=1e-11 * scale / t3)


@pytest.mark.parametrize("which", [2, 5, 8, 11, 0, 7])
def test_quad_dke_matches_central_fd(orc, which):
    X = QUADS["warped"].copy()
    dK = orc.quad_dke(X, QPROPS, which)
    h = 1e-5

    def K_at(delta):
        Y = X.copy()
        Y.flat[which] += delta
        return orc.quad_ke(Y, QPROPS)

    fd = (K_at(h) - K_at(-h)) / (2 * h)
    fd2 = (K_at(h / 2) - K_at(-h / 2)) / h
    rich = (4 * fd2 - fd) / 3
    assert np.abs(dK - rich).max() <= 1e-6 * np.abs(dK).max()


@pytest.mark.parametrize("which", [2, 8, 6, 13, 16])
def test_beam_dke_matches_central_fd(orc, which):
    xi = np.array([0.1, 0.2, 0.3])
    xj = np.array([1.1, 0.7, 1.5])
    props = np.array([E, G, IY, IZ, J, A])
    dK = orc.beam_dke(xi, xj, props, which)
    h = 1e-6 * (1.0 if which < 12 else abs(props[which - 12]))

    def K_at(delta):
        a, b, p = xi.copy(), xj.copy(), props.copy()
        if which < 3:
            a[which] += delta
        elif which < 12:
            b[which - 6] += delta
        else:
            p[which - 12] += delta
        return orc.beam_ke(a, b, p)

    fd = (K_at(h) - K_at(-h)) / (2 * h)
    assert np.abs(dK - fd).max() <= 1e-6 * np.abs(dK).max()


def test_quad_load_partition_of_unity(orc):
    """Sum of the consistent nodal loads = -q * area; for a flat quad the area
    is the shoelace area of its corners."""
    X = QUADS["distorted"]
    q = 2500.0
    f = orc.quad_fe(X, q)
    x, y = X[:, 0], X[:, 1]
    shoelace = 0.5 * abs(np.dot(x, np.roll(y, -1)) - np.dot(y, np.roll(x, -1)))
    assert orc.quad_area(X) == pytest.approx(shoelace, rel=1e-14)
    assert f[2::6].sum() == pytest.approx(-q * shoelace, rel=1e-14)
    assert np.all(f[0::6] == 0) and np.all(f[3::6] == 0)


def test_quad_rotation_covariance(orc):
    """k_e of a rigidly rotated element is Q k_e Q^T (isotropic material)."""
    X = QUADS["warped"]
    K = orc.quad_ke(X, QPROPS)
    Q = _rot(11)
    Kr = orc.quad_ke(X @ Q.T + np.array([0.3, -1.0, 2.0]), QPROPS)
    T = np.kron(np.eye(8), Q)
    np.testing.assert_allclose(Kr, T @ K @ T.T, rtol=0, atol=1e-11 * np.abs(K).max())
