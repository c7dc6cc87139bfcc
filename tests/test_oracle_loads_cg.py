"""Pins of the oracle's consistent area loads and of its FP64 CG.

Consistent area load (reading C-load of the configurations' "self-weight" and
"pressure"): f_i = -e_Z q * integral of N_i dA over the element's flat facet.
For a bilinear facet the Jacobian determinant is exactly linear in the
parent coordinates, detJ = j0 + j1 xi + j2 eta, so

    integral N_i dA = j0 + (xi_i j1 + eta_i j2) / 3,     j0 = area / 4,

with (xi_i, eta_i) the parent corner of node i.  The tests below derive j0, j1,
j2 from the corner coordinates in their own code and compare each node's load,
on a trapezoid, a general distorted quad, a tilted planar quad and a warped
quad (whose facet is its projection on the plane normal to the cross product
of its diagonals).  A quarter ("lumped") split or a shape function paired with
the wrong corner fails them: each case asserts that it would.

CG: the oracle's Jacobi-preconditioned CG (the oracle of the 512 x 512 shell,
too large for the band Cholesky) is compared with the band Cholesky solve on
small models and on a 24 x 24 shell.
"""
import numpy as np
import pytest

import meshgen

# Parent corners of a CCW quad (node k of the connectivity), the standard
# bilinear isoparametric ordering.
XI = np.array([-1.0, 1.0, 1.0, -1.0])
ETA = np.array([-1.0, -1.0, 1.0, 1.0])


def _closed_form_shares(P2):
    """integral of N_i dA for the bilinear map of 2D corners P2 [4, 2]."""
    x, y = P2[:, 0], P2[:, 1]
    # x(xi, eta) = a0 + a1 xi + a2 eta + a3 xi eta (and y with b)
    a1, a2, a3 = (XI @ x) / 4, (ETA @ x) / 4, (XI * ETA @ x) / 4
    b1, b2, b3 = (XI @ y) / 4, (ETA @ y) / 4, (XI * ETA @ y) / 4
    j0 = a1 * b2 - a2 * b1
    j1 = a1 * b3 - a3 * b1
    j2 = a3 * b2 - a2 * b3
    return j0 + (XI * j1 + ETA * j2) / 3.0, 4.0 * j0


def _facet_coordinates(X):
    """2D coordinates of the corners projected on the plane normal to d13 x d24
    (any right-handed in-plane basis: the shares do not depend on it)."""
    n = np.cross(X[2] - X[0], X[3] - X[1])
    n /= np.linalg.norm(n)
    e1 = np.cross([0.3, 0.5, 0.8], n)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(n, e1)
    return np.stack([X @ e1, X @ e2], axis=1)


def _rotation(seed):
    q, r = np.linalg.qr(np.random.default_rng(seed).normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def _planar(P2, seed=None, shift=(0.0, 0.0, 0.0)):
    X = np.concatenate([P2, np.zeros((4, 1))], axis=1)
    if seed is not None:
        X = X @ _rotation(seed).T
    return X + np.asarray(shift)


TRAPEZOID = np.array([[0.0, 0.0], [2.0, 0.0], [1.4, 1.0], [0.3, 1.0]])
DISTORTED = np.array([[0.0, 0.0], [1.3, 0.1], [1.1, 0.9], [-0.2, 1.2]])
CASES = {
    "trapezoid": _planar(TRAPEZOID),
    "distorted": _planar(DISTORTED),
    "tilted": _planar(DISTORTED, seed=7, shift=(0.4, -1.0, 2.0)),
    "warped": np.array([[0, 0, 0.05], [1.2, 0.1, -0.08], [1.1, 1.0, 0.12], [0.1, 0.9, -0.02]]),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_quad_load_equals_bilinear_closed_form(orc, name):
    X = CASES[name]
    q = 2500.0
    shares, area = _closed_form_shares(_facet_coordinates(X))
    assert area > 0
    f = orc.quad_fe(X, q)
    expect = -q * shares
    np.testing.assert_allclose(f[2::6], expect, rtol=0, atol=1e-13 * q * area)
    for k in (0, 1, 3, 4, 5):
        assert np.all(f[k::6] == 0.0)
    assert orc.quad_area(X) == pytest.approx(area, rel=1e-13)
    # the pin discriminates: a lumped quarter split, or the shares of a cyclic
    # relabelling of the corners (a shape function on the wrong node), miss it
    assert np.abs(expect + q * area / 4).max() > 1e-3 * q * area
    assert np.abs(expect - np.roll(expect, 1)).max() > 1e-3 * q * area


def test_model_load_vector_sums_element_shares(orc):
    """The model's load vector is the sum of its elements' closed-form shares
    (area loads from self-weight gamma * t_e and pressure) plus nodal loads."""
    m = meshgen.shell(n_el=3, span=4.0, seed=3, height=1.0)
    m["pressure"] = 1.5e3
    m["nodal_load"][6, 1] = 40.0
    X = np.asarray(m["xyz"])
    expect = np.array(m["nodal_load"], dtype=np.float64).reshape(-1).copy()
    for e, conn in enumerate(np.asarray(m["quad_conn"])):
        q = m["pressure"] + m["gamma"] * m["quad_props"][e, 0]
        shares, _ = _closed_form_shares(_facet_coordinates(X[conn]))
        expect[6 * conn + 2] -= q * shares
    f = orc.load_vector(m)
    np.testing.assert_allclose(f, expect, rtol=0, atol=1e-12 * np.abs(expect).max())


def _cg_models():
    strip = meshgen.shell(n_el=3, span=4.0, seed=1, height=1.0)
    strip["pressure"] = 3e3
    return {
        "gridshell10": meshgen.gridshell(),
        "shell3": strip,
        "shell24": meshgen.shell(n_el=24, seed=5),
    }


@pytest.mark.parametrize("name", ["gridshell10", "shell3", "shell24"])
def test_cg_equals_band_cholesky(orc, name):
    m = _cg_models()[name]
    u_chol, C = orc.solve(m)
    u_cg, iters = orc.cg(m, rtol=1e-13, max_iter=200000)
    assert iters > 0
    rel = np.linalg.norm(u_cg - u_chol) / np.linalg.norm(u_chol)
    assert rel <= 1e-10, (rel, iters)
    fixed = np.asarray(m["fixed"]).reshape(-1).astype(bool)
    assert np.all(u_cg[fixed] == 0.0)
    f = orc.load_vector(m)
    f[fixed] = 0.0

    def true_residual(u):
        r = orc.residual(m, u)
        r[fixed] = 0.0
        return np.linalg.norm(r) / np.linalg.norm(f)

    # the recursive residual stopped at 1e-13; the true one lies on the same
    # rounding floor (about eps * cond(K)) as the backward-stable Cholesky's
    assert true_residual(u_cg) <= 10 * true_residual(u_chol) + 1e-13
