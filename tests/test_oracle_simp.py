"""Pins of the oracle's SIMP topology sensitivity (Eq. simp_eq, E_j = p_j^P E*_j):
the modulus derivative of the stiffness term of Eq. 6 against Euler's theorem
(k_e is homogeneous of degree 1 in E, so dk_e/dE = k_e / E), and dC/dp against
central differences of the compliance."""
import numpy as np
import pytest

import meshgen


def _shell():
    m = meshgen.shell(n_el=4, span=6.0, seed=2, height=1.2)
    m["pressure"] = 3e3
    return m


def test_modulus_derivative_is_k_over_E(orc):
    m = _shell()
    r = orc.gradient(m, w=0.7)
    dE = orc.adjoint_contract_E(m, r["u"], r["lam"])
    u, lam = r["u"], r["lam"]
    ref = np.zeros_like(dE)
    for e, nodes in enumerate(m["quad_conn"]):
        X = m["xyz"][nodes]
        ke = orc.quad_ke(X, m["quad_props"][e])
        dofs = (6 * nodes[:, None] + np.arange(6)).ravel()
        ref[e] = -lam[dofs] @ ke @ u[dofs] / m["quad_props"][e, 1]
    np.testing.assert_allclose(dE, ref, rtol=1e-11, atol=1e-14 * np.abs(ref).max())


def test_density_gradient_matches_central_differences(orc):
    m = _shell()
    rng = np.random.default_rng(0)
    rho = rng.uniform(0.3, 1.0, m["quad_conn"].shape[0])
    penal = 3.0
    r = orc.simp_gradient(m, rho, penal)
    def C(rr):
        return orc.gradient(orc.simp_model(m, rr, penal))["C"]

    def fd(j, h):
        rp, rm = rho.copy(), rho.copy()
        rp[j] += h
        rm[j] -= h
        return (C(rp) - C(rm)) / (2 * h)

    # Richardson: truncation O(h^4); round-off ~ (solve error of C) / h, about
    # 1e-4 absolute here, so the check is norm-wise over the sampled entries
    js = [0, 5, 11, 14]
    d = np.array([(4 * fd(j, 1e-4) - fd(j, 2e-4)) / 3 for j in js])
    g = r["drho"][js]
    assert np.linalg.norm(g - d) <= 1e-7 * np.linalg.norm(d)


def test_unit_density_is_the_plain_model(orc):
    m = _shell()
    rho = np.ones(m["quad_conn"].shape[0])
    a = orc.simp_gradient(m, rho, 3.0)
    b = orc.gradient(m)
    assert np.array_equal(a["u"], b["u"])
    assert a["C"] == b["C"]
