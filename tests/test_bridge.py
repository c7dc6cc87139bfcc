"""The beam-path scaling structure: a 100-span bridge of 30 m x 10 m
parabolic arches on pinned piers (Sec. 2.2.4).

CPU (oracle): the generator gives the paper's DOF counts, the oracle's
solution balances the loads, and the structure's mirror symmetry about its
middle pier holds (uz and the in-plane rotation mirror; the rotation at the
middle pier is zero).  GPU: FP64 CG against the oracle's band Cholesky for u,
C and dC/dz of every node."""
import numpy as np
import pytest

import meshgen


@pytest.mark.parametrize("k,dof", [(2, 1206), (6, 3606), (10, 6006), (20, 12006), (30, 18006),
                                   (80, 48006)])
def test_bridge_sizes_match_the_paper(k, dof):
    m = meshgen.arch_bridge(el_per_span=k)
    assert 6 * m["xyz"].shape[0] == dof
    assert m["beam_conn"].shape[0] == 100 * k
    piers = np.nonzero(m["fixed"].any(axis=1))[0]
    assert np.array_equal(piers, np.arange(0, 100 * k + 1, k))
    # self-weight: the loads add up to unit weight x area x arch length
    length = np.linalg.norm(np.diff(m["xyz"], axis=0), axis=1).sum()
    assert np.isclose(m["nodal_load"][:, 2].sum(), -7.85e4 * 4.3e-3 * length, rtol=1e-12)


def test_bridge_oracle_symmetry_and_equilibrium(orc):
    k = 4
    m = meshgen.arch_bridge(el_per_span=k)
    u = orc.solve(m)[0].reshape(-1, 6)
    n = u.shape[0]
    mid = n // 2  # the middle pier (node 200 of 401)
    assert mid % k == 0
    scale = np.abs(u[:, 2]).max()
    assert scale > 0
    # mirror about x = x_mid: uz(x_mid + d) = uz(x_mid - d), ux and ry flip sign
    assert np.abs(u[mid + 1:, 2] - u[mid - 1::-1, 2]).max() <= 1e-9 * scale
    assert np.abs(u[mid + 1:, 0] + u[mid - 1::-1, 0]).max() <= 1e-9 * np.abs(u[:, 0]).max()
    assert np.abs(u[mid + 1:, 4] + u[mid - 1::-1, 4]).max() <= 1e-9 * np.abs(u[:, 4]).max()
    assert abs(u[mid, 4]) <= 1e-9 * np.abs(u[:, 4]).max()
    # no out-of-plane response to in-plane loads
    assert np.abs(u[:, [1, 3, 5]]).max() <= 1e-12 * scale
    assert np.linalg.norm(orc.residual(m, u.ravel())) <= 1e-9 * np.linalg.norm(orc.load_vector(m))


@pytest.mark.gpu
@pytest.mark.parametrize("k", [2, 6])
def test_bridge_gpu_fp64_matches_oracle(orc, k):
    from paper_2407_20026_gb300 import _build
    _build.build()
    import paper_2407_20026_gb300 as sso
    m = meshgen.arch_bridge(el_per_span=k)
    ref = orc.gradient(m, w=1.0)
    mdl = sso.Model(m)
    st = mdl.solve(sso.options(precision="fp64", precond="block_jacobi", rtol=1e-12,
                               max_iter=200_000))
    assert st["status"] == 0
    mdl.gradient()
    r = mdl.result()
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel(r["u"], ref["u"]) <= 1e-8
    assert abs(r["C"] - ref["C"]) <= 1e-8 * abs(ref["C"])
    assert rel(r["dz"], ref["dz"]) <= 1e-8


def _chain_opts(sso, **kw):
    return sso.options(precision="fp64", precond="chain", rtol=1e-12, **kw)


@pytest.mark.gpu
@pytest.mark.parametrize("k", [2, 6, 31])
def test_chain_direct_solve_matches_oracle(orc, k):
    # block cyclic reduction on the bridge (levels of odd and even node counts)
    from paper_2407_20026_gb300 import _build
    _build.build()
    import paper_2407_20026_gb300 as sso
    m = meshgen.arch_bridge(el_per_span=k, n_spans=7)
    ref = orc.gradient(m, w=1.0)
    mdl = sso.Model(m)
    st = mdl.solve(_chain_opts(sso))
    assert st["status"] == 0 and st["iterations"] == 0 and st["rel_residual"] <= 1e-12
    mdl.gradient()
    r = mdl.result()
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel(r["u"], ref["u"]) <= 1e-10
    assert abs(r["C"] - ref["C"]) <= 1e-10 * abs(ref["C"])
    assert rel(r["dz"], ref["dz"]) <= 1e-10


@pytest.mark.gpu
def test_chain_general_objective_and_batch(orc):
    # J = 0.3 C + g^T u needs a real adjoint solve through the same factors;
    # a batch of two chains of different length gives the solo results bit for bit
    from paper_2407_20026_gb300 import _build
    _build.build()
    import paper_2407_20026_gb300 as sso
    m1 = meshgen.arch_bridge(el_per_span=5, n_spans=9)
    m2 = meshgen.arch_bridge(el_per_span=3, n_spans=4)
    g = np.random.default_rng(3).standard_normal(6 * m1["xyz"].shape[0])
    g[m1["fixed"].ravel().astype(bool)] = 0.0
    ref = orc.gradient(m1, w=0.3, g=g)
    solo = sso.Model(m1)
    solo.solve(_chain_opts(sso))
    solo.gradient(0.3, g)
    r = solo.result()
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel(r["dz"], ref["dz"]) <= 1e-9
    a, b = sso.Model(m1), sso.Model(m2)
    batch = sso.Batch([a, b])
    batch.solve(_chain_opts(sso))
    batch.gradient([0.3, 1.0], [g, None])
    ra = a.result()
    for key in ("u", "dz"):
        assert np.array_equal(ra[key], r[key])
    assert ra["C"] == r["C"]


@pytest.mark.gpu
def test_chain_rejects_other_patterns_and_precisions(orc):
    from paper_2407_20026_gb300 import _build
    _build.build()
    import paper_2407_20026_gb300 as sso
    mdl = sso.Model(meshgen.gridshell(n_side=5, seed=1))
    with pytest.raises(Exception):
        mdl.solve(_chain_opts(sso))
    br = sso.Model(meshgen.arch_bridge(el_per_span=2, n_spans=3))
    with pytest.raises(Exception):
        br.solve(sso.options(precision="fp32_ir", precond="chain"))
    st = br.solve(_chain_opts(sso))
    assert st["status"] == 0


@pytest.mark.gpu
def test_chain_direct_solve_at_120k_dof(orc):
    # 200 elements per span (120,006 DOF): the GPU solution has the residual
    # floor of the oracle's FP64 band Cholesky and the same compliance
    from paper_2407_20026_gb300 import _build
    _build.build()
    import paper_2407_20026_gb300 as sso
    m = meshgen.arch_bridge(el_per_span=200)
    u_o, C_o = orc.solve(m)
    f = orc.load_vector(m)
    f[m["fixed"].ravel().astype(bool)] = 0.0
    res_o = np.linalg.norm(orc.residual(m, u_o)) / np.linalg.norm(f)
    mdl = sso.Model(m)
    st = mdl.solve(_chain_opts(sso, max_sweeps=3), raise_on_error=False)
    r = mdl.result()
    res_g = np.linalg.norm(orc.residual(m, r["u"])) / np.linalg.norm(f)
    assert res_g <= max(10 * res_o, 1e-12), (res_g, res_o)
    assert abs(st["rel_residual"] - res_g) <= 0.5 * res_g + 1e-15
    assert abs(r["C"] - C_o) <= 1e-9 * abs(C_o)
    assert np.linalg.norm(r["u"] - u_o) / np.linalg.norm(u_o) <= 1e-7
