"""CUDA path (through the C-ABI) vs the FP64 oracle.

Elements element by element; assembled K entry by entry (FP64 vs oracle, FP32
bit-exact rounding of FP64, bit-reproducible); loads; solves and adjoint
gradients in FP64 mode (1e-8) and FP32 + FP64 refinement (1e-6) on beam,
shell and mixed models whose node counts are not multiples of the tile.
"""
import numpy as np
import pytest
import torch

import meshgen
from gpu_util import (TOL_ELEMENT, TOL_FP32_IR, TOL_FP64, bsr_to_dense, hub_model, mixed_model,
                      permuted, rel, small_shell, with_supports)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sso():
    import paper_2407_20026_gb300 as pkg
    from paper_2407_20026_gb300 import _build
    _build.build()
    assert torch.cuda.is_available()
    return pkg


def _rand_quads(n, seed):
    rng = np.random.default_rng(seed)
    base = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0]], float)
    X = np.empty((n, 4, 3))
    for e in range(n):
        Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        P = base * rng.uniform(0.3, 3.0, 3) + rng.uniform(-0.15, 0.15, (4, 3)) * [1, 1, 0]
        P[:, 2] += rng.uniform(-0.08, 0.08, 4)  # warp
        X[e] = P @ Q.T + rng.normal(size=3) * 5
    props = np.stack([rng.uniform(0.05, 0.3, n), rng.uniform(1e9, 2e11, n),
                      rng.uniform(0.0, 0.45, n), rng.uniform(0.5, 2.0, n),
                      rng.uniform(0.5, 2.0, n)], 1)
    return X, props


def test_quad_element_matrices(sso, orc):
    X, props = _rand_quads(300, 7)
    xyz = torch.tensor(X.reshape(-1, 3), device="cuda")
    conn = torch.arange(4 * len(X), dtype=torch.int32, device="cuda").reshape(-1, 4)
    ke = sso.quad_stiffness(xyz, conn, torch.tensor(props, device="cuda")).cpu().numpy()
    for e in range(len(X)):
        ref = orc.quad_ke(X[e], props[e])
        got = ke[e].transpose(0, 2, 1, 3).reshape(24, 24)
        assert np.abs(got - ref).max() <= TOL_ELEMENT * np.abs(ref).max(), e


def test_beam_element_matrices(sso, orc):
    rng = np.random.default_rng(3)
    n = 300
    xi = rng.normal(size=(n, 3)) * 3
    d = rng.normal(size=(n, 3))
    d[:10, :2] = 0.0  # vertical members take the e_Y branch
    xj = xi + d * rng.uniform(0.2, 4.0, (n, 1))
    props = np.stack([rng.uniform(1e10, 3e11, n), rng.uniform(1e10, 1e11, n),
                      rng.uniform(1e-6, 1e-4, n), rng.uniform(1e-6, 1e-4, n),
                      rng.uniform(1e-6, 1e-4, n), rng.uniform(1e-4, 1e-2, n)], 1)
    xyz = torch.tensor(np.stack([xi, xj], 1).reshape(-1, 3), device="cuda")
    conn = torch.arange(2 * n, dtype=torch.int32, device="cuda").reshape(-1, 2)
    ke = sso.beam_stiffness(xyz, conn, torch.tensor(props, device="cuda")).cpu().numpy()
    for e in range(n):
        ref = orc.beam_ke(xi[e], xj[e], props[e])
        got = ke[e].transpose(0, 2, 1, 3).reshape(12, 12)
        assert np.abs(got - ref).max() <= TOL_ELEMENT * np.abs(ref).max(), e


MODELS = {
    "gridshell10": lambda: meshgen.gridshell(),
    "gridshell13": lambda: meshgen.gridshell(n_side=13, seed=5),
    "shell5": lambda: small_shell(5),
    "shell9_clamped": lambda: meshgen.shell(n_el=9, span=8.0, supports="clamped",
                                            load="pressure", seed=4),
    "mixed": lambda: mixed_model(5),
    "hub": lambda: hub_model(),
}


@pytest.mark.parametrize("name", sorted(MODELS))
def test_assembled_stiffness_and_loads(sso, orc, name):
    m = MODELS[name]()
    mdl = sso.Model(m)
    mdl.solve(precision="fp64")
    rp, col, K64, K32 = mdl.stiffness()
    Kg = bsr_to_dense(rp, col, K64)
    Ko = with_supports(orc.assemble_dense(m), m["fixed"])
    assert np.abs(Kg - Ko).max() <= 1e-12 * np.abs(Ko).max()
    # K32 is exactly the round-to-nearest of K64
    assert np.array_equal(K32, K64.astype(np.float32))
    # assembly is bit-reproducible
    mdl.solve(precision="fp64")
    _, _, K64b, _ = mdl.stiffness()
    assert np.array_equal(K64, K64b)
    fo = orc.load_vector(m)
    fo[m["fixed"].ravel().astype(bool)] = 0.0
    np.testing.assert_allclose(mdl.load_vector(), fo, rtol=0, atol=1e-12 * np.abs(fo).max())


@pytest.mark.parametrize("precision,tol", [("fp64", TOL_FP64), ("fp32_ir", TOL_FP32_IR)])
@pytest.mark.parametrize("name", sorted(MODELS))
def test_solve_and_gradient(sso, orc, name, precision, tol):
    m = MODELS[name]()
    ref = orc.gradient(m, w=1.0)
    mdl = sso.Model(m)
    rtol = 1e-10 if precision == "fp64" else 1e-9
    st = mdl.solve(precision=precision, rtol=rtol)
    assert st["status"] == 0 and st["rel_residual"] <= rtol
    mdl.gradient(1.0)
    r = mdl.result()
    assert rel(r["u"], ref["u"]) <= tol
    assert abs(r["C"] - ref["C"]) <= tol * abs(ref["C"])
    assert rel(r["dz"], ref["dz"]) <= tol
    if m["quad_conn"].shape[0]:
        assert rel(r["dt"], ref["dt"]) <= tol
    assert np.all(r["u"][m["fixed"].ravel().astype(bool)] == 0.0)


@pytest.mark.parametrize("name", ["gridshell10", "mixed"])
def test_general_objective_adjoint(sso, orc, name):
    """J = w C + g^T u: a real adjoint solve K lambda = w f + g (Eq. 5)."""
    m = MODELS[name]()
    rng = np.random.default_rng(11)
    g = rng.normal(size=6 * m["xyz"].shape[0]) * 1e3
    ref = orc.gradient(m, w=0.5, g=g)
    mdl = sso.Model(m)
    mdl.solve(precision="fp64", rtol=1e-11)
    st = mdl.gradient(0.5, g)
    assert st["status"] == 0
    r = mdl.result()
    free = ~m["fixed"].ravel().astype(bool)
    assert rel(r["lam"][free], ref["lam"][free]) <= TOL_FP64
    assert rel(r["dz"], ref["dz"]) <= TOL_FP64
    if m["quad_conn"].shape[0]:
        assert rel(r["dt"], ref["dt"]) <= TOL_FP64


def test_jacobi_preconditioner(sso, orc):
    m = small_shell(5)
    ref = orc.gradient(m)
    mdl = sso.Model(m)
    st = mdl.solve(precision="fp32_ir", precond="jacobi", rtol=1e-9)
    assert st["status"] == 0
    mdl.gradient(1.0)
    r = mdl.result()
    assert rel(r["u"], ref["u"]) <= TOL_FP32_IR
    assert rel(r["dz"], ref["dz"]) <= TOL_FP32_IR


def test_batch_equals_alone_bitwise(sso):
    """Each system's result is bit-identical alone and inside a mixed batch."""
    ms = [MODELS[k]() for k in ("gridshell13", "shell5", "mixed", "gridshell10")]
    alone = []
    for m in ms:
        mdl = sso.Model(m)
        mdl.solve(precision="fp32_ir", rtol=1e-9)
        mdl.gradient(1.0)
        alone.append(mdl.result())
    models = [sso.Model(m) for m in ms]
    batch = sso.Batch(models)
    stats = batch.solve(precision="fp32_ir", rtol=1e-9)
    assert all(s["status"] == 0 for s in stats)
    batch.gradient()
    for mdl, a in zip(models, alone):
        r = mdl.result()
        for k in ("u", "dz", "dt"):
            assert np.array_equal(r[k], a[k]), k
        assert r["C"] == a["C"]


def test_set_design_matches_fresh_model(sso, orc):
    m = small_shell(5)
    mdl = sso.Model(m)
    mdl.solve(precision="fp64")
    rng = np.random.default_rng(2)
    z = m["xyz"][:, 2] + rng.uniform(-0.1, 0.1, m["xyz"].shape[0])
    t = m["quad_props"][:, 0] * rng.uniform(0.8, 1.2, m["quad_props"].shape[0])
    mdl.set_design(torch.tensor(z, device="cuda"), t)
    mdl.solve(precision="fp64", rtol=1e-11)
    mdl.gradient(1.0)
    m2 = dict(m)
    m2["xyz"] = m["xyz"].copy()
    m2["xyz"][:, 2] = z
    m2["quad_props"] = m["quad_props"].copy()
    m2["quad_props"][:, 0] = t
    ref = orc.gradient(m2)
    r = mdl.result()
    assert rel(r["u"], ref["u"]) <= TOL_FP64
    assert rel(r["dt"], ref["dt"]) <= TOL_FP64


def test_warm_start_converges_in_fewer_iterations(sso):
    m = small_shell(7)
    mdl = sso.Model(m)
    a = mdl.solve(precision="fp32_ir", rtol=1e-9)
    z = m["xyz"][:, 2] * 1.001
    mdl.set_design(z, None)
    cold = sso.Model(m)
    cold.set_design(z, None)
    c = cold.solve(precision="fp32_ir", rtol=1e-9)
    w = mdl.solve(precision="fp32_ir", rtol=1e-9, warm_start=1)
    assert w["status"] == 0 and a["status"] == 0
    assert w["iterations"] < c["iterations"]
    assert rel(mdl.result()["u"], cold.result()["u"]) <= 1e-7


def test_zero_load_and_edge_cases(sso):
    m = small_shell(3)
    m["pressure"] = 0.0
    m["gamma"] = 0.0
    m["nodal_load"][:] = 0.0
    mdl = sso.Model(m)
    st = mdl.solve()
    assert st["status"] == 0 and st["iterations"] == 0
    r = mdl.result()
    assert np.all(r["u"] == 0.0) and r["C"] == 0.0


def test_iteration_cap_reports_not_converged(sso):
    mdl = sso.Model(small_shell(6))
    with pytest.raises(sso.SSOError) as ei:
        mdl.solve(max_iter=5, rtol=1e-12)
    assert ei.value.status == 4


def test_mechanism_reports_error(sso):
    """No supports: K is singular (6 rigid modes); the solve must not report OK."""
    m = small_shell(3)
    m["fixed"][:] = 0
    mdl = sso.Model(m)
    with pytest.raises(sso.SSOError) as ei:
        mdl.solve(max_iter=3000, rtol=1e-12)
    assert ei.value.status in (3, 4)


def test_autograd_function(sso, orc):
    from paper_2407_20026_gb300.autograd import SSOFunction
    m = small_shell(5)
    mdl = sso.Model(m)
    z = torch.tensor(m["xyz"][:, 2], device="cuda", requires_grad=True)
    t = torch.tensor(m["quad_props"][:, 0], device="cuda", requires_grad=True)
    u, C, V = SSOFunction.apply(mdl, z, t, sso.options(precision="fp64", rtol=1e-11))
    rng = np.random.default_rng(5)
    gvec = torch.tensor(rng.normal(size=u.shape[0]), device="cuda")
    J = 0.7 * C + (gvec * u).sum() + 0.3 * V
    J.backward()
    ref = orc.gradient(m, w=0.7, g=gvec.cpu().numpy())
    vol = orc.volume(m)
    assert abs(float(V.detach()) - vol["V"]) <= TOL_ELEMENT * vol["V"]
    assert rel(z.grad.cpu().numpy(), ref["dz"] + 0.3 * vol["dz"]) <= TOL_FP64
    assert rel(t.grad.cpu().numpy(), ref["dt"] + 0.3 * vol["dt"]) <= TOL_FP64


@pytest.mark.parametrize("name", ["shell5", "mixed", "gridshell13", "shell9_clamped"])
def test_two_level_preconditioner_parity(sso, orc, name):
    """Block-Jacobi plus the rigid-body coarse correction: the same solution
    and gradient as the oracle (the preconditioner changes only the path)."""
    m = MODELS[name]()
    ref = orc.gradient(m)
    mdl = sso.Model(m)
    st = mdl.solve(precision="fp32_ir", precond="two_level", rtol=1e-9)
    assert st["status"] == 0 and st["rel_residual"] <= 1e-9
    mdl.gradient(1.0)
    r = mdl.result()
    assert rel(r["u"], ref["u"]) <= TOL_FP32_IR
    assert abs(r["C"] - ref["C"]) <= TOL_FP32_IR * abs(ref["C"])
    assert rel(r["dz"], ref["dz"]) <= TOL_FP32_IR


def test_two_level_cuts_iterations(sso, orc):
    m = meshgen.shell(n_el=24, span=20.0, seed=1)
    its = {}
    for pc in ("block_jacobi", "two_level"):
        mdl = sso.Model(m)
        st = mdl.solve(precision="fp32_ir", precond=pc, rtol=1e-8)
        assert st["status"] == 0
        its[pc] = st["iterations"]
    assert its["two_level"] * 3 < its["block_jacobi"], its
    ref = orc.gradient(m)
    assert rel(mdl.result()["u"], ref["u"]) <= TOL_FP32_IR


def test_two_level_batch_equals_alone_bitwise(sso):
    meshes = [small_shell(5), meshgen.gridshell(n_side=12, seed=2), meshgen.shell(n_el=7, seed=3)]
    opts = sso.options(precision="fp32_ir", precond="two_level", rtol=1e-8)
    alone = []
    for m in meshes:
        mdl = sso.Model(m)
        mdl.solve(opts)
        alone.append(mdl.result()["u"])
    batch = sso.Batch([sso.Model(m) for m in meshes])
    batch.solve(opts)
    for a, mdl in zip(alone, batch.models):
        assert np.array_equal(a, mdl.result()["u"])


def test_two_level_needs_fp32_ir(sso):
    mdl = sso.Model(small_shell(4))
    with pytest.raises(sso.SSOError):
        mdl.solve(precision="fp64", precond="two_level")


@pytest.mark.parametrize("precision,tol", [("fp64", TOL_FP64), ("fp32_ir", TOL_FP32_IR)])
@pytest.mark.parametrize("name", ["shell5", "mixed"])
def test_simp_topology_gradient(sso, orc, name, precision, tol):
    """SIMP densities (Eq. simp_eq, P = 3): u, C, dC/dz, dC/dt and dC/drho vs
    the oracle on the same densities; then densities removed again."""
    m = MODELS[name]()
    nq = m["quad_conn"].shape[0]
    rho = np.random.default_rng(4).uniform(0.3, 1.0, nq)
    ref = orc.simp_gradient(m, rho, 3.0)
    mdl = sso.Model(m)
    mdl.set_topology(rho, 3.0)
    rtol = 1e-10 if precision == "fp64" else 1e-9
    st = mdl.solve(precision=precision, rtol=rtol)
    assert st["status"] == 0
    mdl.gradient(1.0)
    r = mdl.result()
    assert rel(r["u"], ref["u"]) <= tol
    assert abs(r["C"] - ref["C"]) <= tol * abs(ref["C"])
    assert rel(r["dz"], ref["dz"]) <= tol
    assert rel(r["dt"], ref["dt"]) <= tol
    assert rel(mdl.topology_gradient(), ref["drho"]) <= tol
    mdl.set_topology(None)
    mdl.solve(precision=precision, rtol=rtol)
    plain = orc.gradient(m)
    assert rel(mdl.result()["u"], plain["u"]) <= tol


def test_simp_rejects_bad_densities(sso):
    mdl = sso.Model(small_shell(4))
    nq = mdl.n_quads
    with pytest.raises(sso.SSOError):
        mdl.set_topology(np.zeros(nq), 3.0)
    with pytest.raises(sso.SSOError):
        mdl.set_topology(np.ones(nq), 0.5)


@pytest.mark.parametrize("name", ["shell5", "shell9_clamped", "mixed", "gridshell13"])
def test_material_volume(sso, orc, name):
    """W = sum A_e t_e and its z, t gradients vs the oracle (element-level
    tolerance: same formulas, different operation order)."""
    m = MODELS[name]()
    r = sso.Model(m).volume()
    ref = orc.volume(m)
    if m["quad_conn"].shape[0] == 0:
        assert r["V"] == 0.0 and not np.any(r["dz"])
        return
    assert abs(r["V"] - ref["V"]) <= TOL_ELEMENT * ref["V"]
    assert rel(r["dz"], ref["dz"]) <= 1e-10
    assert rel(r["dt"], ref["dt"]) <= TOL_ELEMENT


def test_batched_autograd_with_volume(sso, orc):
    """The batched function's gradient of sum_i (C_i + 0.1 V_i) over three
    designs of one mesh vs the oracle, FP32 CG with refinement."""
    from paper_2407_20026_gb300.autograd import BatchSSOFunction
    meshes = [meshgen.shell(n_el=6, span=8.0, seed=s, thickness=0.1) for s in range(3)]
    batch = sso.Batch([sso.Model(m) for m in meshes])
    z = torch.tensor(np.stack([m["xyz"][:, 2] for m in meshes]), device="cuda",
                     requires_grad=True)
    t = torch.tensor(np.stack([m["quad_props"][:, 0] for m in meshes]), device="cuda",
                     requires_grad=True)
    u, C, V = BatchSSOFunction.apply(batch, z, t, sso.options(rtol=1e-10))
    (C + 0.1 * V).sum().backward()
    for i, m in enumerate(meshes):
        ref = orc.gradient(m)
        vol = orc.volume(m)
        assert abs(float(C[i].detach()) - ref["C"]) <= TOL_FP32_IR * abs(ref["C"])
        assert rel(z.grad[i].cpu().numpy(), ref["dz"] + 0.1 * vol["dz"]) <= TOL_FP32_IR
        assert rel(t.grad[i].cpu().numpy(), ref["dt"] + 0.1 * vol["dt"]) <= TOL_FP32_IR


@pytest.mark.parametrize("name", ["gridshell13", "c1"])
def test_bsr_spmv_entry_point(sso, name):
    """y = K x and x^T y of the assembled K vs a plain FP64 product; the
    fixed-order dot is bit-identical across calls."""
    m = meshgen.shell(64) if name == "c1" else MODELS[name]()
    mdl = sso.Model(m)
    try:
        mdl.solve(precision="fp64", max_iter=10)
    except sso.SSOError:
        pass  # only the assembled K is needed
    rp, col, K64, _ = mdl.stiffness()
    rng = np.random.default_rng(4)
    x = rng.normal(size=6 * mdl.n_nodes)
    n = mdl.n_nodes
    y_ref = np.zeros(6 * n)
    for i in range(n):
        for k in range(rp[i], rp[i + 1]):
            y_ref[6 * i:6 * i + 6] += K64[k] @ x[6 * col[k]:6 * col[k] + 6]
    dev = "cuda"
    args = (torch.tensor(rp, device=dev), torch.tensor(col, device=dev),
            torch.tensor(K64, device=dev), torch.tensor(x, device=dev))
    y1, d1 = sso.bsr_spmv(*args)
    y2, d2 = sso.bsr_spmv(*args)
    torch.cuda.synchronize()
    y1 = y1.cpu().numpy()
    assert np.abs(y1 - y_ref).max() <= 1e-13 * np.abs(y_ref).max()
    assert float(d1) == pytest.approx(float(x @ y_ref), rel=1e-12)
    assert np.array_equal(y1, y2.cpu().numpy()) and float(d1) == float(d2)


def test_scattered_numbering_fallback_path(sso, orc):
    """Random node numbering: tile halos span the mesh, so the FP32 kernel
    reads z and p from global memory instead of shared-memory halos."""
    m = meshgen.shell(n_el=20, span=10.0, seed=6)
    ref = orc.gradient(m)
    mp, perm = permuted(m, np.random.default_rng(3).permutation(m["xyz"].shape[0]))
    mdl = sso.Model(mp)
    st = mdl.solve(precision="fp32_ir", rtol=1e-9)
    assert st["status"] == 0
    mdl.gradient(1.0)
    r = mdl.result()
    u = r["u"].reshape(-1, 6)[perm].ravel()
    assert rel(u, ref["u"]) <= TOL_FP32_IR
    assert rel(r["dz"][perm], ref["dz"]) <= TOL_FP32_IR
    assert rel(r["dt"], ref["dt"]) <= TOL_FP32_IR


def _oracle_gradients(orc, meshes, w=1.0, gs=None):
    """Oracle results of several models, computed in threads (the oracle is a
    C library called through ctypes, which releases the GIL)."""
    import concurrent.futures
    gs = gs if gs is not None else [None] * len(meshes)
    with concurrent.futures.ThreadPoolExecutor(len(meshes)) as ex:
        return list(ex.map(lambda mg: orc.gradient(mg[0], w=w, g=mg[1]), zip(meshes, gs)))


BENCH_SEEDS = [0, 1, 2, 3, 295]
_BENCH_REFS = []  # the oracle's gradients of the BENCH_SEEDS designs, computed once


@pytest.mark.parametrize("inner_rtol", [2e-3, 1e-3])
def test_bench_configuration_against_oracle(sso, orc, inner_rtol):
    """The bench's exact configuration -- 64 x 64 shell designs in one batch,
    FP32 block-Jacobi CG inside FP64 refinement to rtol 1e-6 with inner
    tolerance 2e-3 (the default; and 1e-3), 32 iterations per graph launch --
    against the oracle at the FP32+IR tolerance.  Seed 295 is the design whose
    refinement sweep stalls at an inner tolerance of 1e-3: the solve must
    tighten its later sweeps and still land within the tolerance."""
    meshes = [meshgen.shell(n_el=64, seed=s) for s in BENCH_SEEDS]
    batch = sso.Batch([sso.Model(m) for m in meshes])
    opts = sso.options(precision="fp32_ir", precond="block_jacobi", rtol=1e-6,
                       inner_rtol=inner_rtol, iters_per_launch=32)
    stats = batch.solve(opts, raise_on_error=False)
    batch.gradient()
    if not _BENCH_REFS:
        _BENCH_REFS.extend(_oracle_gradients(orc, meshes))
    for s, st, mdl, ref in zip(BENCH_SEEDS, stats, batch.models, _BENCH_REFS):
        assert st["status"] == 0 and st["rel_residual"] <= 1e-6, (s, st)
        r = mdl.result()
        assert rel(r["u"], ref["u"]) <= TOL_FP32_IR, s
        assert abs(r["C"] - ref["C"]) <= TOL_FP32_IR * abs(ref["C"]), s
        assert rel(r["dz"], ref["dz"]) <= TOL_FP32_IR, s
        assert rel(r["dt"], ref["dt"]) <= TOL_FP32_IR, s


@pytest.mark.parametrize("name", ["shell5", "mixed", "gridshell13"])
def test_general_objective_adjoint_fp32_ir(sso, orc, name):
    """J = w C + g^T u with the adjoint solve K lambda = w f + g (Eq. 5) taken by
    the FP32 CG inside FP64 refinement, against the oracle."""
    m = MODELS[name]()
    rng = np.random.default_rng(13)
    g = rng.normal(size=6 * m["xyz"].shape[0]) * 1e3
    ref = orc.gradient(m, w=0.5, g=g)
    mdl = sso.Model(m)
    st = mdl.solve(precision="fp32_ir", rtol=1e-9)
    assert st["status"] == 0
    st = mdl.gradient(0.5, g)
    assert st["status"] == 0
    r = mdl.result()
    free = ~m["fixed"].ravel().astype(bool)
    assert rel(r["u"], ref["u"]) <= TOL_FP32_IR
    assert rel(r["lam"][free], ref["lam"][free]) <= TOL_FP32_IR
    assert rel(r["dz"], ref["dz"]) <= TOL_FP32_IR
    if m["quad_conn"].shape[0]:
        assert rel(r["dt"], ref["dt"]) <= TOL_FP32_IR


def test_batched_autograd_general_objective_fp32_ir(sso, orc):
    """BatchSSOFunction with an upstream gradient on u (J_i = 0.7 C_i + g_i^T u_i
    + 0.1 V_i): each design's adjoint is a real FP32+IR solve, against the
    oracle."""
    from paper_2407_20026_gb300.autograd import BatchSSOFunction
    meshes = [meshgen.shell(n_el=6, span=8.0, seed=s) for s in range(3)]
    batch = sso.Batch([sso.Model(m) for m in meshes])
    z = torch.tensor(np.stack([m["xyz"][:, 2] for m in meshes]), device="cuda",
                     requires_grad=True)
    t = torch.tensor(np.stack([m["quad_props"][:, 0] for m in meshes]), device="cuda",
                     requires_grad=True)
    u, C, V = BatchSSOFunction.apply(batch, z, t, sso.options(rtol=1e-10))
    rng = np.random.default_rng(21)
    gvec = torch.tensor(rng.normal(size=tuple(u.shape)) * 1e2, device="cuda")
    (0.7 * C + (gvec * u).sum(dim=1) + 0.1 * V).sum().backward()
    refs = _oracle_gradients(orc, meshes, w=0.7, gs=list(gvec.cpu().numpy()))
    for i, (m, ref) in enumerate(zip(meshes, refs)):
        vol = orc.volume(m)
        assert rel(z.grad[i].cpu().numpy(), ref["dz"] + 0.1 * vol["dz"]) <= TOL_FP32_IR
        assert rel(t.grad[i].cpu().numpy(), ref["dt"] + 0.1 * vol["dt"]) <= TOL_FP32_IR


def test_autograd_with_fixed_thickness(sso, orc):
    """t = None keeps the thicknesses: backward returns dz only."""
    from paper_2407_20026_gb300.autograd import BatchSSOFunction, SSOFunction
    m = small_shell(5)
    ref = orc.gradient(m)
    mdl = sso.Model(m)
    z = torch.tensor(m["xyz"][:, 2], device="cuda", requires_grad=True)
    u, C, V = SSOFunction.apply(mdl, z, None, sso.options(precision="fp64", rtol=1e-11))
    C.backward()
    assert rel(z.grad.cpu().numpy(), ref["dz"]) <= TOL_FP64
    batch = sso.Batch([sso.Model(m)])
    zb = torch.tensor(m["xyz"][None, :, 2], device="cuda", requires_grad=True)
    u, C, V = BatchSSOFunction.apply(batch, zb, None, sso.options(precision="fp64", rtol=1e-11))
    C.sum().backward()
    assert rel(zb.grad[0].cpu().numpy(), ref["dz"]) <= TOL_FP64


# ---------------------------------------------------------------------------
# Double-float CG in one CTA per system (precision "f32x2", small systems)

F32X2_MODELS = ["gridshell10", "gridshell13", "shell5", "mixed", "shell9_clamped", "hub"]


@pytest.mark.parametrize("precond", ["block_jacobi", "jacobi", "two_level"])
@pytest.mark.parametrize("name", F32X2_MODELS)
def test_f32x2_solve_and_gradient(sso, orc, name, precond):
    """The one-CTA double-float CG reaches the FP64 tolerance against the
    oracle (u, C, dz, dt), with supports held at exactly zero."""
    m = MODELS[name]()
    ref = orc.gradient(m, w=1.0)
    mdl = sso.Model(m)
    st = mdl.solve(precision="f32x2", precond=precond, rtol=1e-10, raise_on_error=False)
    assert st["status"] == 0 and st["rel_residual"] <= 1e-10, st
    mdl.gradient(1.0)
    r = mdl.result()
    assert rel(r["u"], ref["u"]) <= TOL_FP64
    assert abs(r["C"] - ref["C"]) <= TOL_FP64 * abs(ref["C"])
    assert rel(r["dz"], ref["dz"]) <= TOL_FP64
    if m["quad_conn"].shape[0]:
        assert rel(r["dt"], ref["dt"]) <= TOL_FP64
    assert np.all(r["u"][m["fixed"].ravel().astype(bool)] == 0.0)


@pytest.mark.parametrize("name", ["gridshell10", "mixed"])
def test_f32x2_general_objective_adjoint(sso, orc, name):
    """J = w C + g^T u with the adjoint solve (Eq. 5) in the double-float CG."""
    m = MODELS[name]()
    rng = np.random.default_rng(17)
    g = rng.normal(size=6 * m["xyz"].shape[0]) * 1e3
    ref = orc.gradient(m, w=0.5, g=g)
    mdl = sso.Model(m)
    assert mdl.solve(precision="f32x2", rtol=1e-10)["status"] == 0
    assert mdl.gradient(0.5, g)["status"] == 0
    r = mdl.result()
    free = ~m["fixed"].ravel().astype(bool)
    assert rel(r["lam"][free], ref["lam"][free]) <= TOL_FP64
    assert rel(r["dz"], ref["dz"]) <= TOL_FP64


@pytest.mark.parametrize("precond", ["block_jacobi", "two_level"])
def test_f32x2_batch_equals_alone_bitwise(sso, precond):
    """One CTA per system with fixed-order sums: a system's result is the same
    bit for bit alone and in a batch of systems of different sizes."""
    ms = [MODELS[k]() for k in ("gridshell13", "shell5", "mixed", "gridshell10")]
    alone = []
    for m in ms:
        mdl = sso.Model(m)
        assert mdl.solve(precision="f32x2", precond=precond, rtol=1e-10)["status"] == 0
        mdl.gradient(1.0)
        alone.append(mdl.result())
    models = [sso.Model(m) for m in ms]
    batch = sso.Batch(models)
    stats = batch.solve(precision="f32x2", precond=precond, rtol=1e-10)
    assert all(s["status"] == 0 for s in stats)
    batch.gradient()
    for mdl, a in zip(models, alone):
        r = mdl.result()
        for k in ("u", "dz", "dt"):
            assert np.array_equal(r[k], a[k]), k
        assert r["C"] == a["C"]


def test_f32x2_caps_and_options(sso):
    """Iteration cap -> SSO_ERR_NOT_CONVERGED with the residual reported;
    the chain solver and the server refuse f32x2."""
    from paper_2407_20026_gb300 import _lib
    from paper_2407_20026_gb300.serve import Server
    mdl = sso.Model(MODELS["gridshell13"]())
    st = mdl.solve(precision="f32x2", rtol=1e-12, max_iter=5, raise_on_error=False)
    assert st["status"] == _lib.ERR_NOT_CONVERGED and st["iterations"] == 5
    # CG lowers the energy norm of the error, not the residual norm: after 5
    # iterations the residual is only required to be reported (finite, > 0)
    assert np.isfinite(st["rel_residual"]) and st["rel_residual"] > 0.0
    with pytest.raises(sso.SSOError):
        mdl.solve(precision="f32x2", precond="chain")
    with pytest.raises(sso.SSOError):
        Server(sso.options(precision="f32x2"))


@pytest.mark.parametrize("precond", ["block_jacobi", "two_level"])
def test_f32x2_large_system_global_vectors(sso, orc, precond):
    """A system above the shared-memory limit of the double-float CG (512
    nodes) keeps its vectors in global memory: same tolerance vs the oracle,
    and the same bits alone and next to a small system (whose vectors then
    also live in global memory)."""
    m = meshgen.shell(n_el=26, span=10.0, seed=8)
    assert m["xyz"].shape[0] > 512
    ref = orc.gradient(m)
    mdl = sso.Model(m)
    st = mdl.solve(precision="f32x2", precond=precond, rtol=1e-10, raise_on_error=False)
    assert st["status"] == 0, st
    mdl.gradient(1.0)
    r = mdl.result()
    assert rel(r["u"], ref["u"]) <= TOL_FP64
    assert rel(r["dz"], ref["dz"]) <= TOL_FP64
    assert rel(r["dt"], ref["dt"]) <= TOL_FP64
    small = MODELS["gridshell10"]()
    m_small = sso.Model(small)
    m_small.solve(precision="f32x2", precond=precond, rtol=1e-10)
    alone_small = m_small.result()["u"]
    pair = [sso.Model(small), sso.Model(m)]
    stats = sso.Batch(pair).solve(precision="f32x2", precond=precond, rtol=1e-10)
    assert all(s["status"] == 0 for s in stats)
    assert np.array_equal(pair[0].result()["u"], alone_small)
    assert np.array_equal(pair[1].result()["u"], r["u"])


@pytest.mark.parametrize("precision,precond", [("fp32_ir", "block_jacobi"), ("fp32_ir", "two_level"),
                                               ("fp64", "jacobi"), ("f32x2", "block_jacobi"),
                                               ("f32x2", "two_level")])
def test_split_batch_equals_alone_bitwise(sso, precision, precond):
    """A batch of 32 or more systems runs its CG as two concurrent parts (two
    streams, two host threads); every system's result is still the same bits
    as solving it alone, for the solve and for a general-objective adjoint."""
    ms = []
    for k in range(34):
        if k % 2:
            ms.append(meshgen.gridshell(n_side=4 + k % 5, seed=k))
        else:
            ms.append(meshgen.shell(n_el=3 + k % 4, span=6.0, seed=k))
    opts = sso.options(precision=precision, precond=precond, rtol=1e-9)
    rng = np.random.default_rng(5)
    gs = [rng.normal(size=6 * m["xyz"].shape[0]) for m in ms]
    alone = []
    for m, g in zip(ms, gs):
        mdl = sso.Model(m)
        assert mdl.solve(opts)["status"] == 0
        mdl.gradient(0.5, g)
        alone.append(mdl.result())
    models = [sso.Model(m) for m in ms]
    batch = sso.Batch(models)
    stats = batch.solve(opts)
    assert all(s["status"] == 0 for s in stats)
    assert all(s["status"] == 0 for s in batch.gradient([0.5] * len(ms), gs))
    for mdl, a in zip(models, alone):
        r = mdl.result()
        for key in ("u", "dz", "dt", "lam"):
            assert np.array_equal(r[key], a[key]), key
        assert r["C"] == a["C"]


def test_batch_parts_do_not_change_results(sso):
    """The same batch solved as 1, 2 (default) and 3 concurrent parts gives
    the same bits."""
    ms = [meshgen.shell(n_el=3 + k % 5, span=6.0, seed=100 + k) for k in range(33)]
    batch = sso.Batch([sso.Model(m) for m in ms])
    opts = sso.options(precision="fp32_ir", rtol=1e-9)
    ref = None
    for parts in (2, 1, 3):
        batch.set_parts(parts)
        assert all(s["status"] == 0 for s in batch.solve(opts))
        batch.gradient()
        res = [mdl.result() for mdl in batch.models]
        if ref is None:
            ref = res
            continue
        for r, a in zip(res, ref):
            for key in ("u", "dz", "dt"):
                assert np.array_equal(r[key], a[key]), (parts, key)
    with pytest.raises(sso.SSOError):
        batch.set_parts(0)
