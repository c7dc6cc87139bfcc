"""Failure paths reported as status codes, with nothing faulted, trapped or
hung on the GPU: the iteration cap, the wall-clock cap, a non-finite design
set after creation (and recovery from it), and a server request that can never
fit its HBM budget."""
import time

import numpy as np
import pytest

import meshgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sso():
    from paper_2407_20026_gb300 import _build
    _build.build()
    import paper_2407_20026_gb300 as pkg
    return pkg


def test_iteration_cap_reports_not_converged(sso):
    mdl = sso.Model(meshgen.shell(n_el=16, seed=2))
    st = mdl.solve(precision="fp32_ir", rtol=1e-8, max_iter=10, raise_on_error=False)
    assert st["status"] == 4  # SSO_ERR_NOT_CONVERGED
    assert 0 < st["iterations"] <= 10 + 32  # stops within one graph launch of the cap
    st = mdl.solve(precision="fp32_ir", rtol=1e-6, raise_on_error=False)
    assert st["status"] == 0


def test_wall_clock_cap_reports_timeout(sso):
    mdl = sso.Model(meshgen.shell(n_el=64, seed=1))
    t0 = time.perf_counter()
    st = mdl.solve(precision="fp32_ir", rtol=1e-6, timeout_ms=1e-3, raise_on_error=False)
    assert st["status"] == 5  # SSO_ERR_TIMEOUT
    assert st["iterations"] < 1000
    assert time.perf_counter() - t0 < 5.0
    st = mdl.solve(precision="fp32_ir", rtol=1e-6, raise_on_error=False)
    assert st["status"] == 0


def test_non_finite_design_is_an_error_not_a_hang(sso):
    m = meshgen.shell(n_el=12, seed=3)
    mdl = sso.Model(m)
    z = np.ascontiguousarray(m["xyz"][:, 2]).copy()
    bad = z.copy()
    bad[7] = np.nan
    mdl.set_design(bad)
    for prec in ("fp32_ir", "fp64"):
        st = mdl.solve(precision=prec, rtol=1e-6, raise_on_error=False)
        assert st["status"] in (1, 3), st  # SSO_ERR_INVALID or SSO_ERR_SINGULAR
    mdl.set_design(z)
    st = mdl.solve(precision="fp32_ir", rtol=1e-6, raise_on_error=False)
    assert st["status"] == 0


def test_server_request_beyond_budget_is_refused(sso):
    from paper_2407_20026_gb300.serve import Server
    srv = Server(sso.options(rtol=1e-6), hbm_budget=1 << 20, max_systems=4)
    small = srv.submit(meshgen.gridshell(n_side=4, seed=1))
    big = srv.submit(meshgen.gridshell(n_side=60, seed=2))
    res = {}
    t0 = time.perf_counter()
    while len(res) < 2 and time.perf_counter() - t0 < 60.0:
        srv.step()
        for t in (small, big):
            if t not in res:
                r = srv.poll(t)
                if r is not None:
                    res[t] = r
    assert res[big]["stats"]["status"] == 2  # SSO_ERR_OOM
    assert res[small]["stats"]["status"] == 0
    srv.close()
