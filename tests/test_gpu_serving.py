"""Continuous-batching server: requests of uneven size admitted while others
run give exactly the result of the same request solved alone; admission
respects the HBM budget; invalid requests fail alone."""
import numpy as np
import pytest
import torch

import meshgen
from gpu_util import TOL_FP32_IR, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sso():
    import paper_2407_20026_gb300 as pkg
    from paper_2407_20026_gb300 import _build
    _build.build()
    assert torch.cuda.is_available()
    return pkg


def _requests():
    reqs = []
    for k, n in enumerate([8, 23, 12, 31, 9, 17, 40, 11]):
        reqs.append({"mesh": meshgen.gridshell(n_side=n, seed=100 + k), "w": 1.0})
    reqs.append({"mesh": meshgen.shell(n_el=12, span=10.0, seed=5), "w": 0.5})
    reqs.append({"mesh": meshgen.shell(n_el=7, span=6.0, seed=6, supports="clamped",
                                       load="pressure"), "w": 1.0})
    return reqs


def _alone(sso, req, opts):
    mdl = sso.Model(req["mesh"])
    mdl.solve(opts)
    mdl.gradient(req["w"])
    return mdl.result()


def _serve(srv, reqs, waves):
    """Submit in waves, stepping the server between waves (admission while
    earlier requests are resident)."""
    tickets = []
    out = {}
    k = 0
    for size in waves:
        for r in reqs[k:k + size]:
            tickets.append(srv.submit(r["mesh"], r["w"]))
        k += size
        for _ in range(3):
            srv.step()
            for i, t in enumerate(tickets):
                if i not in out:
                    res = srv.poll(t)
                    if res is not None:
                        out[i] = res
    for _ in range(100000):
        if len(out) == len(tickets):
            break
        srv.step()
        for i, t in enumerate(tickets):
            if i not in out:
                res = srv.poll(t)
                if res is not None:
                    out[i] = res
    return [out[i] for i in range(len(tickets))]


@pytest.mark.parametrize("budget", [8 << 30, 16 << 20])
def test_server_results_equal_alone(sso, budget):
    from paper_2407_20026_gb300.serve import Server
    reqs = _requests()
    opts = sso.options(precision="fp32_ir", rtol=1e-8, iters_per_launch=16)
    alone = [_alone(sso, req, opts) for req in reqs]
    srv = Server(opts, hbm_budget=budget, max_systems=6)
    got = _serve(srv, reqs, waves=[3, 4, 3])
    for req, r, a in zip(reqs, got, alone):
        assert r["stats"]["status"] == 0
        for key in ("u", "dz", "dt"):
            assert np.array_equal(r[key], a[key]), key
        assert r["C"] == a["C"]
        assert r["latency_ms"] > 0


def test_server_against_oracle_and_invalid_request(sso, orc):
    from paper_2407_20026_gb300.serve import Server
    good = meshgen.gridshell(n_side=14, seed=3)
    bad = meshgen.gridshell(n_side=6, seed=4)
    bad["beam_conn"][2, 1] = 10 ** 6  # node index out of range
    srv = Server(sso.options(precision="fp32_ir", rtol=1e-9), max_systems=4)
    t_bad = srv.submit(bad)
    t_good = srv.submit(good)
    res = {}
    for _ in range(100000):
        srv.step()
        for t in (t_bad, t_good):
            if t not in res:
                r = srv.poll(t)
                if r is not None:
                    res[t] = r
        if len(res) == 2:
            break
    assert res[t_bad]["stats"]["status"] == 1  # SSO_ERR_INVALID
    r = res[t_good]
    assert r["stats"]["status"] == 0
    ref = orc.gradient(good)
    assert rel(r["u"], ref["u"]) <= TOL_FP32_IR
    assert rel(r["dz"], ref["dz"]) <= TOL_FP32_IR
    assert abs(r["C"] - ref["C"]) <= TOL_FP32_IR * abs(ref["C"])


def test_stream_driver(sso):
    from paper_2407_20026_gb300.serve import Server, run_stream
    rng = np.random.default_rng(0)
    reqs = [{"mesh": meshgen.gridshell(n_side=int(n), seed=int(s)),
             "t_arrive": float(t)}
            for n, s, t in zip(rng.integers(8, 30, 12), rng.integers(0, 1000, 12),
                               np.cumsum(rng.exponential(0.01, 12)))]
    srv = Server(sso.options(rtol=1e-8), max_systems=8)
    results, elapsed = run_stream(srv, reqs, time_limit_s=120)
    assert all(r is not None and r["stats"]["status"] == 0 for r in results)
    assert all(r["latency_arrival_ms"] >= r["latency_ms"] - 1.0 for r in results)


def test_two_level_server_results_equal_alone(sso):
    """Two-level requests admitted and retired while others iterate (the
    coarse work lists are rebuilt as the resident set changes) give the bits
    of the same request solved alone with the two-level preconditioner."""
    from paper_2407_20026_gb300.serve import Server
    reqs = _requests()
    opts = sso.options(precision="fp32_ir", precond="two_level", rtol=1e-8, iters_per_launch=16)
    alone, iters = [], []
    for req in reqs:
        mdl = sso.Model(req["mesh"])
        iters.append(mdl.solve(opts)["iterations"])
        mdl.gradient(req["w"])
        alone.append(mdl.result())
    srv = Server(opts, max_systems=5)
    got = _serve(srv, reqs, waves=[2, 5, 3])
    for r, a, it in zip(got, alone, iters):
        assert r["stats"]["status"] == 0
        assert r["stats"]["iterations"] == it
        for key in ("u", "dz", "dt"):
            assert np.array_equal(r[key], a[key]), key
        assert r["C"] == a["C"]
    srv.close()


@pytest.mark.parametrize("precond", ["block_jacobi", "two_level"])
def test_lanes_server_results_equal_alone(sso, precond):
    """A server of three lanes (requests routed to the least-loaded lane, the
    lanes stepped at once on their own threads) returns, under its own
    tickets, the bits of every request solved alone; the completion list and
    the phase counters cover all lanes."""
    from paper_2407_20026_gb300.serve import Server, run_stream
    reqs = _requests()
    opts = sso.options(precision="fp32_ir", precond=precond, rtol=1e-8, iters_per_launch=16)
    alone = [_alone(sso, req, opts) for req in reqs]
    srv = Server(opts, hbm_budget=3 << 30, max_systems=9, lanes=3)
    got = _serve(srv, reqs, waves=[3, 4, 3])
    for r, a in zip(got, alone):
        assert r["stats"]["status"] == 0
        for key in ("u", "dz", "dt"):
            assert np.array_equal(r[key], a[key]), key
        assert r["C"] == a["C"]
    info = srv.info()
    assert info["steps"] > 0 and info["graph_launches"] >= info["steps"] // 2
    # the stream driver over lanes: results in request order
    results, _ = run_stream(srv, [{"mesh": r["mesh"], "t_arrive": 0.002 * k, "w": r["w"]}
                                  for k, r in enumerate(reqs)], time_limit_s=120)
    for r, a in zip(results, alone):
        assert np.array_equal(r["u"], a["u"])
    srv.close()


def test_lanes_argument_checks(sso):
    from paper_2407_20026_gb300.serve import Server
    with pytest.raises(sso.SSOError):
        Server(sso.options(), lanes=0)
    with pytest.raises(sso.SSOError):
        Server(sso.options(), max_systems=2, lanes=3)


def test_server_rejects_the_direct_chain_solver(sso):
    from paper_2407_20026_gb300.serve import Server
    with pytest.raises(sso.SSOError):
        Server(sso.options(precision="fp64", precond="chain"))
