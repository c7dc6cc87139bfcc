"""Node aggregates of the two-level preconditioner (host logic, no GPU): every
node in exactly one aggregate, every aggregate connected in the node graph,
sizes near the target, deterministic."""
import collections

import numpy as np
import pytest

import meshgen


@pytest.fixture(scope="module")
def sso():
    import paper_2407_20026_gb300 as pkg
    from paper_2407_20026_gb300 import _build
    _build.build()
    from paper_2407_20026_gb300 import model
    return model


def _adjacency(m):
    n = m["xyz"].shape[0]
    adj = [set([i]) for i in range(n)]
    for conn in (m["beam_conn"], m["quad_conn"]):
        for e in np.asarray(conn):
            for a in e:
                adj[a].update(int(b) for b in e)
    return adj


@pytest.mark.parametrize("mesh", [lambda: meshgen.shell(n_el=64, seed=0),
                                  lambda: meshgen.gridshell(n_side=37, seed=2),
                                  lambda: meshgen.shell(n_el=6, span=5.0, seed=1)])
def test_aggregates_partition_connected(sso, mesh):
    m = mesh()
    n = m["xyz"].shape[0]
    agg, n_agg = sso.aggregate(m)
    assert agg.shape == (n,) and agg.min() == 0 and agg.max() == n_agg - 1
    target = max(16, -(-n // 39))
    sizes = np.bincount(agg, minlength=n_agg)
    assert n_agg <= 39 and sizes.min() >= 1
    assert sizes.min() * 4 >= target or n_agg == 1
    adj = _adjacency(m)
    for g in range(n_agg):  # breadth-first search inside the aggregate reaches all of it
        members = np.nonzero(agg == g)[0]
        seen = {int(members[0])}
        q = collections.deque(seen)
        while q:
            v = q.popleft()
            for u in adj[v]:
                if agg[u] == g and u not in seen:
                    seen.add(u)
                    q.append(u)
        assert len(seen) == len(members)
    agg2, n2 = sso.aggregate(m)
    assert n2 == n_agg and np.array_equal(agg, agg2)
