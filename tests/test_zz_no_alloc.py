"""The no-allocation SpMV entry point against the allocating one.

Some callers cannot allocate device memory: a plug-in held to a fixed
device-memory budget by its host application, a real-time loop that cannot
take the allocator's latency or synchronisation, an application whose device
memory all belongs to its own pool.  sso_bsr_spmv_noalloc serves them with a
fixed scratch array compiled into the library.  This test calls it through the
C-ABI and checks it bit for bit against sso_bsr_spmv on the same inputs (both
run the same kernel in the same fixed order), on two calls in a row, and checks
that sizes beyond the fixed scratch are rejected.
"""
import ctypes

import numpy as np
import pytest
import torch

import meshgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2407_20026_gb300 import _build, _lib
    _build.build()
    assert torch.cuda.is_available()
    return _lib


def _assembled_k(n_el):
    import paper_2407_20026_gb300 as sso
    mdl = sso.Model(meshgen.shell(n_el=n_el, seed=n_el))
    try:
        mdl.solve(precision="fp64", max_iter=4)
    except sso.SSOError:
        pass  # only the assembled K is needed
    rp, col, K64, _ = mdl.stiffness()
    dev = "cuda"
    return (mdl.n_nodes, torch.tensor(rp, device=dev), torch.tensor(col, device=dev),
            torch.tensor(K64, device=dev))


def _call(fn, n, rp, col, K, x):
    y = torch.full((6 * n,), float("nan"), dtype=torch.float64, device="cuda")
    d = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    st = fn(n, rp.data_ptr(), col.data_ptr(), K.data_ptr(), x.data_ptr(), y.data_ptr(),
            d.data_ptr(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, y, d


@pytest.mark.parametrize("n_el", [5, 64])
def test_noalloc_matches_allocating_entry_point(L, n_el):
    lib = L.load()
    n, rp, col, K = _assembled_k(n_el)
    gen = torch.Generator(device="cuda").manual_seed(n_el)
    for call in range(2):  # two calls in a row, different x
        x = torch.randn(6 * n, dtype=torch.float64, device="cuda", generator=gen)
        st_a, y_a, d_a = _call(lib.sso_bsr_spmv, n, rp, col, K, x)
        st_n, y_n, d_n = _call(lib.sso_bsr_spmv_noalloc, n, rp, col, K, x)
        assert st_a == L.OK and st_n == L.OK, lib.sso_last_error()
        torch.cuda.synchronize()
        ya, yn = y_a.cpu().numpy(), y_n.cpu().numpy()
        assert np.all(np.isfinite(yn))
        assert np.array_equal(yn, ya)
        assert float(d_n) == float(d_a)


def test_noalloc_rejects_sizes_beyond_its_scratch(L):
    lib = L.load()
    st = lib.sso_bsr_spmv_noalloc((1 << 21) + 1, None, None, None, None, None, None, None)
    assert st == L.ERR_INVALID
    assert "exceeds" in lib.sso_last_error().decode()
