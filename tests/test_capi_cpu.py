"""The C-ABI library loads and exports every symbol of include/sso.h; argument
validation runs (and fails cleanly) without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import meshgen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2407_20026_gb300 import _build, _lib
    _build.build()
    return _lib


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "sso.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sso_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(L):
    names = _declared_functions()
    assert len(names) >= 18
    lib = L.load()
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(L.SIGNATURES), set(names) ^ set(L.SIGNATURES)


def test_default_options(L):
    o = L.Options()
    L.load().sso_default_options(ctypes.byref(o))
    assert o.precision == L.FP32_IR and o.precond == L.BLOCK_JACOBI
    assert o.rtol == 1e-8 and o.inner_rtol == 2e-3
    assert o.max_iter == 200000 and o.max_sweeps == 40 and o.iters_per_launch == 32


def _create(L, model):
    from paper_2407_20026_gb300.model import _buf
    import torch
    keep = []

    def p(k, dt):
        ptr, a = _buf(model[k], dt)
        keep.append(a)
        return ptr

    m = L.Mesh(model["xyz"].shape[0], p("xyz", torch.float64),
               model["beam_conn"].shape[0], p("beam_conn", torch.int32),
               p("beam_props", torch.float64),
               model["quad_conn"].shape[0], p("quad_conn", torch.int32),
               p("quad_props", torch.float64), p("fixed", torch.uint8),
               p("nodal_load", torch.float64), model["pressure"], model["gamma"])
    h = ctypes.c_void_p()
    st = L.load().sso_model_create(ctypes.byref(m), None, ctypes.byref(h))
    return st, L.load().sso_last_error().decode()


def _bad(kind):
    if kind.startswith("beam"):
        m = meshgen.gridshell(n_side=4)
        if kind == "beam_index":
            m["beam_conn"][3, 1] = 99
        elif kind == "beam_zero_length":
            m["beam_conn"][2, 1] = m["beam_conn"][2, 0]
        elif kind == "beam_props":
            m["beam_props"][1, 5] = 0.0
        return m
    m = meshgen.shell(n_el=3)
    if kind == "quad_index":
        m["quad_conn"][0, 2] = -1
    elif kind == "quad_repeated":
        m["quad_conn"][1, 3] = m["quad_conn"][1, 0]
    elif kind == "quad_nu":
        m["quad_props"][2, 2] = 0.5
    elif kind == "quad_nonconvex":
        m["xyz"][5, :2] = m["xyz"][0, :2] - 0.1
    elif kind == "nan_coord":
        m["xyz"][3, 2] = np.nan
    elif kind == "nan_load":
        m["nodal_load"][3, 2] = np.inf
    return m


@pytest.mark.parametrize("kind", ["beam_index", "beam_zero_length", "beam_props", "quad_index",
                                  "quad_repeated", "quad_nu", "quad_nonconvex", "nan_coord",
                                  "nan_load"])
def test_invalid_models_rejected(L, kind):
    st, msg = _create(L, _bad(kind))
    assert st == L.ERR_INVALID, (st, msg)
    assert msg


def test_null_arguments(L):
    lib = L.load()
    h = ctypes.c_void_p()
    assert lib.sso_model_create(None, None, ctypes.byref(h)) == L.ERR_INVALID
    assert lib.sso_model_solve(None, None, None) == L.ERR_INVALID
    assert lib.sso_batch_solve(None, None, None) == L.ERR_INVALID
    assert lib.sso_batch_create(None, 0, ctypes.byref(h)) == L.ERR_INVALID
    assert lib.sso_beam_stiffness(-1, None, None, None, None, None) == L.ERR_INVALID
    assert lib.sso_quad_stiffness(3, None, None, None, None, None) == L.ERR_INVALID
    assert "NULL" in lib.sso_last_error().decode()
