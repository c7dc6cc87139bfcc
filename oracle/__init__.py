"""ctypes wrapper of the FP64 CPU oracle (``sso_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers.  The oracle shares no code
with the CUDA path; both read the same synthetic models from :mod:`meshgen`.

Every function takes a model ``dict`` (see :mod:`meshgen`) and returns numpy
arrays.  Citations are to arXiv 2407.20026 (JAX-SSO):

* :func:`beam_ke`, :func:`quad_ke`      element stiffness k_e (Sec. 2.2.1)
* :func:`beam_dke`, :func:`quad_dke`    dk_e/dp by forward-mode dual numbers
* :func:`load_vector`                   nodal + consistent area loads
* :func:`assemble_dense`                K of Eq. 1 without supports (small)
* :func:`solve`                         K u = f under supports (Eqs. 1-3)
* :func:`gradient`                      adjoint sensitivity (Eqs. 5-6)
* :func:`residual`                      f - K u element by element
* :func:`cg`                            Jacobi-PCG for meshes too large for
                                        the band Cholesky
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sso_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

OK, ERR_INVALID, ERR_SINGULAR, ERR_NOT_CONVERGED = 0, 1, 3, 4


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` next to the source with g++ (plain -O2)."""
    if force or not os.path.exists(_LIB_PATH) or \
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Mesh(ctypes.Structure):
    _fields_ = [
        ("n_nodes", ctypes.c_int32), ("xyz", ctypes.c_void_p),
        ("n_beams", ctypes.c_int32), ("beam_conn", ctypes.c_void_p),
        ("beam_props", ctypes.c_void_p),
        ("n_quads", ctypes.c_int32), ("quad_conn", ctypes.c_void_p),
        ("quad_props", ctypes.c_void_p),
        ("fixed", ctypes.c_void_p), ("nodal_load", ctypes.c_void_p),
        ("pressure", ctypes.c_double), ("gamma", ctypes.c_double),
    ]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        vp, i32, f64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        mp = ctypes.POINTER(_Mesh)
        sigs = {
            "orc_beam_ke": ([vp, vp, vp, vp], None),
            "orc_beam_dke": ([vp, vp, vp, i32, vp], None),
            "orc_quad_ke": ([vp, vp, vp], None),
            "orc_quad_dke": ([vp, vp, i32, vp], None),
            "orc_quad_fe": ([vp, f64, vp], None),
            "orc_quad_area": ([vp], f64),
            "orc_load_vector": ([mp, vp], None),
            "orc_assemble_dense": ([mp, vp], None),
            "orc_residual": ([mp, vp, vp], None),
            "orc_half_bandwidth": ([mp], i32),
            "orc_solve": ([mp, i32, vp, vp], i32),
            "orc_gradient": ([mp, f64, vp, vp, vp, vp, vp, vp], i32),
            "orc_adjoint_contract": ([mp, vp, vp, f64, vp, vp], None),
            "orc_cg": ([mp, f64, i32, vp, vp], i32),
            "orc_volume": ([mp, vp, vp, vp], None),
            "orc_adjoint_contract_E": ([mp, vp, vp, vp], None),
        }
        for name, (args, res) in sigs.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
    return _lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


class _Bound:
    """Keeps the contiguous arrays of a model alive while C reads them."""

    def __init__(self, model):
        self.xyz = _f64(model["xyz"])
        self.beam_conn = np.ascontiguousarray(model["beam_conn"], dtype=np.int32)
        self.beam_props = _f64(model["beam_props"])
        self.quad_conn = np.ascontiguousarray(model["quad_conn"], dtype=np.int32)
        self.quad_props = _f64(model["quad_props"])
        self.fixed = np.ascontiguousarray(model["fixed"], dtype=np.uint8)
        self.nodal_load = _f64(model["nodal_load"])
        self.n_nodes = self.xyz.shape[0]
        self.s = _Mesh(self.n_nodes, _ptr(self.xyz),
                       self.beam_conn.shape[0], _ptr(self.beam_conn), _ptr(self.beam_props),
                       self.quad_conn.shape[0], _ptr(self.quad_conn), _ptr(self.quad_props),
                       _ptr(self.fixed), _ptr(self.nodal_load),
                       float(model.get("pressure", 0.0)), float(model.get("gamma", 0.0)))

    def ref(self):
        return ctypes.byref(self.s)


def beam_ke(xi, xj, props):
    out = np.zeros((12, 12))
    _load().orc_beam_ke(_ptr(_f64(xi, 3)), _ptr(_f64(xj, 3)), _ptr(_f64(props, 6)), _ptr(out))
    return out


def beam_dke(xi, xj, props, which: int):
    out = np.zeros((12, 12))
    _load().orc_beam_dke(_ptr(_f64(xi, 3)), _ptr(_f64(xj, 3)), _ptr(_f64(props, 6)),
                         int(which), _ptr(out))
    return out


def quad_ke(X, props):
    """X: [4, 3] node coordinates; props: (t, E, nu, kx, ky)."""
    out = np.zeros((24, 24))
    _load().orc_quad_ke(_ptr(_f64(X, 12)), _ptr(_f64(props, 5)), _ptr(out))
    return out


def quad_dke(X, props, which: int):
    """which: 0..11 -> X.flat[which], 12..16 -> props[which - 12]."""
    out = np.zeros((24, 24))
    _load().orc_quad_dke(_ptr(_f64(X, 12)), _ptr(_f64(props, 5)), int(which), _ptr(out))
    return out


def quad_fe(X, q):
    out = np.zeros(24)
    _load().orc_quad_fe(_ptr(_f64(X, 12)), float(q), _ptr(out))
    return out


def quad_area(X):
    return float(_load().orc_quad_area(_ptr(_f64(X, 12))))


def load_vector(model):
    b = _Bound(model)
    out = np.zeros(6 * b.n_nodes)
    _load().orc_load_vector(b.ref(), _ptr(out))
    return out


def assemble_dense(model):
    b = _Bound(model)
    n = 6 * b.n_nodes
    out = np.zeros((n, n))
    _load().orc_assemble_dense(b.ref(), _ptr(out))
    return out


def residual(model, u):
    b = _Bound(model)
    uu = _f64(u, 6 * b.n_nodes)
    out = np.zeros(6 * b.n_nodes)
    _load().orc_residual(b.ref(), _ptr(uu), _ptr(out))
    return out


def half_bandwidth(model) -> int:
    b = _Bound(model)
    return int(_load().orc_half_bandwidth(b.ref()))


class OracleError(RuntimeError):
    pass


def solve(model, method: str = "band"):
    """Returns (u [6 n_nodes], C).  method: band | dense | kkt."""
    code = {"band": 0, "dense": 1, "kkt": 2}[method]
    b = _Bound(model)
    u = np.zeros(6 * b.n_nodes)
    C = ctypes.c_double(0.0)
    st = _load().orc_solve(b.ref(), code, _ptr(u), ctypes.byref(C))
    if st != OK:
        raise OracleError("orc_solve status %d" % st)
    return u, C.value


def gradient(model, w: float = 1.0, g=None):
    """Adjoint sensitivity of J = w C + g^T u.

    Returns dict with u, C, dz [n_nodes], dt [n_quads], lam.
    """
    b = _Bound(model)
    n = 6 * b.n_nodes
    gg = None if g is None else _f64(g, n)
    u = np.zeros(n)
    lam = np.zeros(n)
    dz = np.zeros(b.n_nodes)
    dt = np.zeros(max(b.quad_conn.shape[0], 1))
    C = ctypes.c_double(0.0)
    st = _load().orc_gradient(b.ref(), float(w), _ptr(gg), _ptr(u), ctypes.byref(C),
                              _ptr(dz), _ptr(dt), _ptr(lam))
    if st != OK:
        raise OracleError("orc_gradient status %d" % st)
    return {"u": u, "C": C.value, "dz": dz, "dt": dt[:b.quad_conn.shape[0]], "lam": lam}


def adjoint_contract(model, u, lam, w: float = 1.0):
    b = _Bound(model)
    n = 6 * b.n_nodes
    dz = np.zeros(b.n_nodes)
    dt = np.zeros(max(b.quad_conn.shape[0], 1))
    _load().orc_adjoint_contract(b.ref(), _ptr(_f64(u, n)), _ptr(_f64(lam, n)), float(w),
                                 _ptr(dz), _ptr(dt))
    return dz, dt[:b.quad_conn.shape[0]]


def adjoint_contract_E(model, u, lam):
    """-lambda_e^T (dk_e/dE) u_e per quad (the E part of Eq. 6)."""
    b = _Bound(model)
    n = 6 * b.n_nodes
    dE = np.zeros(max(b.quad_conn.shape[0], 1))
    _load().orc_adjoint_contract_E(b.ref(), _ptr(_f64(u, n)), _ptr(_f64(lam, n)), _ptr(dE))
    return dE[:b.quad_conn.shape[0]]


def simp_model(model, rho, penal):
    """The model with SIMP moduli E_j = rho_j^penal E*_j (Eq. simp_eq), E* the
    model's own moduli."""
    out = dict(model)
    props = np.array(model["quad_props"], dtype=np.float64, copy=True)
    props[:, 1] = np.asarray(rho, np.float64) ** penal * props[:, 1]
    out["quad_props"] = props
    return out


def simp_gradient(model, rho, penal, w: float = 1.0, g=None):
    """gradient() of the SIMP model plus drho: dJ/drho_j = dJ/dE_j P rho_j^(P-1) E*_j."""
    rho = np.asarray(rho, np.float64)
    ms = simp_model(model, rho, penal)
    r = gradient(ms, w, g)
    dE = adjoint_contract_E(ms, r["u"], r["lam"])
    r["drho"] = dE * penal * rho ** (penal - 1.0) * np.asarray(model["quad_props"])[:, 1]
    return r


def volume(model):
    """Material volume W = sum_e A_e t_e of the quads (Sec. 3.3) and its
    gradients: dict with V, dz [n_nodes], dt [n_quads] (= A_e)."""
    b = _Bound(model)
    V = ctypes.c_double(0.0)
    dz = np.zeros(b.n_nodes)
    dt = np.zeros(max(b.quad_conn.shape[0], 1))
    _load().orc_volume(b.ref(), ctypes.byref(V), _ptr(dz), _ptr(dt))
    return {"V": V.value, "dz": dz, "dt": dt[:b.quad_conn.shape[0]]}


def cg(model, rtol: float = 1e-12, max_iter: int = 200000):
    b = _Bound(model)
    u = np.zeros(6 * b.n_nodes)
    it = ctypes.c_int(0)
    st = _load().orc_cg(b.ref(), float(rtol), int(max_iter), _ptr(u), ctypes.byref(it))
    if st != OK:
        raise OracleError("orc_cg status %d after %d iterations" % (st, it.value))
    return u, it.value
