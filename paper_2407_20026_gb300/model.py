"""Python binding of the C-ABI (argument marshalling only).

Every computation runs in libsso.so.  Inputs may be numpy arrays or torch
tensors (CPU or CUDA); the library itself detects host or device pointers.
"""
import ctypes

import numpy as np
import torch

from . import _lib

_NP = {torch.float64: np.float64, torch.float32: np.float32, torch.int32: np.int32,
       torch.uint8: np.uint8}


def _buf(x, dtype):
    """(pointer, keep-alive) of x as a contiguous array of torch dtype `dtype`."""
    if x is None:
        return None, None
    if isinstance(x, torch.Tensor):
        t = x.detach()
        if t.dtype != dtype:
            t = t.to(dtype)
        t = t.contiguous()
        return t.data_ptr(), t
    a = np.ascontiguousarray(x, dtype=_NP[dtype])
    return a.ctypes.data, a


def _stream_ptr(stream):
    if stream is not None:
        return int(getattr(stream, "cuda_stream", stream))
    if torch.cuda.is_available():
        return int(torch.cuda.current_stream().cuda_stream)
    return 0


def options(**kw):
    """sso_options with the library defaults, overridden by keyword.

    precision: "fp32_ir" | "fp64" | "f32x2" (double-float, one CTA per system:
    small systems); precond: "block_jacobi" | "jacobi" | "two_level" | "chain"; and the
    numeric fields of ``sso_options``.
    """
    lib = _lib.load()
    o = _lib.Options()
    lib.sso_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if k == "precision":
            v = {"fp64": _lib.FP64, "fp32_ir": _lib.FP32_IR, "f32x2": _lib.F32X2}.get(v, v)
        elif k == "precond":
            v = {"jacobi": _lib.JACOBI, "block_jacobi": _lib.BLOCK_JACOBI,
                 "two_level": _lib.TWO_LEVEL, "chain": _lib.CHAIN}.get(v, v)
        if not hasattr(o, k):
            raise TypeError("unknown option %r" % k)
        setattr(o, k, v)
    return o


def aggregate(mesh: dict):
    """(agg_of_node [n_nodes] int32, n_aggregates): the node aggregates of the
    two-level preconditioner (host only)."""
    m, keep = mesh_struct(mesh)
    out = np.zeros(m.n_nodes, np.int32)
    n = ctypes.c_int32()
    _lib.check(_lib.load().sso_aggregate(ctypes.byref(m), out.ctypes.data, ctypes.byref(n)))
    return out, n.value


def kernel_launches() -> int:
    return int(_lib.load().sso_kernel_launches())


def mesh_struct(mesh):
    """(sso_mesh, keep-alive list) for a model dict (see meshgen)."""
    keep = []

    def p(key, dtype):
        ptr, k = _buf(mesh[key], dtype)
        keep.append(k)
        return ptr

    m = _lib.Mesh(int(mesh["xyz"].shape[0]), p("xyz", torch.float64),
                  int(mesh["beam_conn"].shape[0]), p("beam_conn", torch.int32),
                  p("beam_props", torch.float64),
                  int(mesh["quad_conn"].shape[0]), p("quad_conn", torch.int32),
                  p("quad_props", torch.float64), p("fixed", torch.uint8),
                  p("nodal_load", torch.float64),
                  float(mesh.get("pressure", 0.0)), float(mesh.get("gamma", 0.0)))
    return m, keep


class Model:
    """One structure (sso_model): nodes, beams, quads, supports, loads."""

    def __init__(self, mesh: dict, stream=None):
        lib = _lib.load()
        m, keep = mesh_struct(mesh)
        self.n_nodes = m.n_nodes
        self.n_beams = m.n_beams
        self.n_quads = m.n_quads
        h = ctypes.c_void_p()
        _lib.check(lib.sso_model_create(ctypes.byref(m), ctypes.c_void_p(_stream_ptr(stream)),
                                        ctypes.byref(h)))
        self._h = h
        nn, nb, ne = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _lib.check(lib.sso_model_info(h, ctypes.byref(nn), ctypes.byref(nb), ctypes.byref(ne)))
        self.n_blocks = nb.value
        self.n_elem_blocks = ne.value
        self.last_stats = None

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            _lib.load().sso_model_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_design(self, z=None, t=None):
        zp, zk = _buf(z, torch.float64)
        tp, tk = _buf(t, torch.float64)
        _lib.check(_lib.load().sso_model_set_design(self._h, zp, tp))

    def set_topology(self, rho=None, penal=3.0):
        """SIMP densities (Eq. simp_eq): E_j = rho_j^penal E*_j; None restores E*."""
        rp, rk = _buf(rho, torch.float64)
        _lib.check(_lib.load().sso_model_set_topology(self._h, rp, float(penal)))
        self.has_topology = rho is not None

    def topology_gradient(self, device=None):
        """dJ/drho [n_quads] of the last gradient call."""
        if device is None:
            out = np.zeros(self.n_quads)
            ptr = out.ctypes.data
        else:
            out = torch.empty(self.n_quads, dtype=torch.float64, device=device)
            ptr = out.data_ptr()
        _lib.check(_lib.load().sso_model_get_topology_gradient(self._h, ptr))
        return out

    def solve(self, opts=None, raise_on_error=True, **kw):
        o = opts if opts is not None else options(**kw)
        st = _lib.Stats()
        code = _lib.load().sso_model_solve(self._h, ctypes.byref(o), ctypes.byref(st))
        if raise_on_error:
            _lib.check(code)
        self.last_stats = st.as_dict()
        return self.last_stats

    def gradient(self, w=1.0, g=None):
        gp, gk = _buf(g, torch.float64)
        st = _lib.Stats()
        _lib.check(_lib.load().sso_model_gradient(self._h, float(w), gp, ctypes.byref(st)))
        return st.as_dict()

    def result(self, device=None):
        """u, C, dz, dt, lam as numpy arrays (device None) or torch tensors on `device`."""
        n = self.n_nodes
        shapes = {"u": (6 * n,), "C": (1,), "dz": (n,), "dt": (max(self.n_quads, 1),),
                  "lam": (6 * n,)}
        if device is None:
            out = {k: np.zeros(s) for k, s in shapes.items()}
            ptrs = [out[k].ctypes.data for k in ("u", "C", "dz", "dt", "lam")]
        else:
            out = {k: torch.empty(s, dtype=torch.float64, device=device)
                   for k, s in shapes.items()}
            ptrs = [out[k].data_ptr() for k in ("u", "C", "dz", "dt", "lam")]
        _lib.check(_lib.load().sso_model_get(self._h, *ptrs))
        out["C"] = float(out["C"][0])
        out["dt"] = out["dt"][:self.n_quads]
        return out

    def volume(self, device=None):
        """Material volume W = sum A_e t_e at the current design: dict with V,
        dz [n_nodes], dt [n_quads] (numpy, or torch tensors on `device`)."""
        n, nq = self.n_nodes, self.n_quads
        if device is None:
            V, dz, dt = np.zeros(1), np.zeros(n), np.zeros(max(nq, 1))
            ptrs = [V.ctypes.data, dz.ctypes.data, dt.ctypes.data]
        else:
            V = torch.empty(1, dtype=torch.float64, device=device)
            dz = torch.empty(n, dtype=torch.float64, device=device)
            dt = torch.empty(max(nq, 1), dtype=torch.float64, device=device)
            ptrs = [V.data_ptr(), dz.data_ptr(), dt.data_ptr()]
        _lib.check(_lib.load().sso_model_volume(self._h, *ptrs))
        return {"V": V[0] if device is not None else float(V[0]), "dz": dz, "dt": dt[:nq]}

    def stiffness(self):
        """(row_ptr, col, K64 [nb,6,6], K32 [nb,6,6]) of the last assembly, numpy."""
        rp = np.zeros(self.n_nodes + 1, np.int32)
        col = np.zeros(self.n_blocks, np.int32)
        K64 = np.zeros((self.n_blocks, 6, 6))
        K32 = np.zeros((self.n_blocks, 6, 6), np.float32)
        _lib.check(_lib.load().sso_model_get_stiffness(self._h, rp.ctypes.data, col.ctypes.data,
                                                       K64.ctypes.data, K32.ctypes.data))
        return rp, col, K64, K32

    def load_vector(self):
        f = np.zeros(6 * self.n_nodes)
        _lib.check(_lib.load().sso_model_get_load(self._h, f.ctypes.data))
        return f


class Batch:
    """Several models solved together by one batched CG (sso_batch)."""

    def __init__(self, models):
        self.models = list(models)
        arr = (ctypes.c_void_p * len(self.models))(*[m.handle for m in self.models])
        h = ctypes.c_void_p()
        _lib.check(_lib.load().sso_batch_create(arr, len(self.models), ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _lib.load().sso_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, opts=None, raise_on_error=True, **kw):
        o = opts if opts is not None else options(**kw)
        st = (_lib.Stats * len(self.models))()
        code = _lib.load().sso_batch_solve(self._h, ctypes.byref(o), st)
        if raise_on_error:
            _lib.check(code)
        return [s.as_dict() for s in st]

    def set_parts(self, parts):
        """Run the CG as `parts` concurrent parts (1: none; default 2 from 32 models)."""
        _lib.check(_lib.load().sso_batch_set_parts(self._h, int(parts)))

    def set_profiling(self, enable=True):
        _lib.check(_lib.load().sso_batch_set_profiling(self._h, 1 if enable else 0))

    def kernel_times(self):
        """(ms in kernel A, ms in kernel B, timed (A, B) pairs) since profiling was enabled."""
        a, b, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
        _lib.check(_lib.load().sso_batch_kernel_times(self._h, ctypes.byref(a), ctypes.byref(b),
                                                      ctypes.byref(n)))
        return a.value, b.value, n.value

    def setup_times(self):
        """Device ms since profiling was enabled: dict with elements, assembly,
        precond (+ loads) -- each one launch for the whole batch per solve --,
        setup_wall (the whole set-up, two-level coarse spaces included),
        adjoint (elapsed contraction passes), setups, gradients."""
        v = [ctypes.c_double() for _ in range(5)]
        n = [ctypes.c_int64() for _ in range(2)]
        _lib.check(_lib.load().sso_batch_setup_times(self._h, *[ctypes.byref(x) for x in v],
                                                     *[ctypes.byref(x) for x in n]))
        return {"elements": v[0].value, "assembly": v[1].value, "precond": v[2].value,
                "adjoint": v[3].value, "setup_wall": v[4].value, "setups": n[0].value,
                "gradients": n[1].value}

    def gradient(self, w=None, g=None, raise_on_error=True):
        n = len(self.models)
        wa = (ctypes.c_double * n)(*([1.0] * n if w is None else [float(x) for x in w]))
        keep = []
        gp = None
        if g is not None:
            ptrs = []
            for gi in g:
                p, k = _buf(gi, torch.float64)
                keep.append(k)
                ptrs.append(p)
            gp = (ctypes.c_void_p * n)(*ptrs)
        st = (_lib.Stats * n)()
        code = _lib.load().sso_batch_gradient(self._h, wa, gp, st)
        if raise_on_error:
            _lib.check(code)
        return [s.as_dict() for s in st]


def beam_stiffness(xyz, conn, props, stream=None):
    """Element matrices of beam-columns on the GPU: [n, 2, 2, 6, 6] float64 (CUDA)."""
    xyz = xyz.to(torch.float64).contiguous()
    conn = conn.to(torch.int32).contiguous()
    props = props.to(torch.float64).contiguous()
    n = conn.shape[0]
    out = torch.empty((n, 2, 2, 6, 6), dtype=torch.float64, device=xyz.device)
    _lib.check(_lib.load().sso_beam_stiffness(n, xyz.data_ptr(), conn.data_ptr(),
                                              props.data_ptr(), out.data_ptr(),
                                              ctypes.c_void_p(_stream_ptr(stream))))
    return out


def quad_stiffness(xyz, conn, props, stream=None):
    """Element matrices of MITC-4 quads on the GPU: [n, 4, 4, 6, 6] float64 (CUDA)."""
    xyz = xyz.to(torch.float64).contiguous()
    conn = conn.to(torch.int32).contiguous()
    props = props.to(torch.float64).contiguous()
    n = conn.shape[0]
    out = torch.empty((n, 4, 4, 6, 6), dtype=torch.float64, device=xyz.device)
    _lib.check(_lib.load().sso_quad_stiffness(n, xyz.data_ptr(), conn.data_ptr(),
                                              props.data_ptr(), out.data_ptr(),
                                              ctypes.c_void_p(_stream_ptr(stream))))
    return out


def bsr_spmv(row_ptr, col, K, x, stream=None):
    """y = K x and x^T y for 6x6-block sparse K (CUDA tensors): returns (y, xty)."""
    row_ptr = row_ptr.to(torch.int32).contiguous()
    col = col.to(torch.int32).contiguous()
    K = K.to(torch.float64).contiguous()
    x = x.to(torch.float64).contiguous()
    n = row_ptr.shape[0] - 1
    y = torch.empty(6 * n, dtype=torch.float64, device=x.device)
    xty = torch.empty(1, dtype=torch.float64, device=x.device)
    _lib.check(_lib.load().sso_bsr_spmv(n, row_ptr.data_ptr(), col.data_ptr(), K.data_ptr(),
                                        x.data_ptr(), y.data_ptr(), xty.data_ptr(),
                                        ctypes.c_void_p(_stream_ptr(stream))))
    return y, xty
