"""Continuous-batching server binding (sso_server_*) and a stream driver.

The server, the admission by HBM budget, the graph-launched batched CG and the
gradient of each request all run in libsso.so; this module marshals arguments
and replays a request stream against wall-clock arrival times.
"""
import ctypes
import time

import numpy as np

from . import _lib
from .model import mesh_struct, options


class Server:
    """sso_server: up to `max_systems` resident requests within `hbm_budget`
    bytes of per-request device memory and `max_tiles` tiles of 30 nodes,
    split over `lanes` lanes stepped at once (sso_server_create_lanes)."""

    def __init__(self, opts=None, hbm_budget=8 << 30, max_systems=256, max_tiles=1 << 20,
                 lanes=1, **kw):
        o = opts if opts is not None else options(**kw)
        h = ctypes.c_void_p()
        _lib.check(_lib.load().sso_server_create_lanes(ctypes.byref(o), int(hbm_budget),
                                                       int(max_systems), int(max_tiles),
                                                       int(lanes), ctypes.byref(h)))
        self._h = h
        self._shapes = {}

    def close(self):
        if getattr(self, "_h", None):
            _lib.load().sso_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, mesh, w=1.0):
        m, keep = mesh_struct(mesh)
        t = ctypes.c_uint64()
        _lib.check(_lib.load().sso_server_submit(self._h, ctypes.byref(m), float(w),
                                                 ctypes.byref(t)))
        self._shapes[t.value] = (m.n_nodes, m.n_quads)
        return t.value

    def step(self):
        """One round; returns (resident, waiting)."""
        r, q = ctypes.c_int32(), ctypes.c_int32()
        _lib.check(_lib.load().sso_server_step(self._h, ctypes.byref(r), ctypes.byref(q)))
        return r.value, q.value

    def completed(self, capacity=4096):
        """Tickets finished since the last call (their results await poll)."""
        buf = (ctypes.c_uint64 * capacity)()
        n = ctypes.c_int32()
        out = []
        while True:
            _lib.check(_lib.load().sso_server_completed(self._h, buf, capacity, ctypes.byref(n)))
            out.extend(buf[:n.value])
            if n.value < capacity:
                return out

    def info(self):
        """Host ms per phase of the steps so far and step / graph-launch counts."""
        ms = (ctypes.c_double * 8)()
        n = (ctypes.c_int64 * 2)()
        _lib.check(_lib.load().sso_server_info(self._h, ms, n))
        return {"admit_ms": ms[0], "upload_ms": ms[1], "wait_ms": ms[2], "harvest_ms": ms[3],
                "admit_prep_ms": ms[4], "admit_device_ms": ms[5], "admit_setup_ms": ms[6],
                "steps": n[0], "graph_launches": n[1]}

    def poll(self, ticket):
        """None while the request is not finished, else a dict of results."""
        n, nq = self._shapes[ticket]
        u = np.zeros(6 * n)
        dz = np.zeros(n)
        dt = np.zeros(max(nq, 1))
        C = np.zeros(1)
        st = _lib.Stats()
        lat = ctypes.c_double()
        code = _lib.load().sso_server_poll(self._h, ctypes.c_uint64(ticket), u.ctypes.data,
                                           C.ctypes.data, dz.ctypes.data, dt.ctypes.data,
                                           ctypes.byref(st), ctypes.byref(lat))
        if code == _lib.ERR_NOT_READY:
            return None
        _lib.check(code)
        del self._shapes[ticket]
        return {"u": u, "C": float(C[0]), "dz": dz, "dt": dt[:nq], "stats": st.as_dict(),
                "latency_ms": lat.value}


def run_stream(server, requests, time_limit_s=600.0):
    """Replays `requests` (dicts with "mesh", "t_arrive" seconds, optional "w")
    against the wall clock: each is submitted when its arrival time has
    passed, and the server is stepped until every result is in.  Returns
    (results in request order, elapsed seconds)."""
    order = sorted(range(len(requests)), key=lambda i: requests[i]["t_arrive"])
    tickets = {}
    results = [None] * len(requests)
    nxt = 0
    outstanding = set()
    t0 = time.perf_counter()
    while nxt < len(order) or outstanding:
        now = time.perf_counter() - t0
        if now > time_limit_s:
            raise TimeoutError("request stream not finished in %.0f s" % time_limit_s)
        while nxt < len(order) and requests[order[nxt]]["t_arrive"] <= now:
            i = order[nxt]
            tk = server.submit(requests[i]["mesh"], requests[i].get("w", 1.0))
            tickets[tk] = i
            outstanding.add(tk)
            nxt += 1
        resident, waiting = server.step()
        for tk in server.completed():
            if tk not in outstanding:
                continue
            r = server.poll(tk)
            if r is not None:
                i = tickets[tk]
                # latency from the arrival time, including any wait before submission
                r["latency_arrival_ms"] = 1000.0 * (time.perf_counter() - t0 -
                                                    requests[i]["t_arrive"])
                results[i] = r
                outstanding.discard(tk)
        if resident == 0 and waiting == 0 and not outstanding and nxt < len(order):
            wait = requests[order[nxt]]["t_arrive"] - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(min(wait, 0.05))
    return results, time.perf_counter() - t0
