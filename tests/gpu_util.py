"""Helpers shared by the GPU parity tests (comparison logic only)."""
import numpy as np

import meshgen

# Tolerances (relative 2-norm error against the FP64 oracle): FP64 mode 1e-8,
# FP32 CG inside FP64 refinement 1e-6 (the two figures the scope fixes).
TOL_FP64 = 1e-8
TOL_FP32_IR = 1e-6
# Element matrices: FP64 kernels vs FP64 oracle, different operation order.
TOL_ELEMENT = 1e-12


def rel(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def bsr_to_dense(row_ptr, col, blocks):
    n = len(row_ptr) - 1
    K = np.zeros((6 * n, 6 * n))
    for i in range(n):
        for k in range(row_ptr[i], row_ptr[i + 1]):
            j = col[k]
            K[6 * i:6 * i + 6, 6 * j:6 * j + 6] = blocks[k]
    return K


def with_supports(K, fixed):
    """K with fixed rows/columns zeroed and 1 on their diagonal."""
    K = K.copy()
    f = np.asarray(fixed, bool).ravel()
    K[f, :] = 0.0
    K[:, f] = 0.0
    K[f, f] = 1.0
    return K


def small_shell(n=5, seed=1):
    m = meshgen.shell(n_el=n, span=6.0, seed=seed, height=1.5)
    m["pressure"] = 2e3
    m["nodal_load"][n + 3, 0] = 1.5e3
    m["nodal_load"][2 * n + 1, 4] = -200.0
    return m


def mixed_model(n=5, seed=3):
    m = small_shell(n, seed)
    side = n + 1
    conn = [(j * side + i, j * side + i + 1) for j in (0, n) for i in range(n)]
    conn += [(j * side, (j + 1) * side) for j in range(n)]
    m["beam_conn"] = np.asarray(conn, np.int32)
    m["beam_props"] = np.tile([2e11, 8e10, 2e-6, 3e-6, 4e-6, 1e-3], (len(conn), 1))
    return m


def hub_model(n_side=8, hub=27):
    """Grid-shell with one node braced to every other node: the hub's block
    row is long enough that its tile cannot be staged in shared memory."""
    m = meshgen.gridshell(n_side=n_side, seed=7)
    have = {tuple(sorted(e)) for e in m["beam_conn"].tolist()}
    extra = [(hub, k) for k in range(n_side * n_side)
             if k != hub and tuple(sorted((hub, k))) not in have]
    conn = np.concatenate([m["beam_conn"], np.asarray(extra, np.int32)])
    m["beam_conn"] = conn.astype(np.int32)
    m["beam_props"] = np.tile(m["beam_props"][:1], (conn.shape[0], 1))
    return m


def permuted(m, perm):
    """The same structure with its nodes renumbered: old node k becomes
    perm[k].  Returns (mesh, perm); u_new[6 perm[k] + d] = u_old[6 k + d]."""
    perm = np.asarray(perm)
    inv = np.argsort(perm)
    out = dict(m)
    for k in ("xyz", "fixed", "nodal_load"):
        out[k] = m[k][inv]
    out["quad_conn"] = perm[m["quad_conn"]].astype(np.int32)
    out["beam_conn"] = perm[m["beam_conn"]].astype(np.int32)
    return out, perm
