"""Seeded synthetic structural models (input generators only).

This module builds meshes, section/material properties, supports and nodal
loads for the workloads the library is exercised on.  It holds none of the
finite-element arithmetic: no element matrix, no assembly, no solve.  Both the
CUDA path and the FP64 oracle consume its output, so it is the one module they
share.

A model is a plain ``dict`` of numpy arrays:

``xyz``         float64 [n_nodes, 3]   node coordinates (m)
``beam_conn``   int32   [n_beams, 2]   beam-column end nodes i, j
``beam_props``  float64 [n_beams, 6]   E, G, Iy, Iz, J, A (the six section and
                                       material numbers of a beam-column,
                                       Sec. 2.2.1, Listing 1)
``quad_conn``   int32   [n_quads, 4]   quad nodes, counter-clockwise seen from
                                       the side the normal points to
``quad_props``  float64 [n_quads, 5]   t, E, nu, kappa_x, kappa_y (the material
                                       part of the quad attribute vector,
                                       Sec. 2.2.1)
``fixed``       uint8   [n_nodes, 6]   1 = DOF fixed; DOF order per node is
                                       (ux, uy, uz, rx, ry, rz) (Listing 1)
``nodal_load``  float64 [n_nodes, 6]   applied nodal forces / moments
``pressure``    float                  area load on quads (Pa), acting in -Z
``gamma``       float                  self-weight density (N/m^3); the area
                                       load of quad e is ``pressure + gamma*t_e``

Generators:

* :func:`gridshell`      -- beam-column grid-shell, orthogonal + one diagonal
                            per cell, sinusoidal z (10 x 10 nodes: 261 beams,
                            600 DOF)
* :func:`shell`          -- quad shell on a square plan with a smooth bump z
                            (64 x 64 quads: 25,350 DOF; 512 x 512: 1,579,014)
* :func:`serving_stream` -- seeded request stream of grid-shell sizes and
                            Poisson arrival times
* :func:`arch2d`, :func:`barrel_arch`, :func:`cantilever_strip`,
  :func:`patch_mesh`     -- small validation models (Sec. 2.2.3)
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "chs_section",
    "empty_model",
    "gridshell",
    "gridshell_z",
    "shell",
    "shell_z",
    "shell_thickness",
    "serving_stream",
    "arch2d",
    "barrel_arch",
    "cantilever_strip",
    "patch_mesh",
    "model_dofs",
]

PINNED = (1, 1, 1, 0, 0, 0)
CLAMPED = (1, 1, 1, 1, 1, 1)


def chs_section(r_out: float = 0.05, wall: float = 0.005):
    """Area, second moment and torsion constant of a circular hollow section.

    ``r_out`` is the outer radius.  Returns (A, I, J) with J = 2 I.
    """
    r_in = r_out - wall
    area = math.pi * (r_out ** 2 - r_in ** 2)
    inertia = math.pi / 4.0 * (r_out ** 4 - r_in ** 4)
    return area, inertia, 2.0 * inertia


def empty_model(n_nodes: int) -> dict:
    return {
        "xyz": np.zeros((n_nodes, 3), np.float64),
        "beam_conn": np.zeros((0, 2), np.int32),
        "beam_props": np.zeros((0, 6), np.float64),
        "quad_conn": np.zeros((0, 4), np.int32),
        "quad_props": np.zeros((0, 5), np.float64),
        "fixed": np.zeros((n_nodes, 6), np.uint8),
        "nodal_load": np.zeros((n_nodes, 6), np.float64),
        "pressure": 0.0,
        "gamma": 0.0,
    }


def model_dofs(model: dict) -> int:
    return int(model["xyz"].shape[0]) * 6


def _grid_nodes(n_side: int, span: float):
    """Row-major node grid: node (i, j) -> j * n_side + i, i along X."""
    s = np.linspace(0.0, span, n_side)
    xx, yy = np.meshgrid(s, s, indexing="xy")
    return xx.ravel(), yy.ravel()


def gridshell_z(x, y, rng, span: float = 10.0, n_waves: int = 4):
    """Sum of ``n_waves`` random sinusoids, each amplitude in [0, 0.5] m.

    z = sum_k a_k sin(2 pi (m_k x + n_k y) / span + phi_k) with
    a_k ~ U(0, 0.5), m_k, n_k uniform in {1, 2, 3}, phi_k ~ U(0, 2 pi);
    |z| <= 2 m by construction.
    """
    a = rng.uniform(0.0, 0.5, n_waves)
    m = rng.integers(1, 4, n_waves)
    n = rng.integers(1, 4, n_waves)
    phi = rng.uniform(0.0, 2.0 * math.pi, n_waves)
    z = np.zeros_like(x)
    for k in range(n_waves):
        z += a[k] * np.sin(2.0 * math.pi * (m[k] * x + n[k] * y) / span + phi[k])
    return z


def gridshell(n_side: int = 10, span: float = 10.0, seed: int = 0,
              E: float = 210e9, nu: float = 0.3, r_out: float = 0.05,
              wall: float = 0.005, load: float = -1000.0) -> dict:
    """Beam-column grid-shell: n_side x n_side nodes on a span x span plan.

    Members: every orthogonal edge of the node grid plus the diagonal
    (i, j) -> (i+1, j+1) of every cell, so 2 n (n-1) + (n-1)^2 members
    (261 for n = 10).  z from :func:`gridshell_z`.  Boundary nodes are pinned
    (ux, uy, uz fixed); every free node carries ``load`` N along Z.
    Circular hollow section with outer radius ``r_out`` and wall ``wall``.
    """
    rng = np.random.default_rng(seed)
    x, y = _grid_nodes(n_side, span)
    z = gridshell_z(x, y, rng, span)
    n_nodes = n_side * n_side
    model = empty_model(n_nodes)
    model["xyz"] = np.stack([x, y, z], axis=1)

    def nid(i, j):
        return j * n_side + i

    conn = []
    for j in range(n_side):
        for i in range(n_side - 1):
            conn.append((nid(i, j), nid(i + 1, j)))
    for j in range(n_side - 1):
        for i in range(n_side):
            conn.append((nid(i, j), nid(i, j + 1)))
    for j in range(n_side - 1):
        for i in range(n_side - 1):
            conn.append((nid(i, j), nid(i + 1, j + 1)))
    conn = np.asarray(conn, np.int32)
    area, inertia, tors = chs_section(r_out, wall)
    G = E / (2.0 * (1.0 + nu))
    props = np.tile(np.array([E, G, inertia, inertia, tors, area], np.float64),
                    (conn.shape[0], 1))
    model["beam_conn"] = conn
    model["beam_props"] = props
    ii = np.arange(n_nodes) % n_side
    jj = np.arange(n_nodes) // n_side
    boundary = (ii == 0) | (jj == 0) | (ii == n_side - 1) | (jj == n_side - 1)
    model["fixed"][boundary] = PINNED
    model["nodal_load"][~boundary, 2] = load
    return model


def shell_z(x, y, rng, span: float = 20.0, height: float = 5.0):
    """Smooth seeded bump with values in [0, height].

    s = sin(pi x / span) sin(pi y / span) (1 + 0.2 sum_{k=1,2} b_k
    sin(2 pi (m_k x + n_k y) / span + phi_k)), b_k ~ U(0, 1),
    m_k, n_k uniform in {1, 2, 3}, phi_k ~ U(0, 2 pi); z = height * s / max s.
    """
    b = rng.uniform(0.0, 1.0, 2)
    m = rng.integers(1, 4, 2)
    n = rng.integers(1, 4, 2)
    phi = rng.uniform(0.0, 2.0 * math.pi, 2)
    mod = np.ones_like(x)
    for k in range(2):
        mod += 0.2 * b[k] * np.sin(2.0 * math.pi * (m[k] * x + n[k] * y) / span + phi[k])
    s = np.sin(math.pi * x / span) * np.sin(math.pi * y / span) * mod
    return height * s / s.max()


def shell_thickness(n_quads: int, rng, lo: float = 0.05, hi: float = 0.2):
    return rng.uniform(lo, hi, n_quads)


def shell(n_el: int = 64, span: float = 20.0, seed: int = 0, height: float = 5.0,
          E: float = 30e9, nu: float = 0.2, thickness=None,
          supports: str = "corners", load: str = "selfweight",
          gamma: float = 25e3, pressure: float = 5e3) -> dict:
    """Quad shell of n_el x n_el elements on a span x span plan.

    Nodes are row-major ((n_el+1)^2 of them), quads are (i,j), (i+1,j),
    (i+1,j+1), (i,j+1).  z from :func:`shell_z`.  ``thickness`` is None for
    t_e ~ U[0.05, 0.2] i.i.d. per element, a float for a uniform value, or an
    array.  ``supports``: "corners" pins the 4 corner nodes (ux, uy, uz);
    "clamped" fixes all 6 DOFs of every boundary node.  ``load``:
    "selfweight" gives an area load gamma * t_e, "pressure" a uniform
    ``pressure``; both act in -Z.
    """
    rng = np.random.default_rng(seed)
    n_side = n_el + 1
    x, y = _grid_nodes(n_side, span)
    z = shell_z(x, y, rng, span, height)
    n_nodes = n_side * n_side
    model = empty_model(n_nodes)
    model["xyz"] = np.stack([x, y, z], axis=1)
    jj, ii = np.meshgrid(np.arange(n_el), np.arange(n_el), indexing="ij")
    n0 = (jj * n_side + ii).ravel()
    conn = np.stack([n0, n0 + 1, n0 + 1 + n_side, n0 + n_side], axis=1).astype(np.int32)
    n_quads = conn.shape[0]
    if thickness is None:
        t = shell_thickness(n_quads, rng)
    elif np.isscalar(thickness):
        t = np.full(n_quads, float(thickness))
    else:
        t = np.asarray(thickness, np.float64).reshape(n_quads)
    props = np.zeros((n_quads, 5), np.float64)
    props[:, 0] = t
    props[:, 1] = E
    props[:, 2] = nu
    props[:, 3] = 1.0
    props[:, 4] = 1.0
    model["quad_conn"] = conn
    model["quad_props"] = props
    ni = np.arange(n_nodes) % n_side
    nj = np.arange(n_nodes) // n_side
    if supports == "corners":
        corner = ((ni == 0) | (ni == n_side - 1)) & ((nj == 0) | (nj == n_side - 1))
        model["fixed"][corner] = PINNED
    elif supports == "clamped":
        boundary = (ni == 0) | (nj == 0) | (ni == n_side - 1) | (nj == n_side - 1)
        model["fixed"][boundary] = CLAMPED
    else:
        raise ValueError(supports)
    if load == "selfweight":
        model["gamma"] = float(gamma)
    elif load == "pressure":
        model["pressure"] = float(pressure)
    else:
        raise ValueError(load)
    return model


def serving_stream(n_requests: int = 512, seed: int = 0, n_min: int = 8,
                   n_max: int = 100, rate_per_s: float = 100.0):
    """Seeded request stream: grid sides n ~ U{n_min..n_max}, per-request
    geometry seeds and Poisson arrival times (exponential gaps, ``rate_per_s``).

    Returns a list of dicts with keys ``side``, ``seed`` and ``t_arrive`` (s).
    """
    rng = np.random.default_rng(seed)
    sides = rng.integers(n_min, n_max + 1, n_requests)
    seeds = rng.integers(0, 2 ** 31 - 1, n_requests)
    gaps = rng.exponential(1.0 / rate_per_s, n_requests)
    t = np.cumsum(gaps) - gaps[0]
    return [{"side": int(s), "seed": int(q), "t_arrive": float(a)}
            for s, q, a in zip(sides, seeds, t)]


def arch2d(n_el: int = 99, span: float = 10.0, rise: float = 5.0, E: float = 1.99e8,
           nu: float = 0.3, Iy: float = 6.6e-5, Iz: float = 3.3e-6, A: float = 4.3e-3,
           load: float = -500.0, J=None) -> dict:
    """2D parabolic arch of beam-columns in the XZ plane (Sec. 2.2.3).

    Both ends fixed in (ux, uy, uz, rx, rz) with ry free, the support vector of
    Listing 1.  ``load`` N along Z at every node.  The torsion constant is not
    given in the text; J defaults to Iy + Iz.
    """
    n_nodes = n_el + 1
    x = np.linspace(0.0, span, n_nodes)
    z = 4.0 * rise * x / span * (1.0 - x / span)
    model = empty_model(n_nodes)
    model["xyz"] = np.stack([x, np.zeros_like(x), z], axis=1)
    conn = np.stack([np.arange(n_el), np.arange(1, n_el + 1)], axis=1).astype(np.int32)
    G = E / (2.0 * (1.0 + nu))
    if J is None:
        J = Iy + Iz
    model["beam_conn"] = conn
    model["beam_props"] = np.tile(np.array([E, G, Iy, Iz, J, A]), (n_el, 1))
    for end in (0, n_nodes - 1):
        model["fixed"][end] = (1, 1, 1, 1, 0, 1)
    model["nodal_load"][:, 2] = load
    return model


def arch_bridge(n_spans: int = 100, el_per_span: int = 2, span: float = 30.0,
                rise: float = 10.0, E: float = 2.0e11, nu: float = 0.3, A: float = 4.3e-3,
                Iy: float = 6.6e-5, Iz: float = 3.3e-6, unit_weight: float = 7.85e4) -> dict:
    """Multi-span bridge of 2D parabolic arches of beam-columns in the XZ plane
    (the scaling structure of Sec. 2.2.4): n_spans arches of span x rise
    placed end to end along X, each cut into el_per_span equal-plan-length
    elements; consecutive arches share their pier node.  Every pier is a pin
    with the support vector of Listing 1 (ux, uy, uz, rx, rz fixed, ry free).
    Loads: self-weight as downward nodal loads, unit_weight * A times half the
    length of each element touching a node.  6 (n_spans el_per_span + 1) DOF:
    1,206 for 100 spans of 2 elements, about 3.9 million for 6,500.
    """
    n_el = n_spans * el_per_span
    n_nodes = n_el + 1
    x = np.arange(n_nodes) * (span / el_per_span)
    xi = (np.arange(n_nodes) % el_per_span) / el_per_span  # position within the span
    z = 4.0 * rise * xi * (1.0 - xi)
    model = empty_model(n_nodes)
    model["xyz"] = np.stack([x, np.zeros_like(x), z], axis=1)
    conn = np.stack([np.arange(n_el), np.arange(1, n_nodes)], axis=1).astype(np.int32)
    G = E / (2.0 * (1.0 + nu))
    model["beam_conn"] = conn
    model["beam_props"] = np.tile(np.array([E, G, Iy, Iz, Iy + Iz, A]), (n_el, 1))
    piers = np.arange(0, n_nodes, el_per_span)
    model["fixed"][piers] = (1, 1, 1, 1, 0, 1)
    length = np.linalg.norm(np.diff(model["xyz"], axis=0), axis=1)
    w = np.zeros(n_nodes)
    w[:-1] += 0.5 * length
    w[1:] += 0.5 * length
    model["nodal_load"][:, 2] = -unit_weight * A * w
    return model


def barrel_arch(n_el: int = 20, span: float = 19.0, rise: float = 4.5, E: float = 1.99e8,
                nu: float = 0.2, t: float = 0.25, load: float = -500e3) -> dict:
    """Parabolic barrel arch of quads (Sec. 2.2.3): parabola along X, extruded
    along Y, span x span plan, n_el x n_el quads, ground nodes (z = 0, the two
    edges x = 0 and x = span) pinned, ``load`` N along Z at every node.
    """
    n_side = n_el + 1
    x, y = _grid_nodes(n_side, span)
    z = 4.0 * rise * x / span * (1.0 - x / span)
    n_nodes = n_side * n_side
    model = empty_model(n_nodes)
    model["xyz"] = np.stack([x, y, z], axis=1)
    jj, ii = np.meshgrid(np.arange(n_el), np.arange(n_el), indexing="ij")
    n0 = (jj * n_side + ii).ravel()
    model["quad_conn"] = np.stack([n0, n0 + 1, n0 + 1 + n_side, n0 + n_side], 1).astype(np.int32)
    nq = n_el * n_el
    model["quad_props"] = np.tile(np.array([t, E, nu, 1.0, 1.0]), (nq, 1))
    ni = np.arange(n_nodes) % n_side
    ground = (ni == 0) | (ni == n_side - 1)
    model["fixed"][ground] = PINNED
    model["nodal_load"][:, 2] = load
    return model


def cantilever_strip(length: float = 10.0, width: float = 1.0, nx: int = 40, ny: int = 4,
                     t: float = 0.1, E: float = 1e9, nu: float = 0.0) -> dict:
    """Flat strip of quads along X in the XY plane, clamped at x = 0.

    No load is set; callers put the tip load where they need it.
    """
    xs = np.linspace(0.0, length, nx + 1)
    ys = np.linspace(0.0, width, ny + 1)
    xx, yy = np.meshgrid(xs, ys, indexing="xy")
    n_nodes = (nx + 1) * (ny + 1)
    model = empty_model(n_nodes)
    model["xyz"] = np.stack([xx.ravel(), yy.ravel(), np.zeros(n_nodes)], axis=1)
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    n0 = (jj * (nx + 1) + ii).ravel()
    model["quad_conn"] = np.stack([n0, n0 + 1, n0 + 1 + (nx + 1), n0 + (nx + 1)], 1).astype(np.int32)
    model["quad_props"] = np.tile(np.array([t, E, nu, 1.0, 1.0]), (nx * ny, 1))
    model["fixed"][np.isclose(model["xyz"][:, 0], 0.0)] = CLAMPED
    return model


def patch_mesh(distort: float = 0.0, warp: float = 0.0, seed: int = 0, t: float = 0.1,
               E: float = 1e6, nu: float = 0.25) -> dict:
    """Classic 2 x 2-cell patch on [0,2]^2 with the interior node moved.

    Nodes are row-major on a 3 x 3 grid; the interior node (index 4) is moved
    by ``distort`` (a fraction of the cell size, seeded direction) and every
    node gets a seeded z offset of amplitude ``warp``.  Nothing is fixed or
    loaded.
    """
    rng = np.random.default_rng(seed)
    s = np.linspace(0.0, 2.0, 3)
    xx, yy = np.meshgrid(s, s, indexing="xy")
    xyz = np.stack([xx.ravel(), yy.ravel(), np.zeros(9)], axis=1)
    ang = rng.uniform(0.0, 2.0 * math.pi)
    xyz[4, 0] += distort * math.cos(ang)
    xyz[4, 1] += distort * math.sin(ang)
    if warp:
        xyz[:, 2] += rng.uniform(-warp, warp, 9)
    model = empty_model(9)
    model["xyz"] = xyz
    conn = []
    for j in range(2):
        for i in range(2):
            n0 = j * 3 + i
            conn.append((n0, n0 + 1, n0 + 4, n0 + 3))
    model["quad_conn"] = np.asarray(conn, np.int32)
    model["quad_props"] = np.tile(np.array([t, E, nu, 1.0, 1.0]), (4, 1))
    return model
