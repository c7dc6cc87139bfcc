"""Pins of the oracle's material volume W = sum_e A_e t_e (Sec. 3.3): the exact
area of a flat plan, linearity in t, invariance under a rigid z shift, and
central finite differences of the z gradient on a warped mesh."""
import numpy as np
import pytest

import meshgen


def _flat(n_el=4, span=6.0, t=0.12):
    m = meshgen.shell(n_el=n_el, span=span, seed=0, thickness=t)
    m["xyz"][:, 2] = 0.0
    return m


def test_flat_plan_volume_is_exact(orc):
    m = _flat()
    r = orc.volume(m)
    assert r["V"] == pytest.approx(6.0 * 6.0 * 0.12, rel=1e-13)
    np.testing.assert_allclose(r["dt"], (6.0 / 4) ** 2, rtol=1e-13)
    # a flat surface is stationary in area under normal (z) motion
    assert np.max(np.abs(r["dz"])) <= 1e-12


def test_volume_is_linear_in_thickness(orc):
    m = meshgen.shell(n_el=5, span=8.0, seed=3)
    r = orc.volume(m)
    t = m["quad_props"][:, 0]
    assert r["V"] == pytest.approx(float(np.dot(r["dt"], t)), rel=1e-13)
    m2 = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in m.items()}
    m2["quad_props"][:, 0] *= 2.5
    assert orc.volume(m2)["V"] == pytest.approx(2.5 * r["V"], rel=1e-13)


def test_rigid_z_shift_leaves_volume_unchanged(orc):
    m = meshgen.shell(n_el=5, span=8.0, seed=4)
    r = orc.volume(m)
    # translation invariance: the z gradient sums to zero
    assert abs(r["dz"].sum()) <= 1e-10 * np.abs(r["dz"]).sum()
    m2 = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in m.items()}
    m2["xyz"][:, 2] += 0.37
    assert orc.volume(m2)["V"] == pytest.approx(r["V"], rel=1e-13)


def test_z_gradient_matches_central_differences(orc):
    m = meshgen.shell(n_el=4, span=6.0, seed=5)
    r = orc.volume(m)
    h = 1e-5
    fd = np.zeros(len(r["dz"]))
    for i in range(len(fd)):
        mp = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in m.items()}
        mm = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in m.items()}
        mp["xyz"][i, 2] += h
        mm["xyz"][i, 2] -= h
        fd[i] = (orc.volume(mp)["V"] - orc.volume(mm)["V"]) / (2 * h)
    assert np.linalg.norm(fd - r["dz"]) <= 1e-7 * np.linalg.norm(r["dz"])
