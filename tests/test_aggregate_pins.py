"""Pins of the aggregate-body oracle (Eqs. aggregate_mass to aggregate_rot_vel)
against closed forms and invariants: a rigid motion is recovered exactly, the
inertia of two particles and of a cubic lattice match their textbook values,
a translation has no spin, and membership follows the first containing zone.
Each pin fails for a plausible slip (unsquared norm, wrong sign on the outer
product, moments about the origin instead of the centre of mass, a wrong
membership rule)."""
import numpy as np
import pytest

from oracle import aggregate as AG
from paper_2011_00459_gb300.scenes import box_planes

RHO = 2000.0


def mass(r):
    return RHO * 4.0 / 3.0 * np.pi * np.asarray(r, np.float64) ** 3


def big_box():
    return [{"scene": 0, "planes": box_planes((0.0, 0.0, 0.0), (100.0, 100.0, 100.0))}]


def test_rigid_motion_is_recovered():
    g = np.random.Generator(np.random.PCG64(1))
    x = g.uniform(-0.5, 0.5, (300, 3)) + np.array([3.0, -2.0, 1.0])
    r = g.uniform(0.02, 0.04, 300)
    c = np.array([2.5, -1.5, 0.7])
    v0 = np.array([0.3, -0.1, 0.2])
    w0 = np.array([0.7, -1.3, 0.4])
    v = v0 + np.cross(w0, x - c)
    a = AG.aggregate(x, v, r, RHO, big_box())[0]
    assert a["count"] == 300
    assert np.allclose(a["omega"], w0, rtol=0, atol=1e-10)
    assert np.allclose(a["vel"], v0 + np.cross(w0, a["com"] - c), atol=1e-12)
    m = mass(r)
    assert a["mass"] == pytest.approx(m.sum(), rel=1e-14)
    assert np.allclose(a["com"], (m[:, None] * x).sum(0) / m.sum(), atol=1e-13)


def test_two_particle_inertia_and_spin():
    d, u = 0.3, 0.8
    x = np.array([[1.0 + d, 2.0, 3.0], [1.0 - d, 2.0, 3.0]])
    v = np.array([[0.0, u, 0.0], [0.0, -u, 0.0]])
    r = np.array([0.05, 0.05])
    m = mass(r)[0]
    a = AG.aggregate(x, v, r, RHO, big_box())[0]
    assert np.allclose(a["com"], [1.0, 2.0, 3.0], atol=1e-15)
    # squared distance, minus the outer product: no inertia about the pair's axis
    assert np.allclose(a["inertia"], np.diag([0.0, 2 * m * d * d, 2 * m * d * d]), atol=1e-15)
    # spin about z at u / d, nothing about the axis without inertia
    assert np.allclose(a["omega"], [0.0, 0.0, u / d], atol=1e-12)
    assert np.allclose(a["vel"], 0.0, atol=1e-15)


def test_cubic_lattice_inertia():
    k, s = 5, 0.1
    ii = np.stack(np.meshgrid(*[np.arange(k)] * 3, indexing="ij"), -1).reshape(-1, 3)
    x = ii * s + np.array([10.0, -4.0, 2.0])
    r = np.full(len(x), 0.04)
    a = AG.aggregate(x, np.zeros_like(x), r, RHO, big_box())[0]
    M = mass(r).sum()
    var = s * s * (k * k - 1) / 12.0  # per-axis variance of k evenly spaced points
    assert np.allclose(a["inertia"], np.eye(3) * M * 2 * var, rtol=1e-12, atol=1e-14)
    assert np.allclose(a["omega"], 0.0) and np.allclose(a["vel"], 0.0)


def test_translation_has_no_spin():
    g = np.random.Generator(np.random.PCG64(2))
    x = g.uniform(-1, 1, (50, 3))
    v = np.tile([0.4, -0.2, 1.1], (50, 1))
    a = AG.aggregate(x, v, g.uniform(0.02, 0.05, 50), RHO, big_box())[0]
    assert np.allclose(a["vel"], [0.4, -0.2, 1.1], atol=1e-14)
    assert np.allclose(a["omega"], 0.0, atol=1e-12)


def test_membership_first_zone_scene_and_faces():
    x = np.array([[0.0, 0.0, 0.0],   # in both boxes -> first
                  [0.5, 0.0, 0.0],   # exactly on the first box's +x face -> inside
                  [0.75, 0.0, 0.0],  # only in the second
                  [5.0, 5.0, 5.0],   # in none
                  [0.0, 0.0, 0.0]])  # other scene
    zones = [{"scene": 0, "planes": box_planes((0.0, 0.0, 0.0), (0.5, 0.5, 0.5))},
             {"scene": 0, "planes": box_planes((0.5, 0.0, 0.0), (0.5, 0.5, 0.5))},
             {"scene": 1, "planes": box_planes((0.0, 0.0, 0.0), (0.5, 0.5, 0.5))}]
    z = AG.zone_of(x, zones, scene_of=[0, 0, 0, 0, 1])
    assert list(z) == [0, 0, 1, -1, 2]
    out = AG.aggregate(x, np.zeros_like(x), np.full(5, 0.05), RHO, zones, scene_of=[0, 0, 0, 0, 1])
    assert [o["count"] for o in out] == [2, 1, 1]
    empty = AG.aggregate(x, np.zeros_like(x), np.full(5, 0.05), RHO,
                         [{"scene": 0, "planes": box_planes((9, 9, 9), (0.1, 0.1, 0.1))}])[0]
    assert empty["count"] == 0 and empty["mass"] == 0.0


def test_rotated_box_planes():
    th = 0.6
    R = np.array([[np.cos(th), -np.sin(th), 0.0], [np.sin(th), np.cos(th), 0.0], [0.0, 0.0, 1.0]])
    zones = [{"scene": 0, "planes": box_planes((1.0, 1.0, 0.0), (0.4, 0.1, 0.2), R)}]
    along = np.array([1.0, 1.0, 0.0]) + 0.35 * R[:, 0]
    across = np.array([1.0, 1.0, 0.0]) + 0.35 * R[:, 1]
    assert list(AG.zone_of(np.stack([along, across]), zones)) == [0, -1]
