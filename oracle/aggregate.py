"""FP64 oracle of the aggregate bodies (section "Macroscale model", Eqs.
aggregate_mass to aggregate_rot_vel): each active zone's particles are lumped
into one rigid body with their mass, centre of mass, velocity, inertia tensor
and angular velocity.

TEST INFRASTRUCTURE ONLY (tests, smoke check); the product path never calls it.

Readings (the printed inertia is garbled):
* I_A = sum_a m_a (|x_a - x_A|^2 delta - (x_a - x_A)(x_a - x_A)^T): the squared
  distance and the minus sign of a point-mass inertia tensor about the centre of
  mass (the printed form has an unsquared norm and a plus sign on x_alpha x_beta,
  which is not an inertia tensor);
* point masses as printed: the spheres' own spin and 2/5 m r^2 are not summed;
* omega_A = I_A^+ L_A with L_A = sum_a m_a (x_a - x_A) x v_a, I_A^+ the
  pseudo-inverse (singular for fewer than three non-collinear particles:
  no angular velocity about an axis with no inertia);
* only particles: voxels with fluidized mass are not part of this build.

A zone is a convex region, the intersection of half-spaces n . x <= d, and
belongs to one scene of a batch; a particle belongs to the first zone (in the
given order) that contains it. Membership is decided in FP32 with the
operation order (n_x x + n_y y) + n_z z, which is what the GPU evaluates, so
both sides select the same particles.
"""
from __future__ import annotations

import numpy as np


def zone_of(x, zones, scene_of=None) -> np.ndarray:
    """Index of the first zone containing each particle (-1: none)."""
    xf = np.asarray(x, np.float32).reshape(-1, 3)
    n = xf.shape[0]
    sid = np.zeros(n, np.int64) if scene_of is None else np.asarray(scene_of, np.int64)
    out = np.full(n, -1, np.int64)
    for z, zone in enumerate(zones):
        inside = (sid == int(zone.get("scene", 0))) & (out < 0)
        for p in np.asarray(zone["planes"], np.float32).reshape(-1, 4):
            s = (p[0] * xf[:, 0] + p[1] * xf[:, 1]) + p[2] * xf[:, 2]  # float32, this order
            inside &= s <= p[3]
        out[inside] = z
    return out


def aggregate(x, v, r, density: float, zones, scene_of=None) -> list:
    """Per zone: dict(count, mass, com, vel, inertia (3x3), omega), FP64."""
    x = np.asarray(x, np.float64).reshape(-1, 3)
    v = np.asarray(v, np.float64).reshape(-1, 3)
    r = np.asarray(r, np.float64).reshape(-1)
    m = density * 4.0 / 3.0 * np.pi * r ** 3
    which = zone_of(x, zones, scene_of)
    out = []
    for z in range(len(zones)):
        sel = which == z
        if not sel.any():
            out.append({"count": 0, "mass": 0.0, "com": np.zeros(3), "vel": np.zeros(3),
                        "inertia": np.zeros((3, 3)), "omega": np.zeros(3)})
            continue
        mz, xz, vz = m[sel], x[sel], v[sel]
        M = mz.sum()
        com = (mz[:, None] * xz).sum(0) / M
        vel = (mz[:, None] * vz).sum(0) / M
        dx = xz - com
        I = np.zeros((3, 3))
        for a in range(3):
            for b in range(3):
                I[a, b] = np.sum(mz * ((dx * dx).sum(1) * (a == b) - dx[:, a] * dx[:, b]))
        L = (mz[:, None] * np.cross(dx, vz)).sum(0)
        omega = np.linalg.pinv(I, rcond=1e-12) @ L
        out.append({"count": int(sel.sum()), "mass": M, "com": com, "vel": vel, "inertia": I, "omega": omega})
    return out
