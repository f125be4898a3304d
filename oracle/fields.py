"""FP64 oracle of the coarse-grained fields (section "Coarse-graining", Eq.
cg_velocity) and of the conservative advection of fluidized mass (Eq.
advection) on a voxel grid.

TEST INFRASTRUCTURE ONLY (tests, smoke check); the product path never calls it.

Grid: voxel (i, j, k) has centre o + (i + 1/2, j + 1/2, k + 1/2) l0, i fastest.

Coarse-graining (readings):
* the fields are sampled at voxel centres: rho(x_v) = sum_a m_a zeta(x_v - x_a),
  p(x_v) = sum_a m_a v_a zeta(x_v - x_a), u = p / rho (0 where rho = 0);
* kernel 0, Heaviside: zeta = 1 / l0^3 on the voxel that contains the particle
  centre (coordinates clamped to the grid), which preserves mass exactly;
* kernel 1, Gaussian: zeta(x) = (sqrt(2 pi) R)^-3 exp(-|x|^2 / 2R^2), truncated
  where |x| > 3R (the printed kernel has unbounded support);
* the voxel of a particle is decided in FP32: floor((x - o) / l0) with the
  subtraction and division rounded to FP32, as the GPU evaluates it.

Advection of fluidized mass, d rho_f/dt + div(rho_f u) = r_f, first-order
upwind finite volumes: the face between voxels L and R (next along an axis)
carries F = u_f rho_upwind with u_f the mean of the two voxels' velocity
components along that axis and rho_upwind = rho_L if u_f > 0 else rho_R; faces
on the grid boundary carry nothing (closed domain); then
rho_new = rho + dt (sum F_in - sum F_out) / l0 + dt r_f. Each face flux
leaves one voxel and enters the other, so total mass changes only by the
sources. Stable for max |u| dt / l0 <= 1/3.
"""
from __future__ import annotations

import numpy as np


def voxel_index(x, origin, l0, dims):
    """Voxel (i, j, k) of each position, FP32 floor((x - o) / l0), clamped."""
    xf = np.asarray(x, np.float32).reshape(-1, 3)
    o = np.asarray(origin, np.float32)
    t = np.floor((xf - o) / np.float32(l0))
    idx = np.empty(t.shape, np.int64)
    for a in range(3):
        idx[:, a] = np.clip(np.nan_to_num(t[:, a], nan=0.0), 0, dims[a] - 1)
    return idx


def coarse_grain(x, v, m, origin, l0, dims, kernel: int = 0, R: float = 0.0):
    """rho (nz, ny, nx) and p (nz, ny, nx, 3) and u = p / rho."""
    x = np.asarray(x, np.float64).reshape(-1, 3)
    v = np.asarray(v, np.float64).reshape(-1, 3)
    m = np.asarray(m, np.float64).reshape(-1)
    nx, ny, nz = dims
    rho = np.zeros((nz, ny, nx))
    p = np.zeros((nz, ny, nx, 3))
    o = np.asarray(origin, np.float64)
    if kernel == 0:
        idx = voxel_index(x, origin, l0, dims)
        vol = l0 ** 3
        np.add.at(rho, (idx[:, 2], idx[:, 1], idx[:, 0]), m / vol)
        for a in range(3):
            np.add.at(p[..., a], (idx[:, 2], idx[:, 1], idx[:, 0]), m * v[:, a] / vol)
    else:
        norm = (np.sqrt(2.0 * np.pi) * R) ** -3
        centres = [o[a] + (np.arange(dims[a]) + 0.5) * l0 for a in range(3)]
        for a_ in range(len(m)):  # plain sum over particles and voxel centres
            d = [centres[a] - x[a_, a] for a in range(3)]
            r2 = d[2][:, None, None] ** 2 + d[1][None, :, None] ** 2 + d[0][None, None, :] ** 2
            w = np.where(r2 <= 9.0 * R * R, norm * np.exp(-r2 / (2.0 * R * R)), 0.0)
            rho += m[a_] * w
            p += (m[a_] * w)[..., None] * v[a_]
    with np.errstate(invalid="ignore", divide="ignore"):
        u = np.where(rho[..., None] > 0, p / rho[..., None], 0.0)
    return rho, p, u


def advect(rho, u, l0, dt, source=None):
    """One upwind step; rho (nz, ny, nx), u (nz, ny, nx, 3)."""
    rho = np.asarray(rho, np.float64)
    u = np.asarray(u, np.float64)
    out = rho.copy()
    for a in range(3):  # axis a of (x, y, z) is array axis 2 - a
        ax = 2 - a
        n = rho.shape[ax]
        for f in range(n - 1):  # face between cells f and f + 1 along the axis
            L = [slice(None)] * 3
            Rr = [slice(None)] * 3
            L[ax], Rr[ax] = f, f + 1
            uf = 0.5 * (u[tuple(L)][..., a] + u[tuple(Rr)][..., a])
            F = np.where(uf > 0, uf * rho[tuple(L)], uf * rho[tuple(Rr)])
            out[tuple(L)] -= dt * F / l0
            out[tuple(Rr)] += dt * F / l0
    if source is not None:
        out += dt * np.asarray(source, np.float64)
    return out
