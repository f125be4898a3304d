"""Pins of the coarse-graining and advection oracle (Eqs. cg_velocity and
advection) against closed forms: the truncated Gaussian kernel's mass fraction,
exact mass and momentum of the voxel kernel, a uniform velocity field, an
exact one-voxel shift at Courant number 1, a hand-computed two-cell step, and
conservation with closed boundaries."""
import math

import numpy as np
import pytest

from oracle import fields as F


def test_voxel_kernel_places_mass_and_momentum():
    l0, o, dims = 0.1, (0.0, 0.0, 0.0), (4, 3, 2)
    # particles at the centres of voxels (1,2,0), (3,0,1), (1,2,0)
    x = np.array([[0.15, 0.25, 0.05], [0.35, 0.05, 0.15], [0.15, 0.25, 0.05]])
    v = np.array([[1.0, 0.0, 0.0], [0.0, 2.0, 0.0], [0.0, 0.0, 3.0]])
    m = np.array([2.0, 5.0, 1.0])
    rho, p, u = F.coarse_grain(x, v, m, o, l0, dims, kernel=0)
    vol = l0 ** 3
    assert rho.shape == (2, 3, 4)
    assert rho[0, 2, 1] == pytest.approx(3.0 / vol) and rho[1, 0, 3] == pytest.approx(5.0 / vol)
    assert np.count_nonzero(rho) == 2
    assert np.allclose(u[0, 2, 1], [2.0 / 3.0, 0.0, 1.0])
    assert np.allclose(u[1, 0, 3], [0.0, 2.0, 0.0]) and np.all(u[0, 0, 0] == 0.0)
    assert rho.sum() * vol == pytest.approx(m.sum(), rel=1e-14)
    assert np.allclose(p.sum((0, 1, 2)) * vol, (m[:, None] * v).sum(0), rtol=1e-14)
    # outside the grid: clamped into the border voxels, mass still counted
    rho2, _, _ = F.coarse_grain([[-1.0, 9.0, 0.05]], [[0, 0, 0]], [1.0], o, l0, dims, kernel=0)
    assert rho2[0, 2, 0] == pytest.approx(1.0 / vol)


def test_gaussian_kernel_mass_inside_three_radii():
    l0, R = 0.1, 0.29  # 3R is no lattice distance, so no voxel centre sits on the cutoff
    n = 25
    o = np.full(3, -n * l0 / 2)
    x = np.zeros((1, 3))  # the centre of voxel (12, 12, 12)
    rho, p, u = F.coarse_grain(x, [[0.5, -0.25, 1.0]], [2.0], o, l0, (n, n, n), kernel=1, R=R)
    # mass of a 3-D Gaussian within 3R: P(chi_3 <= 3)
    frac = math.erf(3 / math.sqrt(2)) - math.sqrt(2 / math.pi) * 3 * math.exp(-4.5)
    assert rho.sum() * l0 ** 3 == pytest.approx(2.0 * frac, rel=3e-3)
    assert np.allclose(u[rho > 0], [0.5, -0.25, 1.0])
    # symmetric about the particle, peak at its voxel
    assert np.allclose(rho, rho[::-1, ::-1, ::-1])
    assert np.unravel_index(np.argmax(rho), rho.shape) == (12, 12, 12)
    assert rho.max() == pytest.approx(2.0 * (math.sqrt(2 * math.pi) * R) ** -3, rel=1e-12)
    # nothing beyond 3R
    assert rho[12, 12, 12 + 9] == 0.0 and rho[12, 12, 12 + 8] > 0.0


def test_advection_shifts_exactly_at_courant_one():
    dims = (10, 4, 3)
    rho = np.zeros(dims[::-1])
    rho[1, 2, 3] = 2.0
    rho[1, 1, 4] = 0.5
    u = np.zeros(dims[::-1] + (3,))
    u[..., 0] = 0.5
    l0, dt = 0.2, 0.4  # u dt / l0 = 1
    out = F.advect(rho, u, l0, dt)
    want = np.zeros_like(rho)
    want[1, 2, 4] = 2.0
    want[1, 1, 5] = 0.5
    assert np.allclose(out, want, atol=1e-15)


def test_advection_two_cells_by_hand_and_sources():
    rho = np.array([[[1.0, 0.0]]])
    u = np.zeros((1, 1, 2, 3))
    u[..., 0] = 1.0
    out = F.advect(rho, u, 1.0, 0.25)
    assert np.allclose(out, [[[0.75, 0.25]]])
    # flow towards -x uses the right cell's density
    u[..., 0] = -1.0
    out = F.advect(np.array([[[0.0, 1.0]]]), u, 1.0, 0.25)
    assert np.allclose(out, [[[0.25, 0.75]]])
    # no velocity: only the source acts
    out = F.advect(np.array([[[1.0, 2.0]]]), np.zeros((1, 1, 2, 3)), 1.0, 0.5, source=np.array([[[4.0, -2.0]]]))
    assert np.allclose(out, [[[3.0, 1.0]]])


def test_advection_conserves_mass_in_a_closed_box():
    g = np.random.Generator(np.random.PCG64(5))
    rho = g.uniform(0, 1, (5, 6, 7))
    u = g.normal(0, 1, (5, 6, 7, 3))
    src = g.normal(0, 0.1, (5, 6, 7))
    l0 = 0.1
    dt = l0 / (3 * np.abs(u).max())
    out = F.advect(rho, u, l0, dt, source=src)
    assert out.sum() == pytest.approx(rho.sum() + dt * src.sum(), rel=1e-13)
    assert out.min() >= -1e-12 - dt * np.abs(src).max()  # upwind keeps densities >= 0 under the CFL bound
