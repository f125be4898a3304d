"""Coarse-grained fields and fluidized-mass advection on the GPU against the
FP64 oracle on identical seeded inputs: voxel and Gaussian kernels, velocity
fields, mass conservation of the advection, batches sampled per scene."""
import numpy as np
import pytest

from oracle import fields as F
from tests.parity_cases import packed_scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tds():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2011_00459_gb300 import build, tds

    build.build()
    return tds


def masses(scene):
    return scene["density"] * 4.0 / 3.0 * np.pi * np.asarray(scene["r"], np.float64) ** 3


def grid_over(tds, x, l0, scene=0, pad=2):
    lo = x.min(0) - pad * l0
    dims = np.ceil((x.max(0) + pad * l0 - lo) / l0).astype(int)
    return tds.make_grid(lo, l0, dims, scene), lo, tuple(int(d) for d in dims)


def rel_field(a, b):
    return float(np.abs(np.asarray(a, np.float64) - b).max() / max(np.abs(b).max(), 1e-30))


@pytest.mark.parametrize("kernel,R", [(0, 0.0), (1, 0.04), (1, 0.09)])
def test_fields_match_oracle(tds, kernel, R):
    scene = packed_scene(2500, 31)
    l0 = 0.05
    g = tds.Scene(scene)
    grid, lo, dims = grid_over(tds, scene["x"], l0)
    rho, p, u = g.coarse_grain(grid, kernel, R)
    rho, p, u = rho.cpu().numpy(), p.cpu().numpy(), u.cpu().numpy()
    g.close()
    ro, po, uo = F.coarse_grain(scene["x"], scene["v"], masses(scene), lo, l0, dims, kernel, R)
    assert rel_field(rho, ro) <= 1e-5
    assert rel_field(p, po) <= 1e-5
    big = ro > 1e-3 * ro.max()  # velocities where there is mass to define them
    assert np.abs(u[big] - uo[big]).max() <= 1e-4 * max(np.abs(uo[big]).max(), 1e-3)
    if kernel == 0:  # exact mass: every particle in one voxel
        assert np.array_equal(rho > 0, ro > 0)
        assert rho.sum() * l0 ** 3 == pytest.approx(masses(scene).sum(), rel=1e-5)


def test_batch_grids_sample_their_scene(tds):
    a, b = packed_scene(800, 32), packed_scene(1200, 33)
    bat = tds.Batch([a, b])
    l0 = 0.05
    for q, sc in enumerate((a, b)):
        grid, lo, dims = grid_over(tds, sc["x"], l0, scene=q)
        rho, _, _ = bat.coarse_grain(grid, 0)
        ro, _, _ = F.coarse_grain(sc["x"], sc["v"], masses(sc), lo, l0, dims, 0)
        assert rel_field(rho.cpu().numpy(), ro) <= 1e-5
    bat.close()


def test_advection_matches_oracle_and_conserves_mass(tds):
    import torch

    g = np.random.Generator(np.random.PCG64(7))
    nz, ny, nx = 9, 11, 13
    rho = g.uniform(0, 1, (nz, ny, nx)).astype(np.float32)
    u = g.normal(0, 1, (nz, ny, nx, 3)).astype(np.float32)
    src = g.normal(0, 0.1, (nz, ny, nx)).astype(np.float32)
    l0 = 0.1
    dt = float(l0 / (3.0 * np.abs(u).max()))
    grid = tds.make_grid((0.0, 0.0, 0.0), l0, (nx, ny, nz))
    dev = lambda a: torch.from_numpy(a).cuda()
    cur, ref = dev(rho), rho.astype(np.float64)
    for _ in range(20):
        cur = tds.advect_fluid(grid, dev(u), cur, dt, source=dev(src))
        ref = F.advect(ref, u, l0, dt, source=src)
    out = cur.cpu().numpy()
    assert rel_field(out, ref) <= 1e-5
    total = rho.astype(np.float64).sum() + 20 * dt * src.astype(np.float64).sum()
    assert out.astype(np.float64).sum() == pytest.approx(total, rel=1e-5)
    with pytest.raises(tds.TdsError):
        tds.advect_fluid(tds.make_grid((0, 0, 0), 0.0, (nx, ny, nz)), dev(u), cur, dt)
