"""Pins of the active-zone oracle (Eq. failure_plane and the terrain-to-particle
conversion): the failure angle reduces to Rankine's for an upright blade, the
volume cut from a flat bed is the wedge's closed-form prism, mass is conserved,
new particles sit in their columns without overlaps and clear the terrain
around their node (FP64 geometry), an existing particle blocks
the positions it overlaps, dormant ids are used in order, and nothing is cut
above the surface or behind the blade."""
import math

import numpy as np
import pytest

from oracle import active_zone as AZ
from paper_2011_00459_gb300 import scenes as S

RHO_P, RHO_B = 2000.0, 1500.0


def upright(depth, phi=math.radians(35.0), length=0.5, rs=0.01, x=0.3):
    tool = {"pos": (x, 0.2, -depth), "quat": (1.0, 0.0, 0.0, 0.0), "vel": (0, 0, 0), "angvel": (0, 0, 0)}
    cutter = {"edge": (0.0, 0.0, 0.0), "dir": (0.0, 1.0, 0.0), "length": length, "normal": (1.0, 0.0, 0.0),
              "phi": phi, "bank_density": RHO_B, "spawn_radius": rs}
    return tool, cutter


def run(hf, W, x=np.zeros((0, 3)), r=np.zeros(0)):
    z = np.zeros_like(hf["h"])
    return AZ.cut_and_spawn(hf, z, hf["h"], W, x, r)


def test_failure_angle():
    phi = math.radians(35.0)
    tool, cutter = upright(0.1, phi)
    W = AZ.wedge(tool, cutter, RHO_P)
    assert W["theta"] == pytest.approx(math.pi / 4 - phi / 2, abs=1e-7)  # Rankine (phi as FP32)
    # a separation plane inclined 30 degrees from the vertical: beta = 60 degrees
    c = dict(cutter, normal=(math.cos(math.radians(30)), 0.0, math.sin(math.radians(30))))
    assert AZ.wedge(tool, c, RHO_P)["theta"] == pytest.approx(math.pi / 2 - (phi + math.radians(60)) / 2,
                                                               abs=1e-7)


@pytest.mark.parametrize("depth", [0.05, 0.12])
def test_flat_bed_cut_is_the_wedge_prism(depth):
    hf = S.flat_heightfield(600, 800, 0.0, 0.0, 0.001)
    tool, cutter = upright(depth, rs=0.0004)
    W = AZ.wedge(tool, cutter, RHO_P)
    h, pend, ids, pos, lib = run(hf, W)
    t = math.tan(W["theta"])
    rs = float(W["rs"])
    vol = 0.5 * cutter["length"] * (depth - rs * t) ** 2 / t  # ahead of the blade by at least r_s
    assert lib == pytest.approx(RHO_B * vol, rel=0.01)
    cut = h < 0
    xs = np.arange(hf["nx"] + 1) * hf["cell"]
    zf = -depth + (xs - 0.3) * t  # cut nodes lie on the failure plane, the rest is untouched
    assert np.allclose(h[cut], np.broadcast_to(zf, h.shape)[cut], atol=1e-6)
    assert np.all(h[~cut] == 0.0)
    ys = np.arange(hf["ny"] + 1) * hf["cell"]
    jj = np.nonzero(cut.any(1))[0]
    assert ys[jj].min() >= 0.2 - 1e-6 and ys[jj].max() <= 0.7 + 1e-6
    assert len(ids) == 0 and pend.sum() == pytest.approx(lib, rel=1e-5)  # no dormant slot: all pending


def conversion_case(n_dormant=5000):
    hf = S.flat_heightfield(60, 40, 0.0, 0.0, 0.02)  # cell = 2 r_s
    tool, cutter = upright(0.1)
    W = AZ.wedge(tool, cutter, RHO_P)
    return hf, W, np.zeros((n_dormant, 3)), np.zeros(n_dormant)


def test_mass_is_conserved_and_particles_fit_their_columns():
    hf, W, x, r = conversion_case()
    h, pend, ids, pos, lib = run(hf, W, x, r)
    assert len(ids) > 50
    assert list(ids) == list(range(len(ids)))  # dormant ids in order
    total = len(ids) * float(W["ms"]) + pend.astype(np.float64).sum()
    assert total == pytest.approx(lib, rel=1e-5)
    rs = float(W["rs"])
    i = np.rint(pos[:, 0] / hf["cell"]).astype(int)
    j = np.rint(pos[:, 1] / hf["cell"]).astype(int)
    assert np.all(pos[:, 2] - rs >= h[j, i] - 1e-6) and np.all(pos[:, 2] + rs <= 1e-6)  # within [new, old]
    from scipy.spatial import cKDTree

    assert len(cKDTree(pos.astype(np.float64)).query_pairs(2 * rs - 1e-6)) == 0  # no overlaps


def terrain_clearance(hf, h, i, j, z):
    """FP64 distance of the point z above node (i, j) from the nearest plane
    of the triangles having the node as a corner (cells split along the
    (a+1, b)-(a, b+1) diagonal)."""
    c = float(hf["cell"])
    corner = lambda a, b: np.array([a * c, b * c, float(h[b, a])])
    p = np.array([i * c, j * c, z])
    best = np.inf
    for a in (i - 1, i):
        for b in (j - 1, j):
            if not (0 <= a < hf["nx"] and 0 <= b < hf["ny"]):
                continue
            for tri in ([(a, b), (a + 1, b), (a, b + 1)], [(a + 1, b + 1), (a, b + 1), (a + 1, b)]):
                if (i, j) not in tri:
                    continue
                A, B, C = (corner(*t) for t in tri)
                n = np.cross(B - A, C - A)
                n /= np.linalg.norm(n) * np.sign(n[2])
                best = min(best, float(n @ (p - A)))
    return best


def test_new_particles_clear_the_terrain_around_their_node():
    hf, W, x, r = conversion_case()
    h, pend, ids, pos, lib = run(hf, W, x, r)
    rs = float(W["rs"])
    cell = float(hf["cell"])
    first = {}
    for p in pos.astype(np.float64):
        i, j = int(round(p[0] / cell)), int(round(p[1] / cell))
        assert terrain_clearance(hf, h, i, j, p[2]) >= rs - 1e-6
        first[(i, j)] = min(first.get((i, j), np.inf), p[2])
    # nothing else in the way: each column starts at the lowest position
    # z_f + r_s (1 + 2q) that clears the terrain
    steep = 0
    for (i, j), z in first.items():
        zf = float(h[j, i])
        q0 = next(q for q in range(64) if terrain_clearance(hf, h, i, j, zf + rs * (1 + 2 * q)) >= rs + 1e-6)
        assert z == pytest.approx(zf + rs * (1 + 2 * q0), abs=1e-6) or (
            z == pytest.approx(zf + rs * (1 + 2 * (q0 - 1)), abs=1e-6)
            and terrain_clearance(hf, h, i, j, z) == pytest.approx(rs, abs=1e-6))
        steep += q0 > 0
    assert steep > 0  # columns beside uncut terrain start higher up


def test_an_existing_particle_blocks_what_it_overlaps():
    hf, W, x, r = conversion_case()
    h0, _, ids0, pos0, _ = run(hf, W, x, r)
    target = pos0[len(pos0) // 2].astype(np.float64)
    # an active particle (radius 0.015) sitting at that position
    x1 = np.concatenate([[target], x])
    r1 = np.concatenate([[0.015], r])
    h1, _, ids1, pos1, _ = run(hf, W, x1, r1)
    assert np.array_equal(h1, h0)
    d = np.linalg.norm(pos1.astype(np.float64) - target, axis=1)
    assert d.min() >= 0.01 + 0.015 - 1e-6  # nothing placed where it overlaps
    blocked = np.linalg.norm(pos0.astype(np.float64) - target, axis=1) < 0.025
    assert blocked.sum() >= 1 and len(ids1) == len(ids0) - blocked.sum()
    assert ids1[0] == 1  # the active particle is id 0; dormant ids follow


def test_capacity_and_no_cut_cases():
    hf, W, _, _ = conversion_case()
    r = np.ones(50)
    r[[7, 11, 40]] = 0.0  # three dormant slots
    x = np.full((50, 3), 100.0)
    h, pend, ids, pos, lib = run(hf, W, x, r)
    assert list(ids) == [7, 11, 40]
    assert pend.astype(np.float64).sum() == pytest.approx(lib - 3 * float(W["ms"]), rel=1e-5)
    # edge above the surface: nothing
    tool, cutter = upright(0.1)
    W_up = AZ.wedge(dict(tool, pos=(0.3, 0.2, 0.05)), cutter, RHO_P)
    _, _, ids2, _, lib2 = run(hf, W_up, x, r)
    assert lib2 == 0.0 and len(ids2) == 0
    # the blade faces -x: the cut is on the other side
    W_back = AZ.wedge(tool, dict(cutter, normal=(-1.0, 0.0, 0.0)), RHO_P)
    h3, _, _, _, lib3 = run(hf, W_back, x, r)
    xs = np.arange(hf["nx"] + 1) * hf["cell"]
    assert lib3 > 0 and np.all(h3[:, xs > 0.3] == 0.0)
