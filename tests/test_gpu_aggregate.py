"""Aggregate bodies on the GPU against the FP64 oracle: zone membership
bit-exact (FP32 half-space test), mass, centre of mass, velocity, inertia and
angular velocity within FP32 rounding of the inputs on identical states, and
within the step's tolerances after stepping; batches take per-scene zones."""
import numpy as np
import pytest

from oracle import aggregate as AG
from paper_2011_00459_gb300 import scenes as S
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


def zones_for(x, scene=0):
    """Overlapping zones of several shapes inside the block: an axis box, a
    rotated box, a wedge (5 planes, the shape of an active zone) and one that
    holds everything left."""
    lo, hi = x.min(0), x.max(0)
    c, ext = 0.5 * (lo + hi), hi - lo
    th = 0.5
    R = np.array([[np.cos(th), 0.0, np.sin(th)], [0.0, 1.0, 0.0], [-np.sin(th), 0.0, np.cos(th)]])
    wedge = np.array([[-1.0, 0.0, 0.0, -(c[0] - 0.1 * ext[0])],                       # x >= ...
                      [0.0, 1.0, 0.0, c[1] + 0.3 * ext[1]], [0.0, -1.0, 0.0, -(c[1] - 0.3 * ext[1])],
                      [0.0, 0.0, -1.0, -lo[2]],                                        # z >= bottom
                      [0.6, 0.0, 0.8, 0.6 * (c[0] + 0.3 * ext[0]) + 0.8 * c[2]]], np.float32)  # failure plane
    return [{"scene": scene, "planes": S.box_planes(c - 0.25 * ext, 0.2 * ext)},
            {"scene": scene, "planes": S.box_planes(c, (0.3 * ext[0], 0.35 * ext[1], 0.25 * ext[2]), R)},
            {"scene": scene, "planes": wedge},
            {"scene": scene, "planes": S.box_planes(c, ext)}]


def compare(got, ref, rel):
    assert got["count"] == ref["count"]
    if ref["count"] == 0:
        assert got["mass"] == 0.0
        return
    scale_x = max(1.0, np.abs(ref["com"]).max())
    assert got["mass"] == pytest.approx(ref["mass"], rel=rel)
    assert np.abs(got["com"] - ref["com"]).max() <= rel * scale_x
    vs = max(np.abs(ref["vel"]).max(), 1e-3)
    assert np.abs(got["vel"] - ref["vel"]).max() <= rel * vs
    Is = np.abs(ref["inertia"]).max()
    assert np.abs(got["inertia"] - ref["inertia"]).max() <= rel * Is
    ws = max(np.abs(ref["omega"]).max(), 1e-3)
    assert np.abs(got["omega"] - ref["omega"]).max() <= 10 * rel * ws


def test_aggregates_of_the_initial_state(tds):
    scene = packed_scene(3000, 21)
    zones = zones_for(scene["x"])
    g = tds.Scene(scene)
    got = g.aggregate_bodies(zones)
    g.close()
    ref = AG.aggregate(scene["x"], scene["v"], scene["r"], scene["density"], zones)
    assert sum(r["count"] for r in ref) == len(scene["r"])
    assert all(r["count"] > 50 for r in ref)
    for a, b in zip(got, ref):
        compare(a, b, 1e-6)


def test_aggregates_after_steps(tds, orc):
    scene = packed_scene(2500, 22, iters=50)
    zones = zones_for(scene["x"])
    st = orc.State(scene)
    g = tds.Scene(scene)
    for _ in range(3):
        orc.step(scene, st)
        g.step(1)
    got = g.aggregate_bodies(zones)
    g.close()
    ref = AG.aggregate(st.x, st.v, scene["r"], scene["density"], zones)
    for a, b in zip(got, ref):
        compare(a, b, 2e-3)


def test_batch_zones_follow_their_scene(tds):
    a, b = packed_scene(900, 23, iters=30), packed_scene(1300, 24, iters=30)
    za, zb = zones_for(a["x"], 0), zones_for(b["x"], 1)
    bat = tds.Batch([a, b])
    got = bat.aggregate_bodies(za + zb)
    bat.close()
    ref = AG.aggregate(np.concatenate([a["x"], b["x"]]), np.concatenate([a["v"], b["v"]]),
                       np.concatenate([a["r"], b["r"]]), a["density"], za + zb,
                       scene_of=np.r_[np.zeros(900, int), np.ones(1300, int)])
    for x, y in zip(got, ref):
        compare(x, y, 1e-6)
    assert sum(r["count"] for r in got[:4]) == 900 and sum(r["count"] for r in got[4:]) == 1300


def test_invalid_zones_are_rejected(tds):
    scene = packed_scene(300, 25)
    g = tds.Scene(scene)
    with pytest.raises(tds.TdsError):
        g.aggregate_bodies([{"scene": 1, "planes": S.box_planes((0, 0, 0), (1, 1, 1))}])
    with pytest.raises(tds.TdsError):
        g.aggregate_bodies([{"scene": 0, "planes": np.zeros((0, 4))}])
    with pytest.raises(tds.TdsError):
        g.aggregate_bodies([{"scene": 0, "planes": S.box_planes((0, 0, 0), (1, 1, 1))}] * 65)
    assert g.aggregate_bodies([]) == []
    g.close()
