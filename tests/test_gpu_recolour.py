"""Incremental colouring on the GPU: with a recolour period k, every k-th step
colours every contact and the steps between keep each persisting contact's
colour and colour only the new contacts. Checked against the oracle from
identical inputs (the oracle given the GPU's state, warm-start memory and
colours): contact sets and colourings bit-exact, impulses within 1e-4,
positions within 1e-6 m, in incremental and full steps; and bitwise equality
of graph replay with launches, of a batch with its scenes alone, and of a
resumed checkpoint with the uninterrupted run."""
import numpy as np
import pytest

from tests.parity_cases import packed_scene, rel_impulse_error

pytestmark = pytest.mark.gpu

PERIOD = 4


@pytest.fixture(scope="module")
def tds():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2011_00459_gb300 import build, tds

    build.build()
    return tds


def moved(tool, k):
    t = dict(tool)
    t["pos"] = tuple(np.asarray(tool["pos"]) + np.asarray(tool["vel"]) * (k + 1) / 60.0)
    return t


def test_incremental_and_full_steps_match_the_oracle_from_identical_inputs(tds, orc):
    scene = packed_scene(3000, 51, iters=40, recolour_every=PERIOD)
    g = tds.Scene(scene)
    checked = []
    for k in range(PERIOD + 2):
        parts = g.read_particles()
        prev = g.read_contacts() if k else None
        st = orc.State(scene)
        st.x = parts["x"].astype(np.float64)
        st.v = parts["v"].astype(np.float64)
        st.w = parts["w"].astype(np.float64)
        st.steps = k
        if prev is not None:
            st.prev_keys = prev["keys"].copy()
            st.prev_lam = prev["lam"].astype(np.float64)
            st.prev_colour = prev["colour"].astype(np.int32)
        tool = moved(scene["tool"], k)
        ref = orc.step(scene, st, tool=tool)
        g.set_tool_pose(tool)
        g.step(1)
        out = g.read_contacts()
        after = g.read_particles()
        stats = g.stats()
        assert np.array_equal(out["keys"], ref["keys"]), k
        assert np.array_equal(out["colour"].astype(np.int64), ref["colour"].astype(np.int64)), k
        assert stats["n_colours"] == ref["n_colours"], k
        assert rel_impulse_error(out["lam"], ref["lam"]) <= 1e-4, k
        assert np.abs(after["x"].astype(np.float64) - st.x).max() <= 1e-6, k
        if prev is not None and k % PERIOD != 0:  # incremental: persisting keys kept their colour
            pos = np.searchsorted(prev["keys"], out["keys"])
            pos = np.minimum(pos, len(prev["keys"]) - 1)
            kept = prev["keys"][pos] == out["keys"]
            assert np.array_equal(out["colour"][kept], prev["colour"][pos[kept]]), k
            checked.append((k, int(kept.sum()), int((~kept).sum()), stats["n_colours"]))
    g.close()
    print("incremental steps (step, kept, new, colours):", checked)
    assert len(checked) == PERIOD and all(n > 0 for _, _, n, _ in checked)  # steps 1-3 and 5


def run(tds, scenes, steps, graph=False, batch=False, split=None):
    import torch

    stream = torch.cuda.Stream()
    g = tds.Batch(scenes, stream=stream) if batch else tds.Scene(scenes[0], stream=stream)
    g.set_graph(graph)
    for k in range(steps):
        if split is not None and k == split:  # resume from a checkpoint in a new scene
            buf = g.save_state()
            g.close()
            g = tds.Scene(scenes[0], stream=stream)
            g.set_graph(graph)
            g.load_state(buf)
        if batch:
            g.set_tool_poses([moved(s["tool"], k) for s in scenes])
        else:
            g.set_tool_pose(moved(scenes[0]["tool"], k))
        g.step(1)
    out = [g.read_scene(q) for q in range(len(scenes))] if batch else [g.read_particles()]
    c = g.read_contacts()
    g.close()
    return out, c


def test_graph_replay_checkpoint_and_batch_keep_the_same_colourings(tds):
    steps = 2 * PERIOD + 1
    a = packed_scene(1500, 52, iters=30, recolour_every=PERIOD)
    b = packed_scene(900, 53, iters=30, mu_t=0.8, recolour_every=PERIOD)
    base, cb = run(tds, [a], steps)
    for kw in (dict(graph=True), dict(split=PERIOD + 2), dict(graph=True, split=3)):
        got, c = run(tds, [a], steps, **kw)
        for key in ("x", "v", "w"):
            assert np.array_equal(got[0][key], base[0][key]), (kw, key)
        assert np.array_equal(c["colour"], cb["colour"]), kw
    alone_b, _ = run(tds, [b], steps)
    both, _ = run(tds, [a, b], steps, graph=True, batch=True)
    for q, ref in enumerate((base[0], alone_b[0])):
        for key in ("x", "v", "w"):
            assert np.array_equal(both[q][key], ref[key]), (q, key)
