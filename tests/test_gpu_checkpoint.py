"""Checkpoint and resume: a scene created from the same description that
loads a saved state continues bit for bit like the scene that saved it
(particles, warm-start memory, tool poses, heightfield with a cutter), with
launches or graph replay; a state from another layout is refused."""

import numpy as np
import pytest

from paper_2011_00459_gb300 import scenes as S

pytestmark = pytest.mark.gpu

@pytest.fixture(scope="module")
def tds():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2011_00459_gb300 import build, tds

    build.build()
    return tds

def state(g):
    p = g.read_particles()
    return {k: p[k].copy() for k in ("x", "v", "w")}

@pytest.mark.parametrize("graph", [False, True])
def test_resume_continues_bit_for_bit(tds, graph):
    import torch

    scene = S.small(seed=4, n=1500)
    path = S.tool_path(scene, 0.3)
    a = tds.Scene(scene, stream=torch.cuda.Stream())
    a.set_graph(graph)
    a.set_solver(30, 1e-4, 0)
    a.set_tool_pose(S.parked_tool(scene))
    a.step(20)
    for k in range(5):
        a.set_tool_pose(path(k / 60.0))
        a.step(1)
    saved = a.save_state()
    assert a.stats()["steps"] == 25
    for k in range(5, 10):
        a.set_tool_pose(path(k / 60.0))
        a.step(1)
    want, want_f, want_c = state(a), a.read_tool_force(), a.read_contacts()
    a.close()

    b = tds.Scene(scene, stream=torch.cuda.Stream())
    b.set_graph(graph)
    b.set_solver(30, 1e-4, 0)
    b.load_state(saved)
    assert b.stats()["steps"] == 25
    for k in range(5, 10):
        b.set_tool_pose(path(k / 60.0))
        b.step(1)
    got, got_f, got_c = state(b), b.read_tool_force(), b.read_contacts()
    b.close()
    for key in ("x", "v", "w"):
        assert np.array_equal(got[key], want[key]), key
    assert np.array_equal(got_f[0], want_f[0]) and np.array_equal(got_c["lam"], want_c["lam"])

def test_resume_keeps_the_dug_heightfield_and_new_particles(tds):
    from tests.test_gpu_cut import CUTTER, bed, tool_at

    scene = bed(76)
    a = tds.Scene(scene)
    a.set_cutter(CUTTER)
    for k in range(4):
        a.set_tool_pose(tool_at(scene, k))
        a.step(1)
    saved = a.save_state()
    for k in range(4, 7):
        a.set_tool_pose(tool_at(scene, k))
        a.step(1)
    want, want_h, want_r = state(a), a.read_heightfield(), a.read_radii()
    a.close()
    b = tds.Scene(scene)
    b.set_cutter(CUTTER)
    b.load_state(saved)
    for k in range(4, 7):
        b.set_tool_pose(tool_at(scene, k))
        b.step(1)
    got, got_h, got_r = state(b), b.read_heightfield(), b.read_radii()
    b.close()
    assert np.array_equal(got_h[0], want_h[0]) and np.array_equal(got_h[1], want_h[1])
    assert np.array_equal(got_r, want_r) and (got_r == np.float32(CUTTER["spawn_radius"])).sum() > 50
    for key in ("x", "v", "w"):
        assert np.array_equal(got[key], want[key]), key

def test_a_state_of_another_layout_is_refused(tds):
    a = tds.Scene(S.small(seed=4, n=1500))
    saved = a.save_state()
    a.close()
    b = tds.Scene(S.small(seed=4, n=1400))
    with pytest.raises(tds.TdsError):
        b.load_state(saved)
    with pytest.raises(tds.TdsError):
        b.load_state(np.zeros(64, np.uint8))
    b.close()
