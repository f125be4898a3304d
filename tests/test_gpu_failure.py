"""Failure handling on the GPU without a fault: a capacity overflow (the
contact writes are bounded by the capacity, the overflow is latched) makes
the step that meets it and the steps queued after it change nothing; the
next waiting call reports TDS_ERR_CAPACITY and puts the scene back at the
state before the failing step, warm-start memory included, after which the
scene steps on exactly like one that never failed."""
import numpy as np
import pytest

from paper_2011_00459_gb300 import scenes as S

pytestmark = pytest.mark.gpu

K = 12  # a K x K layer of touching spheres: 2 K (K - 1) pair contacts


@pytest.fixture(scope="module")
def tds():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2011_00459_gb300 import build, tds

    build.build()
    return tds


def layer() -> dict:
    """No gravity, no terrain: one layer of cohesive spheres of radius 0.05 m
    at 0.101 m spacing (every lattice neighbour 1 mm apart, inside the
    cohesive band, so the layer holds together), and a flat tool plate."""
    ii, jj = np.meshgrid(np.arange(K), np.arange(K), indexing="ij")
    x = np.stack([ii.ravel() * 0.101, jj.ravel() * 0.101, np.zeros(K * K)], 1)
    p = S.base_params(gravity=(0.0, 0.0, 0.0), cohesion=5000.0, iters=20,
                      tool_boxes=S.box((0.0, 0.0, 0.0), (1.0, 1.0, 0.01))[None, :])
    return S.with_particles(p, x, np.full(K * K, 0.05))


PARKED = {"pos": (0.5, 0.5, 50.0), "quat": (1.0, 0.0, 0.0, 0.0), "vel": (0.0, 0.0, 0.0), "angvel": (0.0, 0.0, 0.0)}
# the plate's lower face 2 mm into every sphere: one more contact per sphere
PRESSING = dict(PARKED, pos=(0.5, 0.5, 0.05 + 0.01 - 0.002))


def make(tds, graph: bool):
    import torch

    g = tds.Scene(layer(), stream=torch.cuda.Stream(), contacts_per_particle=2)  # capacity 2 K^2
    g.set_graph(graph)
    g.set_tool_pose(PARKED)
    return g


def state(g):
    p = g.read_particles()
    return {k: p[k].copy() for k in ("x", "v", "w")}


@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("queued", [4, 5])
def test_failed_step_rolls_back_and_the_scene_steps_on(tds, graph, queued):
    g = make(tds, graph)
    g.step(3)
    before = state(g)
    assert g.stats()["steps"] == 3
    g.set_tool_pose(PRESSING)  # 2 K (K - 1) + K^2 contacts > 2 K^2
    g.step(queued)  # the first of these overflows, the rest change nothing
    with pytest.raises(tds.TdsError) as e:
        g.synchronize()
    assert tds.STATUS[e.value.status] == "TDS_ERR_CAPACITY"
    assert g.stats()["steps"] == 3
    after = state(g)
    for k in ("x", "v", "w"):
        assert np.array_equal(after[k], before[k]), k
    # usable again: two more steps with the plate parked equal five steps of
    # a scene that never failed (warm-start memory restored as well)
    g.set_tool_pose(PARKED)
    g.step(2)
    got = state(g)
    assert g.stats()["steps"] == 5
    g.close()
    ref = make(tds, graph)
    ref.step(5)
    want = state(ref)
    ref.close()
    for k in ("x", "v", "w"):
        assert np.array_equal(got[k], want[k]), k


def test_every_waiting_call_reports_the_failure_once(tds):
    g = make(tds, False)
    g.step(1)
    g.set_tool_pose(PRESSING)
    g.step(1)
    with pytest.raises(tds.TdsError):
        g.read_particles()  # the read that meets the error reports it
    assert g.stats()["steps"] == 1  # the next call sees the restored scene
    g.synchronize()
    g.close()


@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("sync", [1, 0])
def test_waits_that_run_out_fail_the_step_and_roll_it_back(tds, graph, sync):
    """Every wait of a CTA on other CTAs (grid barriers, neighbours' progress
    flags) gives up after the scene's wait limit. With the
    limit set to 1 us, far below the waits of a normal step, the step fails:
    the next waiting call returns TDS_ERR_BARRIER_TIMEOUT, the scene is back
    at the state before that step, and with the limit restored it steps on
    exactly like a scene that never failed (no kernel is left waiting)."""
    import torch

    from tests.parity_cases import packed_scene

    scene = packed_scene(3000, 31, iters=40)

    def make_packed():
        g = tds.Scene(scene, stream=torch.cuda.Stream())
        g.set_graph(graph)
        g.set_launch_config(pgs_sync=sync)
        return g

    g = make_packed()
    g.step(2)
    assert g.launch_config()["wait_limit_us"] == 2_000_000
    g.set_launch_config(wait_limit_us=1)
    failed = None
    for _ in range(5):  # a step whose waits all end within 1 us is still a valid step
        before = state(g)
        steps0 = g.stats()["steps"]
        g.step(1)
        try:
            g.synchronize()
        except tds.TdsError as e:
            failed = e
            break
    assert failed is not None
    assert tds.STATUS[failed.status] == "TDS_ERR_BARRIER_TIMEOUT"
    assert g.stats()["steps"] == steps0
    after = state(g)
    for k in ("x", "v", "w"):
        assert np.array_equal(after[k], before[k]), k
    g.set_launch_config(wait_limit_us=2_000_000)
    g.step(2)
    got = state(g)
    total = g.stats()["steps"]
    g.close()
    ref = make_packed()
    ref.step(total)
    want = state(ref)
    ref.close()
    for k in ("x", "v", "w"):
        assert np.array_equal(got[k], want[k]), k
