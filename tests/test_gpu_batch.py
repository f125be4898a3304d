"""Batches of independent scenes and CUDA-graph replay on the GPU: every scene
of a batch against the FP64 oracle (contact keys and colourings bit-exact,
impulses within 1e-4, positions within 1e-6 m), every scene of a batch
bitwise equal to the same scene stepped alone, and graph replay bitwise equal
to kernel-by-kernel launches."""
import numpy as np
import pytest

from paper_2011_00459_gb300 import scenes as S
from tests.parity_cases import packed_scene, rel_impulse_error

pytestmark = pytest.mark.gpu

STATIC_BIT = 0x80000000


@pytest.fixture(scope="module")
def tds():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2011_00459_gb300 import build, tds

    build.build()
    return tds


def scene_part(out, o, n):
    """Contacts of the scene owning particle ids [o, o + n), keys made local."""
    keys = out["keys"].astype(np.uint64)
    a = (keys >> np.uint64(32)).astype(np.int64)
    sel = (a >= o) & (a < o + n)
    keys, lam, col = keys[sel], out["lam"][sel], out["colour"][sel]
    b = (keys & np.uint64(0xFFFFFFFF)).astype(np.int64)
    pair = (b & STATIC_BIT) == 0
    b = np.where(pair, b - o, b)
    local = ((a[sel] - o).astype(np.uint64) << np.uint64(32)) | b.astype(np.uint64)
    order = np.argsort(local, kind="stable")
    return local[order], lam[order], col[order]


def three_scenes():
    """Overlapping in space on purpose (scenes must still never interact);
    different sizes, friction, rolling resistance and tool poses."""
    return [packed_scene(900, 31, mu_t=0.5, mu_r=0.1, iters=30),
            packed_scene(1531, 32, mu_t=0.7, mu_r=0.2, iters=30),
            packed_scene(617, 33, mu_t=0.9, mu_r=0.0, iters=30)]


def moved(tool, k):
    t = dict(tool)
    t["pos"] = tuple(np.asarray(tool["pos"]) + np.asarray(tool["vel"]) * (k + 1) / 60.0)
    return t


def test_batch_scenes_match_oracle(tds, orc):
    scenes = three_scenes()
    b = tds.Batch(scenes)
    b.step(1)
    out = b.read_contacts()
    st_all = b.stats()
    for q, sc in enumerate(scenes):
        st = orc.State(sc)
        ref = orc.step(sc, st)
        o, n = int(b.offsets[q]), b.sizes[q]
        keys, lam, col = scene_part(out, o, n)
        assert np.array_equal(keys, ref["keys"]), q
        assert np.array_equal(col.astype(np.int64), ref["colour"].astype(np.int64)), q
        assert rel_impulse_error(lam, ref["lam"]) <= 1e-4, q
        parts = b.read_scene(q)
        assert np.abs(parts["x"].astype(np.float64) - st.x).max() <= 1e-6, q
    assert st_all["n_contacts"] == len(out["keys"])
    b.close()


def test_batch_equals_scenes_run_alone(tds):
    """Five steps with moving tools: positions and velocities bitwise equal,
    tool forces equal up to the summation order."""
    scenes = three_scenes()
    steps = 5
    b = tds.Batch(scenes)
    for k in range(steps):
        b.set_tool_poses([moved(s["tool"], k) for s in scenes])
        b.step(1)
    forces = b.read_tool_forces()
    for q, sc in enumerate(scenes):
        g = tds.Scene(sc)
        for k in range(steps):
            g.set_tool_pose(moved(sc["tool"], k))
            g.step(1)
        alone = g.read_particles()
        f, t = g.read_tool_force()
        g.close()
        got = b.read_scene(q)
        for key in ("x", "v", "w"):
            assert np.array_equal(got[key], alone[key]), (q, key)
        ft = np.concatenate([f, t])
        assert np.abs(forces[q] - ft).max() <= 1e-5 * max(np.abs(ft).max(), 1e-3), q
    b.close()


def test_batch_rejects_mixed_settings(tds):
    a = packed_scene(300, 1, iters=30)
    c = packed_scene(300, 2, iters=40)
    with pytest.raises(tds.TdsError):
        tds.Batch([a, c])
    d = packed_scene(300, 3, cohesion=0.0, iters=30)
    with pytest.raises(tds.TdsError):
        tds.Batch([a, d])


def run_steps(tds, scene, graph, steps=8):
    import torch

    g = tds.Scene(scene, stream=torch.cuda.Stream())
    g.set_graph(graph)
    for k in range(steps):
        if k == 4:
            g.set_solver(40, 0.0, 10)  # settings change: the graph is captured again
        g.set_tool_pose(moved(scene["tool"], k))
        g.step(1)
    parts = g.read_particles()
    f, t = g.read_tool_force()
    st = g.stats()
    contacts = g.read_contacts()
    g.close()
    return parts, np.concatenate([f, t]), st, contacts


def test_graph_replay_equals_launches(tds):
    scene = packed_scene(1200, 41, iters=30)
    p0, f0, s0, c0 = run_steps(tds, scene, False)
    p1, f1, s1, c1 = run_steps(tds, scene, True)
    for key in ("x", "v", "w"):
        assert np.array_equal(p0[key], p1[key]), key
    assert np.array_equal(c0["keys"], c1["keys"])
    assert np.array_equal(c0["lam"], c1["lam"])
    assert np.allclose(f0, f1, rtol=1e-6, atol=1e-6)
    assert s0["kernel_launches"] == s1["kernel_launches"]


def test_graph_replay_of_a_batch_in_residual_mode(tds):
    """The batched workload's beds (small instances) settle under graph
    replay with a residual target; the result equals plain launches."""
    import torch

    beds = S.batched(3, scenes=6, n_lo=800, n_hi=2500)
    results = []
    for graph in (False, True):
        b = tds.Batch(beds, stream=torch.cuda.Stream())
        b.set_graph(graph)
        b.set_tool_poses([S.parked_tool(s) for s in beds])
        b.set_solver(200, 1e-3, 10)
        b.step(10)
        results.append([b.read_scene(q)["x"] for q in range(len(beds))])
        st = b.stats()
        assert st["residual"] <= 1e-3 or st["iterations"] == 200
        b.close()
    for q in range(len(beds)):
        assert np.array_equal(results[0][q], results[1][q]), q


def test_phase_timing_under_graph_replay(tds):
    """The graph carries the phase events: every phase gets a time and the
    phases add up to the step."""
    import torch

    scene = packed_scene(1500, 42, iters=30)
    g = tds.Scene(scene, stream=torch.cuda.Stream())
    g.set_graph(True)
    g.step(2)
    g.stats()
    g.set_timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(g.stream)
    g.step(4)
    e1.record(g.stream)
    st = g.stats()
    torch.cuda.synchronize()
    total = e0.elapsed_time(e1)
    g.close()
    assert st["timed_steps"] == 4
    ph = st["phase_ms"]
    assert all(v > 0 for v in ph.values()), ph
    assert ph["pgs"] > ph["broadphase"]
    assert sum(ph.values()) <= total * 1.01 + 0.05


@pytest.mark.parametrize("graph,solver", [(False, (40, 1e-9, 5)), (True, (40, 1e-9, 5)),
                                          (False, (2000, 1e-4, 0)), (True, (2000, 1e-4, 0))])
def test_launch_shapes_give_identical_results(tds, graph, solver):
    """Neighbour synchronisation vs grid barrier, fewer solver and colouring
    CTAs, every compiled solver CTA shape (threads x contacts per thread):
    every launch shape gives the same states and impulses bit for bit
    (a batch of uneven beds, moving tools; residual checks every 5 sweeps of
    40, or solved to the 1e-4 residual with adaptive checks, where the
    residual's value decides the sweep count and must not depend on the
    shape)."""
    import torch

    beds = S.batched(5, scenes=5, n_lo=800, n_hi=4000)
    shapes = [dict(pgs_sync=1), dict(pgs_sync=0), dict(pgs_sync=1, pgs_blocks=7, colour_blocks=13),
              dict(pgs_sync=0, pgs_blocks=3), dict(pgs_sync=1, pgs_threads=512, pgs_per_thread=3),
              dict(pgs_sync=1, pgs_threads=512, pgs_per_thread=2, pgs_blocks=5),
              dict(pgs_sync=0, pgs_threads=640, pgs_per_thread=2),
              # three CTAs per SM: more CTAs than threads per CTA, so a CTA's
              # neighbour range can be wider than its threads
              dict(pgs_sync=1, pgs_threads=256, pgs_per_thread=1, pgs_blocks="max")]
    out = []
    for shape in shapes:
        b = tds.Batch(beds, stream=torch.cuda.Stream())
        b.set_graph(graph)
        if shape.get("pgs_blocks") == "max":  # every co-resident CTA of the shape
            b.set_launch_config(**dict(shape, pgs_blocks=0))
            b.set_launch_config(**dict(shape, pgs_blocks=b.launch_config()["max_pgs_blocks"]))
            assert b.launch_config()["pgs_blocks"] > shape["pgs_threads"]
        else:
            b.set_launch_config(**shape)
        b.set_tool_poses([S.parked_tool(s) for s in beds])
        b.set_solver(40, 1e-9, 5)
        b.step(6)
        b.set_solver(*solver)
        paths = [S.tool_path(s, 0.3) for s in beds]
        for k in range(4):
            b.set_tool_poses([p(0.5 + k / 60.0) for p in paths])
            b.step(1)
        c = b.read_contacts()
        x = [b.read_scene(q) for q in range(len(beds))]
        cfg = b.launch_config()
        st = b.stats()
        b.close()
        assert cfg["pgs_sync"] == shape["pgs_sync"]
        if "pgs_threads" in shape:
            assert (cfg["pgs_threads"], cfg["pgs_per_thread"]) == (shape["pgs_threads"], shape["pgs_per_thread"])
        out.append((c, x, (st["sweep_contacts_pp"], st["sweep_contacts_static"], st["residual"])))
    c0, x0, s0 = out[0]
    if solver[1] > 1e-6:
        assert s0[0] < 2000 * 4 * len(c0["keys"])  # the residual test stopped the solves
    for c, x, sw in out[1:]:
        assert sw == s0
        assert np.array_equal(c["keys"], c0["keys"])
        assert np.array_equal(c["colour"], c0["colour"])
        assert np.array_equal(c["lam"], c0["lam"])
        for q in range(len(beds)):
            for key in ("x", "v", "w"):
                assert np.array_equal(x[q][key], x0[q][key]), (q, key)


def test_launch_config_rejects_a_shape_that_is_not_compiled(tds):
    b = tds.Batch(S.batched(6, scenes=2, n_lo=800, n_hi=900))
    with pytest.raises(tds.TdsError):
        b.set_launch_config(pgs_threads=100, pgs_per_thread=1)
    cfg = b.launch_config()
    assert (cfg["pgs_threads"], cfg["pgs_per_thread"]) == tds.SHAPES[0]
    b.close()


def test_autotuner_picks_a_candidate_and_caches_it(tds, tmp_path):
    import torch

    from paper_2011_00459_gb300 import autotune

    beds = S.batched(6, scenes=4, n_lo=800, n_hi=3000)

    class Sim:
        def __init__(self):
            self.g = tds.Batch(beds, stream=torch.cuda.Stream())
            self.g.set_graph(True)
            self.g.set_tool_poses([S.parked_tool(s) for s in beds])
            self.g.set_solver(20, 1e-4, 5)
            self.g.step(3)

        def advance(self):
            self.g.step(1)

    path = str(tmp_path / "tune.json")
    sim = Sim()
    cfg0 = sim.g.launch_config()
    r = autotune.tune(sim, steps=1, sweeps=10, path=path)
    assert r["source"] == "timed"
    assert r["shape"] in autotune.candidates(cfg0, torch.cuda.get_device_properties(0).multi_processor_count)
    cfg = sim.g.launch_config()
    assert {k: cfg[k] for k in r["shape"]} == r["shape"]
    assert sim.g.solver == (20, 1e-4, 5)  # solver settings restored
    again = autotune.tune(sim, path=path)
    assert again["source"] == "cache" and again["shape"] == r["shape"]
    sim.g.close()


@pytest.mark.parametrize("graph", [False, True])
def test_every_bed_stops_at_its_own_residual(tds, graph):
    """In residual mode each bed of a batch has its own residual and stops
    sweeping at the first check where it is below the tolerance, exactly as
    when stepped alone: per bed the same sweeps, the same residual (<= tol)
    and the same state, bit for bit, over several steps with moving tools."""
    import torch

    tol, every, steps = 1e-3, 5, 3
    scenes = [packed_scene(900, 41, mu_t=0.5, mu_r=0.1, iters=3000, tol=tol),
              packed_scene(1900, 42, mu_t=0.7, mu_r=0.2, iters=3000, tol=tol),
              packed_scene(400, 43, mu_t=0.9, mu_r=0.0, iters=3000, tol=tol),
              packed_scene(1200, 44, mu_t=0.4, mu_r=0.3, iters=3000, tol=tol)]
    b = tds.Batch(scenes, stream=torch.cuda.Stream())
    b.set_graph(graph)
    b.set_solver(3000, tol, every)
    per_step = []
    for k in range(steps):
        b.set_tool_poses([moved(s["tool"], k) for s in scenes])
        b.step(1)
        per_step.append(b.read_solve())
    st = b.stats()
    for q, sc in enumerate(scenes):
        g = tds.Scene(sc, stream=torch.cuda.Stream())
        g.set_graph(graph)
        g.set_solver(3000, tol, every)
        for k in range(steps):
            g.set_tool_pose(moved(sc["tool"], k))
            g.step(1)
            alone = g.stats()
            got = per_step[k]
            assert got["sweeps"][q] == alone["iterations"], (q, k)
            assert got["residual"][q] == np.float32(alone["residual"]), (q, k)
            assert got["residual"][q] <= tol and got["sweeps"][q] < 3000, (q, k)
        a = g.read_particles()
        g.close()
        mine = b.read_scene(q)
        for key in ("x", "v", "w"):
            assert np.array_equal(mine[key], a[key]), (q, key)
    sweeps = np.stack([p["sweeps"] for p in per_step])
    print("sweeps per bed and step:", sweeps.tolist())
    assert len(set(sweeps[-1].tolist())) > 1  # the beds do stop at different sweeps
    assert st["iterations"] == sweeps[-1].max()
    assert st["residual"] == per_step[-1]["residual"].max()
    b.close()
