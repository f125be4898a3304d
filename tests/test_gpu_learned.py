"""Learned warm start on the GPU: the BF16 tensor-core network against the
FP64 oracle (forward and gradients, on BF16-rounded weights and inputs,
within the BF16 bound 1e-2), training, per-contact features and targets
against the oracle's, and the learned mode inside the step (same residual
as the plain solve; sweeps reported)."""
import numpy as np
import pytest

from paper_2011_00459_gb300 import scenes as S
from tests.parity_cases import packed_scene, rel_impulse_error

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tds():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2011_00459_gb300 import build, tds

    build.build()
    return tds


def bf16(a):
    """Round float32 values to the nearest BF16 (ties to even), as float32."""
    u = np.ascontiguousarray(np.asarray(a, np.float32)).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32)


def rand_params(tds, seed, scale=1.0):
    g = S.rng(seed)
    p = {"W1": g.normal(0, 0.4 * scale, (64, 10)), "b1": g.normal(0, 0.1, 64),
         "W2": g.normal(0, 0.2 * scale, (64, 64)), "b2": g.normal(0, 0.1, 64),
         "W3": g.normal(0, 0.2 * scale, (3, 64)), "b3": g.normal(0, 0.1, 3)}
    return tds.flatten_params(p)


def rounded(tds, flat):
    """Oracle view of the GPU's weights: matrices BF16-rounded, biases FP32."""
    p = tds.unflatten_params(flat)
    return {k: (bf16(v).astype(np.float64) if k.startswith("W") else np.float32(v).astype(np.float64))
            for k, v in p.items()}


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def test_forward_matches_oracle(tds, orc):
    flat = rand_params(tds, 1)
    X = S.rng(2).normal(0, 1, (1003, 10)).astype(np.float32)
    net = tds.Net(flat)
    Y = net.forward(X).cpu().numpy()
    Yo = orc.mlp_forward(bf16(X), rounded(tds, flat))
    assert rel(Y, Yo) <= 1e-2


def test_loss_and_gradients_match_oracle(tds, orc):
    flat = rand_params(tds, 3)
    g = S.rng(4)
    X = g.normal(0, 1, (777, 10)).astype(np.float32)
    T = g.normal(0, 1, (777, 3)).astype(np.float32)
    net = tds.Net(flat)
    loss, grad = net.loss_grad(X, T)
    loss = float(loss.item())
    grad = tds.unflatten_params(grad.cpu().numpy())
    lo, go = orc.mlp_loss_grad(bf16(X), T, rounded(tds, flat))
    assert loss == pytest.approx(lo, rel=1e-2)
    for k in go:
        assert rel(grad[k], go[k]) <= 1e-2, k


def test_training_fits_a_teacher_network(tds, orc):
    """Adam on the GPU kernels fits targets produced by a fixed teacher net."""
    teacher = rand_params(tds, 5)
    g = S.rng(6)
    X = g.normal(0, 1, (8192, 10)).astype(np.float32)
    T = orc.mlp_forward(X, tds.unflatten_params(teacher)).astype(np.float32)
    net = tds.Net(seed=7)
    first = float(net.train_step(X, T, lr=3e-3).item())
    for _ in range(400):
        last = float(net.train_step(X, T, lr=3e-3).item())
    assert last < 0.1 * first


def test_features_and_targets_match_oracle(tds, orc):
    """Recorded features and targets of two steps against the oracle's: the
    first step from identical inputs (no previous impulses), the second with
    warm-start impulses and persistence (states then differ by FP32 rounding)."""
    scene = packed_scene(2000, 12, iters=40)
    st = orc.State(scene)
    g = tds.Scene(scene)
    g.set_recording(True)
    for step in range(2):
        ref = orc.step(scene, st)
        g.step(1)
        got = g.read_training_samples()
        common, ia, ib = np.intersect1d(got["keys"], ref["keys"], return_indices=True)
        assert len(common) >= 0.999 * len(ref["keys"])
        F, Fo = got["features"][ia], ref["features"][ib]
        for col in (5, 6, 7, 9):  # persisted, coordination numbers, type: exact
            assert np.array_equal(F[:, col], Fo[:, col]), col
        if step == 1:
            assert F[:, 5].mean() > 0.5
        for col in (0, 1, 2, 3, 8):
            assert rel(F[:, col], Fo[:, col]) <= (1e-4 if step == 0 else 1e-3), col
        Tg, To = got["targets"][ia], ref["targets"][ib]
        assert rel(Tg[:, 0], To[:, 0]) <= 1e-3
        assert rel(np.hypot(Tg[:, 1], Tg[:, 2]), np.hypot(To[:, 1], To[:, 2])) <= 1e-3
    g.close()


def settled_bed(tds, seed, settle=120):
    """The small workload (2000 spheres) spawned, settled on the GPU with the
    blade parked, and its blade path over the settled surface."""
    scene = S.small(seed)
    g = tds.Scene(scene)
    g.set_tool_pose(S.parked_tool(scene))
    g.set_solver(20)
    g.step(settle)
    parts = g.read_particles()
    return g, scene, S.tool_path(scene, S.surface_level(parts["x"], scene["r"]))


def run_digging(tds, g, scene, path, steps, t0=0.5):
    """Steps with the blade moving; yields after each step."""
    for k in range(steps):
        g.set_tool_pose(path(t0 + k * scene["dt"]))
        g.step(1)
        yield k


def test_learned_warm_start_reaches_the_same_residual(tds):
    """Train on the new contacts of plain solves (previous-step warm start,
    residual 1e-6) of one settled bed being dug, then dig another seed's bed
    to residual 1e-4 with the learned and with the previous-step warm start:
    both reach it on every step; the sweeps are reported."""
    g, scene, path = settled_bed(tds, 20)
    g.set_recording(True)
    g.set_solver(3000, 1e-6, 10)
    X, T = [], []
    for _ in run_digging(tds, g, scene, path, 24):
        s = g.read_training_samples()
        X.append(s["features"])
        T.append(s["targets"])
    g.close()
    X, T = np.concatenate(X), np.concatenate(T)
    new = X[:, 5] == 0  # the network starts the contacts without previous impulses
    X, T = X[new], T[new]
    net = tds.Net(seed=1)
    order = np.random.Generator(np.random.PCG64(2)).permutation(len(X))
    X, T = X[order], T[order]
    for epoch in range(40):
        for b in range(0, len(X), 8192):
            net.train_step(X[b:b + 8192], T[b:b + 8192], lr=2e-3)
    params = net.host_params()
    sweeps = {}
    for name, warm in (("previous-step", tds.WARM_PREV), ("learned", tds.WARM_LEARNED)):
        g, scene, path = settled_bed(tds, 21)
        if warm == tds.WARM_LEARNED:
            g.set_mlp_weights(params)
            g.set_warm_start(tds.WARM_LEARNED)
        g.set_solver(6000, 1e-4, 5)
        its, res = [], []
        for _ in run_digging(tds, g, scene, path, 12):
            st = g.stats()
            its.append(st["iterations"])
            res.append(st["residual"])
        g.close()
        assert max(res) <= 1e-4, (name, res)
        sweeps[name] = its
    print("sweeps to 1e-4:", sweeps)
    assert np.mean(sweeps["learned"]) <= 2.0 * np.mean(sweeps["previous-step"])


def test_learned_steps_equal_with_and_without_recording(tds):
    """Without recording the network runs on the new contacts only (their
    features compacted first); with recording on every contact. Each row's
    prediction depends on its own features alone, so the steps are identical."""
    flat = rand_params(tds, 9, scale=0.3)
    out = []
    for record in (False, True):
        scene = packed_scene(2500, 19, iters=30)
        g = tds.Scene(scene)
        g.set_mlp_weights(flat)
        g.set_warm_start(tds.WARM_LEARNED)
        g.set_recording(record)
        path = scene["tool"]
        for k in range(4):
            t = dict(path)
            t["pos"] = tuple(np.asarray(path["pos"]) + np.asarray(path["vel"]) * k / 60.0)
            g.set_tool_pose(t)
            g.step(1)
        out.append(g.read_particles())
        g.close()
    for key in ("x", "v", "w"):
        assert np.array_equal(out[0][key], out[1][key]), key


def test_shipped_network_saves_sweeps_on_a_held_out_bed(tds):
    """What the trained network gains: the shipped weights (trained on the
    new contacts of plain solves of the small and bulldozing beds) on the
    excavation bed, a workload they never saw, dug by its bucket. Every step
    is solved to the 1e-4 residual twice from the same saved state, once
    with the network's initial impulses for the new contacts and once with
    zero (the previous-step warm start); the trajectory continues from the
    latter. Both reach the residual; the network needs fewer sweeps in total
    and in more steps than not."""
    from paper_2011_00459_gb300 import learned as LR

    scene = S.excavation(seed=3)
    g = tds.Scene(scene)
    g.set_tool_pose(S.parked_tool(scene))
    g.set_solver(30)
    g.step(150)
    path = S.tool_path(scene, S.surface_level(g.read_particles()["x"], scene["r"]), seed=3)
    g.set_solver(3000, 1e-4, 0)
    g.set_mlp_weights(LR.load_weights())
    t0 = 0.3 * path.length / path.speed
    k = 0
    while k * scene["dt"] < t0:
        g.set_tool_pose(path(k * scene["dt"]))
        g.step(1)
        k += 1
    prev, learned, res = [], [], []
    for _ in range(8):
        saved = g.save_state()
        g.set_tool_pose(path(k * scene["dt"]))
        g.set_warm_start(tds.WARM_LEARNED)
        g.step(1)
        st = g.stats()
        learned.append(st["iterations"])
        res.append(st["residual"])
        g.load_state(saved)  # (the state holds the tool pose of the save: set this step's again)
        g.set_tool_pose(path(k * scene["dt"]))
        g.set_warm_start(tds.WARM_PREV)
        g.step(1)
        st = g.stats()
        prev.append(st["iterations"])
        res.append(st["residual"])
        k += 1
    g.close()
    prev, learned = np.array(prev), np.array(learned)
    print("sweeps to 1e-4 on the held-out bed: previous step", prev.tolist(), "learned", learned.tolist())
    assert max(res) <= 1e-4
    assert learned.sum() < prev.sum()
    assert (learned < prev).sum() > (learned > prev).sum()
