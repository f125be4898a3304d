"""GPU path (through the C ABI) against the FP64 oracle on the same seeded
inputs: contact key sets and colourings bit-exact, impulses within 1e-4
relative (aggregate 2-norm over all rows), positions within 1e-6 m."""
import numpy as np
import pytest

from paper_2011_00459_gb300 import scenes as S
from tests.parity_cases import packed_scene, per_contact_impulse_error, rel_impulse_error

pytestmark = pytest.mark.gpu

IMPULSE_TOL = 1e-4
POS_TOL = 1e-6
# per contact: |Lambda_gpu - Lambda_oracle| over the contact's weight scale
# W = |g| h / (1/m_a + 1/m_b), at the 99.9th percentile of the contacts
PER_CONTACT_TOL = 1e-3


@pytest.fixture(scope="module")
def tds():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2011_00459_gb300 import build, tds

    build.build()
    return tds


def one_step(tds, orc, scene, **gpu_kw):
    st = orc.State(scene)
    ref = orc.step(scene, st)
    g = tds.Scene(scene, **gpu_kw)
    g.step(1)
    out = g.read_contacts()
    parts = g.read_particles()
    stats = g.stats()
    f, t = g.read_tool_force()
    g.close()
    return ref, st, out, parts, stats, (f, t)


def assert_parity(ref, st, out, parts, stats, scene=None):
    assert stats["n_contacts"] == ref["n_contacts"]
    assert np.array_equal(out["keys"], ref["keys"])
    assert np.array_equal(out["colour"].astype(np.int64), ref["colour"].astype(np.int64))
    assert stats["n_colours"] == ref["n_colours"]
    if ref["n_contacts"]:
        assert rel_impulse_error(out["lam"], ref["lam"]) <= IMPULSE_TOL
        if scene is not None:
            e = per_contact_impulse_error(scene, out["keys"], out["lam"], ref["lam"])
            print(f"per-contact impulse error / W: median {np.median(e):.2e}, "
                  f"99.9th pct {np.percentile(e, 99.9):.2e}, max {e.max():.2e}")
            assert np.percentile(e, 99.9) <= PER_CONTACT_TOL
    assert np.abs(parts["x"].astype(np.float64) - st.x).max() <= POS_TOL


def assert_residual_parity(stats, ref):
    """The GPU's natural-map residual after the same sweeps equals the
    oracle's within 1e-3 relative (FP32 impulses against FP64)."""
    rel = abs(stats["residual"] - ref["residual"]) / ref["residual"]
    print(f"residual after {stats['iterations']} sweeps: gpu {stats['residual']:.6e} "
          f"oracle {ref['residual']:.6e} (relative difference {rel:.2e})")
    assert stats["iterations"] == ref["iterations"]
    assert rel <= 1e-3


@pytest.mark.parametrize("n,seed,cohesion,mu_r", [
    (3000, 0, 1000.0, 0.1),     # several bucketing tiles and a ragged tail, cohesive
    (2500, 1, 0.0, 0.3),        # cohesionless, strong rolling resistance
    (777, 2, 5000.0, 0.0),      # odd size, no rolling resistance
])
def test_one_step_parity_packed(tds, orc, n, seed, cohesion, mu_r):
    scene = packed_scene(n, seed, cohesion=cohesion, mu_r=mu_r, iters=50)
    ref, st, out, parts, stats, (f, t) = one_step(tds, orc, scene)
    assert ref["n_pp"] > n and ref["n_static"] > 0
    assert_parity(ref, st, out, parts, stats, scene)
    assert_residual_parity(stats, ref)
    np.testing.assert_allclose(f, ref["tool_force"], rtol=1e-3, atol=1e-3 * (1 + np.abs(ref["tool_force"]).max()))
    np.testing.assert_allclose(t, ref["tool_torque"], rtol=1e-3, atol=1e-3 * (1 + np.abs(ref["tool_torque"]).max()))


def test_one_step_parity_library_workspace(tds, orc):
    scene = packed_scene(1200, 3, iters=20)
    ref, st, out, parts, stats, _ = one_step(tds, orc, scene, workspace="library")
    assert_parity(ref, st, out, parts, stats)


def test_residual_mode_parity(tds, orc):
    scene = packed_scene(1500, 4, iters=400, tol=1e-3)
    ref, st, out, parts, stats, _ = one_step(tds, orc, scene)
    assert np.array_equal(out["keys"], ref["keys"])
    assert stats["residual"] <= 1e-3 and ref["residual"] <= 1e-3
    # same stopping sweep within one check period
    assert abs(stats["iterations"] - ref["iterations"]) <= 5
    assert rel_impulse_error(out["lam"], ref["lam"]) <= 1e-3


def test_free_fall_without_contacts(tds, orc):
    scene = S.with_particles(S.base_params(iters=5), [[0.1, 0.2, 5.0], [3.0, 0.0, 1.0]],
                             [0.05, 0.04], [[0.3, -0.2, 1.5], [0.0, 0.0, 0.0]])
    ref, st, out, parts, stats, _ = one_step(tds, orc, scene)
    assert ref["n_contacts"] == 0 and stats["n_contacts"] == 0 and stats["n_colours"] == 0
    assert np.abs(parts["x"] - st.x).max() <= POS_TOL
    assert np.abs(parts["v"] - st.v).max() <= 1e-6


def test_particles_outside_the_grid_domain(tds, orc):
    """Particles beyond the broadphase box fall into its border cells and
    still find every contact."""
    scene = packed_scene(600, 6, iters=20)
    ref, st, out, parts, stats, _ = one_step(tds, orc, scene, domain=((0.1, 0.1, 0.1), (0.2, 0.2, 0.2)))
    assert_parity(ref, st, out, parts, stats)


def test_multi_step_warm_start(tds, orc):
    """Five steps with previous-step warm start: contact sets agree up to
    borderline pairs, impulses of common contacts within 1e-3, positions
    within 1e-5 m (FP32 state vs FP64 state)."""
    scene = packed_scene(1500, 7, iters=30)
    st = orc.State(scene)
    g = tds.Scene(scene)
    for _ in range(5):
        ref = orc.step(scene, st)
        g.step(1)
    out = g.read_contacts()
    parts = g.read_particles()
    g.close()
    common, ia, ib = np.intersect1d(out["keys"], ref["keys"], return_indices=True)
    assert len(common) >= 0.999 * max(len(out["keys"]), len(ref["keys"]))
    assert rel_impulse_error(out["lam"][ia], ref["lam"][ib]) <= 1e-3
    assert np.abs(parts["x"].astype(np.float64) - st.x).max() <= 1e-5


def test_warm_start_parity_from_identical_inputs(tds, orc):
    """Previous-step warm start at the one-step tolerances: the GPU takes a
    step, then the oracle is given exactly the GPU's FP32 state and its
    warm-start memory (keys and impulses); both take the next step, warm
    started from those impulses."""
    scene = packed_scene(3000, 21, iters=50)
    g = tds.Scene(scene)
    g.step(1)
    parts = g.read_particles()
    prev = g.read_contacts()
    st = orc.State(scene)
    st.x = parts["x"].astype(np.float64)
    st.v = parts["v"].astype(np.float64)
    st.w = parts["w"].astype(np.float64)
    st.prev_keys = prev["keys"].copy()
    st.prev_lam = prev["lam"].astype(np.float64)
    ref = orc.step(scene, st)
    g.step(1)
    out = g.read_contacts()
    parts2 = g.read_particles()
    stats = g.stats()
    g.close()
    persisted = np.isin(ref["keys"], prev["keys"]).mean()
    print(f"contacts {ref['n_contacts']}, persisting from the first step {persisted:.4f}")
    assert persisted > 0.7  # a jammed block with random velocities loses some contacts
    assert_parity(ref, st, out, parts2, stats, scene)
    assert_residual_parity(stats, ref)
    assert np.abs(parts2["v"].astype(np.float64) - st.v).max() <= 1e-4


def test_warm_start_parity_residual_mode(tds, orc):
    """The same from identical inputs, both solving to the 1e-4 residual:
    each stops at the first check below it (every 5 sweeps), within one
    check period of the other."""
    scene = packed_scene(2500, 22, iters=2000, tol=1e-4)
    g = tds.Scene(scene)
    g.set_solver(2000, 1e-4, 5)
    g.step(1)
    parts = g.read_particles()
    prev = g.read_contacts()
    st = orc.State(scene)
    st.x = parts["x"].astype(np.float64)
    st.v = parts["v"].astype(np.float64)
    st.w = parts["w"].astype(np.float64)
    st.prev_keys = prev["keys"].copy()
    st.prev_lam = prev["lam"].astype(np.float64)
    ref = orc.step(scene, st, residual_every=5)
    g.step(1)
    out = g.read_contacts()
    stats = g.stats()
    g.close()
    print(f"sweeps to 1e-4: gpu {stats['iterations']} oracle {ref['iterations']}")
    assert np.array_equal(out["keys"], ref["keys"])
    assert stats["residual"] <= 1e-4 and ref["residual"] <= 1e-4
    assert abs(stats["iterations"] - ref["iterations"]) <= 5
    assert rel_impulse_error(out["lam"], ref["lam"]) <= 1e-4


def test_steps_are_deterministic(tds):
    scene = packed_scene(2000, 8, iters=20)
    res = []
    for _ in range(2):
        g = tds.Scene(scene)
        g.step(3)
        res.append((g.read_particles(), g.read_contacts(), g.read_tool_force()))
        g.close()
    (pa, ca, fa), (pb, cb, fb) = res
    for k in ("x", "v", "w"):
        assert np.array_equal(pa[k], pb[k])
    assert np.array_equal(ca["lam"], cb["lam"])
    assert np.array_equal(fa[0], fb[0])


def test_adaptive_residual_checks_stop_like_fixed_sweeps(tds):
    """Checks scheduled from the residual's decay stop at a residual below the
    tolerance, and the state equals that many fixed sweeps bit for bit (a
    check reads, it never writes)."""
    scene = packed_scene(3000, 17, iters=2000, tol=1e-5)
    g = tds.Scene(scene)
    g.set_solver(2000, 1e-5, 0)
    g.step(1)
    st = g.stats()
    adaptive = g.read_particles()
    g.close()
    assert st["residual"] <= 1e-5 and st["iterations"] < 2000
    g = tds.Scene(scene)
    g.set_solver(st["iterations"], 0.0, 10)
    g.step(1)
    fixed = g.read_particles()
    g.close()
    for k in ("x", "v", "w"):
        assert np.array_equal(adaptive[k], fixed[k]), k
    g = tds.Scene(scene)
    g.set_solver(2000, 1e-5, 5)
    g.step(1)
    every5 = g.stats()
    g.close()
    assert every5["residual"] <= 1e-5
    print("sweeps: adaptive", st["iterations"], "every 5", every5["iterations"])
