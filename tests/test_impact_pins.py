"""Pins of the oracle's impact stage (Newton impact law G_n v+ = -e G_n v-,
section "Contacting rigid multibodies") against closed-form collisions: head-on
elastic and perfectly inelastic pairs of equal and unequal spheres, a rebound
off the terrain, nothing below the impact speed, no tension in the impact
solve. The spheres start overlapping by 1e-6 m, so the main solve that
follows adds at most ~1e-5 m/s to the separating (or resting) result."""
import numpy as np
import pytest

from paper_2011_00459_gb300 import scenes as S

RHO = 2000.0


def pair_scene(ra, rb, u_a, u_b, e, v_imp=0.5, iters=10, cohesion=0.0):
    gap = 1e-6  # overlap (resolved by the FP32 contact predicate)
    x = np.array([[0.0, 0.0, 1.0], [ra + rb - gap, 0.0, 1.0]])
    v = np.array([[u_a, 0.0, 0.0], [u_b, 0.0, 0.0]])
    p = S.base_params(mu_t=0.5, mu_r=0.1, cohesion=cohesion, iters=iters, gravity=(0.0, 0.0, 0.0),
                      restitution=e, impact_speed=v_imp, impact_iters=20)
    return S.with_particles(p, x, np.array([ra, rb]), v=v)


def masses(r):
    return RHO * 4.0 / 3.0 * np.pi * np.asarray(r) ** 3


def run(orc, scene):
    st = orc.State(scene)
    out = orc.step(scene, st)
    return out, st


@pytest.mark.parametrize("ra,rb", [(0.05, 0.05), (0.05, 0.035)])
@pytest.mark.parametrize("e", [1.0, 0.0, 0.4])
def test_head_on_collisions(orc, ra, rb, e):
    ua, ub = 2.0, -1.0
    out, st = run(orc, pair_scene(ra, rb, ua, ub, e))
    assert out["impacts"] == 1
    ma, mb = masses([ra, rb])
    vc = (ma * ua + mb * ub) / (ma + mb)  # centre-of-mass velocity
    # Newton's law with momentum conservation along the line of centres
    va = vc - e * mb / (ma + mb) * (ua - ub)
    vb = vc + e * ma / (ma + mb) * (ua - ub)
    assert st.v[0, 0] == pytest.approx(va, abs=5e-5)
    assert st.v[1, 0] == pytest.approx(vb, abs=5e-5)
    assert np.abs(st.v[:, 1:]).max() < 1e-12 and np.abs(st.w).max() < 1e-12


def test_rebound_off_the_terrain(orc):
    r = 0.05
    p = S.base_params(mu_t=0.5, mu_r=0.1, cohesion=0.0, iters=10, hf=S.flat_heightfield(4, 4, -0.2, -0.2, 0.1),
                      restitution=0.5, impact_speed=0.5, impact_iters=10)
    x = np.array([[0.01, 0.02, r - 1e-6]])
    scene = S.with_particles(p, x, np.array([r]), v=np.array([[0.0, 0.0, -3.0]]))
    out, st = run(orc, scene)
    assert out["impacts"] == 1 and out["n_contacts"] == 1
    # the impact target replaces the approach, gravity of this step included
    assert st.v[0, 2] == pytest.approx(0.5 * 3.0, abs=5e-5)


def test_no_impacts_below_the_impact_speed(orc):
    a = pair_scene(0.05, 0.05, 0.2, -0.2, 1.0, v_imp=0.5)  # approach 0.4 < 0.5
    b = dict(a, impact_iters=0)
    oa, sa = run(orc, a)
    ob, sb = run(orc, b)
    assert oa["impacts"] == 0
    assert np.array_equal(sa.v, sb.v) and np.array_equal(oa["lam"], ob["lam"])


def test_impact_solve_never_pulls(orc):
    # separating fast with cohesion: no impact, and the impact solve applies no tension
    a = pair_scene(0.05, 0.05, -2.0, 2.0, 0.0, cohesion=1e4)
    oa, sa = run(orc, a)
    assert oa["impacts"] == 0
    # an impact elsewhere in the scene runs the stage; the separating pair is untouched by it
    x = np.concatenate([a["x"], [[1.0, 0.0, 1.0], [1.0 + 0.1 - 1e-6, 0.0, 1.0]]])
    v = np.concatenate([a["v"], [[3.0, 0.0, 0.0], [-3.0, 0.0, 0.0]]])
    both = S.with_particles(a, x, np.full(4, 0.05), v=v)
    ob, sb = run(orc, both)
    assert ob["impacts"] == 1
    assert np.allclose(sb.v[:2], sa.v, atol=1e-12)
