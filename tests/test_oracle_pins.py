"""Pins of the FP64 oracle against what the paper and mechanics fix.

Each test checks the oracle against something other than itself: published
test vectors, closed forms of rigid-body mechanics (free fall, Hertz
equilibrium, Coulomb sliding, slide-to-roll, rolling resistance, cohesive
hanging), conservation laws, brute force, and the definitions of the
colouring. A plausible slip in the oracle (a dropped term, a sign, a
transposed lever arm) breaks at least one of them.
"""
import math
import os

import numpy as np
import pytest

from paper_2011_00459_gb300 import scenes as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
H = 1.0 / 60.0
GZ = 9.81


def mass(r, rho=S.RHO):
    r = float(r)
    return rho * 4.0 / 3.0 * math.pi * r ** 3


def kn_static(r):
    r = float(r)
    return S.E_YOUNG / (1 - S.NU ** 2) * math.sqrt(2 * r) / 3.0


def kn_pair(ra, rb):
    estar = S.E_YOUNG / (2 * (1 - S.NU ** 2))
    dstar = 1.0 / (1.0 / (2 * ra) + 1.0 / (2 * rb))
    return estar * math.sqrt(dstar) / 3.0


def run(orc, scene, steps, **kw):
    st = orc.State(scene)
    res = None
    for _ in range(steps):
        res = orc.step(scene, st, **kw)
    return st, res


# --------------------------------------------------------------------------
# published vectors
# --------------------------------------------------------------------------

def test_priority_matches_splitmix64_vectors(orc):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64.txt"))
            if l.strip() and not l.startswith("#")]
    golden = 0x9E3779B97F4A7C15
    for idx, out in rows:
        key = ((int(idx) - 1) * golden) % (1 << 64)
        assert orc.priority(key) == int(out, 16)


def test_rolling_polygon_values():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "rolling_polygon.txt"))
            if l.strip() and not l.startswith("#")]
    for n, printed in rows:
        mu = 0.0 if n == "inf" else 0.25 * math.tan(math.pi / (2 * int(n)))
        assert abs(mu - float(printed)) < 0.005


# --------------------------------------------------------------------------
# contact detection
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed,cohesion", [(0, 0.0), (1, 1000.0), (2, 5000.0)])
def test_grid_contacts_equal_brute_force(orc, seed, cohesion):
    x, r, v, w = S.packed_block(400, 0.02, 0.03, seed)
    p = S.base_params(cohesion=cohesion, hf=S.rough_heightfield(16, 16, -0.1, -0.1, 0.05, 0.02, 0.4, seed),
                      walls=S.bed_walls(0.4, 0.4, 1.0, 0.0, 0.0),
                      tool_boxes=S.blade(0.3, 0.2, 0.02))
    p["tool"] = {"pos": (0.2, 0.2, 0.15), "quat": S.quat_axis_angle((0, 0, 1), 0.3),
                 "vel": (0.5, 0, 0), "angvel": (0, 0, 0)}
    s = S.with_particles(p, x, r, v, w)
    kb = orc.find_contacts(s, brute=True)
    kg = orc.find_contacts(s)
    assert len(kb) > 500
    assert np.array_equal(kb, kg)


def test_pair_predicate_matches_exact_distance(orc):
    """The FP32 predicate agrees with the FP64 distance test on every pair
    except those within 1e-6 m of the reach (borderline)."""
    x, r, _, _ = S.packed_block(300, 0.02, 0.03, 5)
    s = S.with_particles(S.base_params(cohesion=1000.0), x, r)
    keys = set(int(k) for k in orc.find_contacts(s, brute=True))
    X = x.astype(np.float64)
    R = r.astype(np.float64)
    bad = 0
    for a in range(len(r)):
        d = np.linalg.norm(X[a + 1:] - X[a], axis=1)
        reach = 1.025 * (R[a] + R[a + 1:])
        for j in np.nonzero(np.abs(d - reach) > 1e-6)[0]:
            b = a + 1 + j
            bad += ((d[j] < reach[j]) != (((a << 32) | b) in keys))
    assert bad == 0


def test_heightfield_and_box_predicates_match_exact_geometry(orc):
    """Static predicates against the FP64 distance to a tilted plane and to a
    rotated box (centre inside the box included)."""
    g = S.rng(3)
    n = 400
    slope = 0.3
    hf = S.flat_heightfield(20, 20, -1.0, -1.0, 0.1)
    X, Y = np.meshgrid(-1.0 + 0.1 * np.arange(21), -1.0 + 0.1 * np.arange(21))
    hf["h"] = (slope * X + 0.1 * Y).astype(np.float32)
    bx = S.box((0.3, -0.2, 0.5), (0.2, 0.1, 0.15), S.quat_axis_angle((1, 1, 0), 0.5))
    x = np.stack([g.uniform(-0.9, 0.9, n), g.uniform(-0.9, 0.9, n), g.uniform(-0.3, 0.9, n)], 1)
    r = g.uniform(0.02, 0.06, n)
    s = S.with_particles(S.base_params(cohesion=0.0, hf=hf, walls=bx[None]), x, r)
    keys = set(int(k) for k in orc.find_contacts(s, brute=True))
    nrm = np.array([-slope, -0.1, 1.0]) / math.sqrt(1 + slope ** 2 + 0.01)
    q = bx[3:7].astype(np.float64)
    w_, i_, j_, k_ = q / np.linalg.norm(q)
    Rm = np.array([[1 - 2 * (j_ * j_ + k_ * k_), 2 * (i_ * j_ - w_ * k_), 2 * (i_ * k_ + w_ * j_)],
                   [2 * (i_ * j_ + w_ * k_), 1 - 2 * (i_ * i_ + k_ * k_), 2 * (j_ * k_ - w_ * i_)],
                   [2 * (i_ * k_ - w_ * j_), 2 * (j_ * k_ + w_ * i_), 1 - 2 * (i_ * i_ + j_ * j_)]])
    checked_hf = checked_box = 0
    for a in range(n):
        p = x[a].astype(np.float64)
        sd = float(np.dot(nrm, p - np.array([0.0, 0.0, 0.0])))
        if abs(sd - r[a]) > 1e-5:
            checked_hf += 1
            assert ((sd < r[a]) == (((a << 32) | S_BIT | 0) in keys)), a
        loc = Rm.T @ (p - bx[:3])
        cl = np.clip(loc, -bx[7:10], bx[7:10])
        dist = np.linalg.norm(loc - cl)
        if abs(dist - r[a]) > 1e-5:
            checked_box += 1
            assert ((dist < r[a]) == (((a << 32) | S_BIT | 1) in keys)), a
    assert checked_hf > 350 and checked_box > 350
    assert any(((a << 32) | S_BIT | 1) in keys for a in range(n))


S_BIT = 0x80000000


# --------------------------------------------------------------------------
# closed forms of single-body mechanics
# --------------------------------------------------------------------------

def test_free_fall_is_symplectic_euler(orc):
    """x_{n+1} = x_n + h v_{n+1} with v_{n+1} = v_n + h g: after n steps
    v = v0 + n h g and x = x0 + n h v0 + h^2 g n(n+1)/2."""
    v0 = np.array([0.3, -0.2, 1.5])
    x0 = np.array([0.1, 0.2, 5.0])
    s = S.with_particles(S.base_params(iters=5), [x0], [0.05], [v0])
    st, _ = run(orc, s, 40)
    n = 40
    g = np.array(S.G)
    x0f = x0.astype(np.float32).astype(np.float64)
    v0f = v0.astype(np.float32).astype(np.float64)
    np.testing.assert_allclose(st.v[0], v0f + n * H * g, rtol=0, atol=1e-12)
    np.testing.assert_allclose(st.x[0], x0f + n * H * v0f + H * H * g * n * (n + 1) / 2,
                               rtol=0, atol=1e-12)


def test_resting_sphere_hertz_equilibrium(orc):
    """At rest on flat ground, the physical normal force equals the weight
    and the overlap is the Hertz overlap (m g / k_n)^{2/3}."""
    r = 0.05
    s = S.with_particles(S.base_params(hf=S.flat_heightfield(4, 4, -1, -1, 0.5), iters=20),
                         [[0.0, 0.0, r]], [r])
    st, res = run(orc, s, 240)
    m = mass(np.float32(r))
    assert res["lam"][0, 0] / H == pytest.approx(m * GZ, rel=1e-9)
    assert res["delta"][0] == pytest.approx((m * GZ / kn_static(np.float32(r))) ** (2 / 3), rel=1e-6)
    assert abs(st.v[0, 2]) < 1e-9


def test_resting_column_forces_and_overlaps(orc):
    """K equal spheres stacked on flat ground: the j-th contact from the top
    carries j m g h, the ground K m g h, and each pair overlap is the Hertz
    overlap of its load."""
    K, r = 5, 0.05
    x = [[0.0, 0.0, r + 2 * r * k] for k in range(K)]
    s = S.with_particles(S.base_params(hf=S.flat_heightfield(4, 4, -1, -1, 0.5), mu_t=0.5,
                                       iters=400, tol=1e-12, residual_every=5),
                         x, [r] * K)
    st, res = run(orc, s, 300)
    assert res["residual"] < 1e-8
    m = mass(np.float32(r))
    rf = float(np.float32(r))
    keys = res["keys"]
    for j in range(1, K):
        a = K - 1 - j
        idx = int(np.nonzero(keys == ((a << 32) | (a + 1)))[0][0])
        assert res["lam"][idx, 0] == pytest.approx(j * m * GZ * H, rel=1e-6)
        assert res["delta"][idx] == pytest.approx((j * m * GZ / kn_pair(rf, rf)) ** (2 / 3), rel=1e-5)
    g = int(np.nonzero(keys == ((0 << 32) | S_BIT))[0][0])
    assert res["lam"][g, 0] == pytest.approx(K * m * GZ * H, rel=1e-6)


def _slope_scene(theta, mu, mu_r, r=0.05):
    hf = S.flat_heightfield(40, 4, -2.0, -0.2, 0.1)
    X = -2.0 + 0.1 * np.arange(41)
    hf["h"][:] = (-math.tan(theta) * X)[None, :].astype(np.float32)
    nrm = np.array([math.sin(theta), 0.0, math.cos(theta)])
    c = np.array([0.0, 0.0, 0.0]) + r * nrm
    return S.with_particles(S.base_params(hf=hf, mu_t=mu, mu_r=mu_r, iters=60), [c], [r])


@pytest.mark.parametrize("theta_deg,mu", [(20.0, 0.5), (30.0, 0.3)])
def test_sliding_block_friction_limit(orc, theta_deg, mu):
    """Rolling locked (large mu_r): the sphere rests iff tan(theta) <= mu,
    otherwise slides with a = g (sin(theta) - mu cos(theta))."""
    th = math.radians(theta_deg)
    s = _slope_scene(th, mu, 100.0)
    st = orc.State(s)
    for _ in range(30):
        orc.step(s, st)
    v1 = st.v[0].copy()
    for _ in range(30):
        orc.step(s, st)
    v2 = st.v[0].copy()
    down = np.array([math.cos(th), 0.0, -math.sin(th)])  # downhill along the slope (z falls with x)
    if math.tan(th) <= mu:
        assert np.linalg.norm(v2) < 1e-6
    else:
        a = np.dot(v2 - v1, down) / (30 * H)
        assert a == pytest.approx(GZ * (math.sin(th) - mu * math.cos(th)), rel=2e-3)
        assert abs(np.linalg.norm(st.w[0])) < 1e-3


def test_slide_to_roll(orc):
    """mu_r = 0, launched sliding with no spin: friction decelerates it until
    t* = 2 v0 / (7 mu g), after which it rolls at 5/7 v0."""
    r, v0, mu = 0.05, 2.0, 0.3
    s = S.with_particles(S.base_params(hf=S.flat_heightfield(100, 4, -1, -0.2, 0.1), mu_t=mu,
                                       mu_r=0.0, iters=50), [[0.0, 0.0, r]], [r], [[v0, 0, 0]])
    st = orc.State(s)
    tstar = 2 * v0 / (7 * mu * GZ)
    st.v[:] = 0.0
    for _ in range(60):  # come to rest on the ground first
        orc.step(s, st)
    st.v[0, 0] = v0
    for _ in range(2):
        orc.step(s, st)
    va = st.v[0, 0]
    for _ in range(5):
        orc.step(s, st)
    assert (va - st.v[0, 0]) / (5 * H) == pytest.approx(mu * GZ, rel=1e-3)
    for _ in range(int(2 * tstar / H) + 10):
        orc.step(s, st)
    assert st.v[0, 0] == pytest.approx(5.0 / 7.0 * v0, rel=2e-3)
    assert st.w[0, 1] * r == pytest.approx(st.v[0, 0], rel=2e-3)


def test_rolling_resistance_deceleration(orc):
    """Rolling without slip against a rolling-resistance torque r mu_r m g
    decelerates at (5/7) mu_r g."""
    r, v0, mur = 0.05, 1.0, 0.1
    s = S.with_particles(S.base_params(hf=S.flat_heightfield(100, 4, -1, -0.2, 0.1), mu_t=0.9,
                                       mu_r=mur, iters=50),
                         [[0.0, 0.0, r]], [r], [[v0, 0, 0]], [[0, v0 / r, 0]])
    st = orc.State(s)
    st.v[:] = 0.0
    st.w[:] = 0.0
    for _ in range(60):  # come to rest on the ground first
        orc.step(s, st)
    st.v[0, 0] = v0
    st.w[0, 1] = v0 / r
    for _ in range(3):
        orc.step(s, st)
    va = st.v[0, 0]
    for _ in range(20):
        orc.step(s, st)
    assert (va - st.v[0, 0]) / (20 * H) == pytest.approx(5.0 / 7.0 * mur * GZ, rel=2e-3)


@pytest.mark.parametrize("cp,sticks", [(2000.0, True), (1000.0, False)])
def test_cohesive_hanging_sphere(orc, cp, sticks):
    """A sphere touching the underside of a static box hangs on cohesion iff
    c_p pi r^2 >= m g; hanging, the normal impulse is the tension -m g h;
    otherwise it accelerates down at g - c_p pi r^2 / m inside the band."""
    r = 0.05
    ceiling = S.box((0.0, 0.0, 1.0), (0.5, 0.5, 0.1))
    z = 0.9 - r
    s = S.with_particles(S.base_params(cohesion=cp, walls=ceiling[None], iters=30),
                         [[0.0, 0.0, z]], [r])
    m = mass(np.float32(r))
    rf = float(np.float32(r))
    st = orc.State(s)
    res = orc.step(s, st)
    if sticks:
        for _ in range(60):
            res = orc.step(s, st)
        assert res["n_contacts"] == 1
        assert res["lam"][0, 0] == pytest.approx(-m * GZ * H, rel=1e-6)
        assert abs(st.v[0, 2]) < 1e-9
    else:
        a = -st.v[0, 2] / H
        assert a == pytest.approx(GZ - cp * math.pi * rf * rf / m, rel=1e-6)


def test_moving_tool_carries_sphere_and_feels_its_weight(orc):
    """A sphere on a tool plate moving at v_T (rolling locked) reaches v_T;
    the soil-on-tool force is then its weight (0, 0, -m g)."""
    r = 0.05
    plate = S.box((0.0, 0.0, -0.05), (2.0, 2.0, 0.05))
    tool = {"pos": (0.0, 0.0, 0.0), "quat": (1, 0, 0, 0), "vel": (0.5, 0.0, 0.0),
            "angvel": (0, 0, 0)}
    s = S.with_particles(S.base_params(tool_boxes=plate[None], tool=tool, mu_t=0.5, mu_r=100.0,
                                       iters=40), [[0.0, 0.0, r]], [r])
    st = orc.State(s)
    for _ in range(120):
        res = orc.step(s, st)
    m = mass(np.float32(r))
    assert st.v[0, 0] == pytest.approx(0.5, rel=1e-6)
    np.testing.assert_allclose(res["tool_force"], [0.0, 0.0, -m * GZ], atol=1e-6 * m * GZ)


# --------------------------------------------------------------------------
# conservation and solver structure
# --------------------------------------------------------------------------

def _momenta(st, rho=S.RHO):
    m = rho * 4.0 / 3.0 * np.pi * st.r ** 3
    I = 0.4 * m * st.r ** 2
    P = (m[:, None] * st.v).sum(0)
    L = (np.cross(st.x, m[:, None] * st.v) + I[:, None] * st.w).sum(0)
    return P, L


def test_momentum_conservation_without_gravity(orc):
    x, r, v, w = S.packed_block(300, 0.02, 0.03, 11)
    s = S.with_particles(S.base_params(gravity=(0.0, 0.0, 0.0), cohesion=2000.0, iters=30), x, r, v, w)
    st = orc.State(s)
    P0, L0 = _momenta(st)
    res = orc.step(s, st)
    assert res["n_pp"] > 200 and res["n_static"] == 0
    P1, L1 = _momenta(st)
    scale_p = np.abs(st.v).sum() * 2000 * 4 / 3 * np.pi * 0.03 ** 3
    np.testing.assert_allclose(P1, P0, atol=1e-12 * scale_p + 1e-14)
    np.testing.assert_allclose(L1, L0, atol=1e-11 * scale_p + 1e-14)


def test_one_contact_converges_in_one_sweep(orc):
    """Two spheres approaching head-on, frictionless: the single normal row
    is solved exactly by one sweep, so the residual after it vanishes and
    further sweeps change nothing."""
    r = 0.05
    x = [[0.0, 0.0, 0.0], [0.099, 0.0, 0.0]]
    v = [[0.5, 0.0, 0.0], [-0.5, 0.0, 0.0]]
    s = S.with_particles(S.base_params(gravity=(0, 0, 0), mu_t=0.0, mu_r=0.0, iters=1), x, [r, r], v)
    st1 = orc.State(s)
    r1 = orc.step(s, st1)
    st5 = orc.State(s)
    r5 = orc.step(s, st5, iters=5)
    assert r1["residual"] < 1e-14
    np.testing.assert_allclose(st1.v, st5.v, rtol=0, atol=1e-15)
    assert r1["lam"][0, 0] > 0.0
    # momentum exchange is symmetric
    np.testing.assert_allclose(st1.v[0], -st1.v[1], atol=1e-15)


def test_colouring_is_greedy_in_priority_order(orc):
    """Proper: no two contacts of one colour share a particle. Greedy: a
    contact of colour c has, for every c' < c, a neighbour of higher priority
    coloured c'."""
    x, r, v, w = S.packed_block(500, 0.02, 0.03, 4)
    s = S.with_particles(S.base_params(iters=1, cohesion=1000.0,
                                       hf=S.flat_heightfield(10, 10, 0, 0, 0.05, 0.05)), x, r, v, w)
    res = orc.step(s, orc.State(s))
    keys, col = res["keys"], res["colour"]
    a = (keys >> np.uint64(32)).astype(np.int64)
    lo = (keys & np.uint64(0xFFFFFFFF)).astype(np.int64)
    b = np.where(lo & S_BIT, -1, lo)
    prio = np.array([orc.priority(int(k)) for k in keys], dtype=np.uint64)
    inc = {}
    for c in range(len(keys)):
        for p in (a[c], b[c]):
            if p >= 0:
                inc.setdefault(int(p), []).append(c)
    for c in range(len(keys)):
        nb = set()
        for p in (a[c], b[c]):
            if p >= 0:
                nb.update(inc[int(p)])
        nb.discard(c)
        assert all(col[d] != col[c] for d in nb)
        higher = {int(col[d]) for d in nb if prio[d] > prio[c]}
        assert all(cc in higher for cc in range(col[c]))
    assert res["n_colours"] == col.max() + 1


def test_within_colour_order_is_bitwise_irrelevant(orc):
    x, r, v, w = S.packed_block(400, 0.02, 0.03, 8)
    s = S.with_particles(S.base_params(iters=20, cohesion=1000.0,
                                       hf=S.flat_heightfield(10, 10, 0, 0, 0.05, 0.05)), x, r, v, w)
    sa, sb = orc.State(s), orc.State(s)
    ra = orc.step(s, sa)
    rb = orc.step(s, sb, shuffle_seed=12345)
    assert np.array_equal(ra["lam"], rb["lam"])
    assert np.array_equal(sa.x, sb.x) and np.array_equal(sa.v, sb.v) and np.array_equal(sa.w, sb.w)


def test_colour_sweep_agrees_with_sequential_pgs_at_convergence(orc):
    """Colour-major and plain key-order Gauss-Seidel solve the same MCP: at a
    tight residual the per-body velocities and the total impulses agree."""
    x, r, v, w = S.packed_block(120, 0.02, 0.03, 9, vel_scale=0.05)
    s = S.with_particles(S.base_params(iters=20000, tol=1e-10, residual_every=10, mu_t=0.5,
                                       hf=S.flat_heightfield(10, 10, 0, 0, 0.05, 0.05)), x, r, v, w)
    sa, sb = orc.State(s), orc.State(s)
    ra = orc.step(s, sa)
    rb = orc.step(s, sb, order=1)
    assert ra["residual"] <= 1e-10 and rb["residual"] <= 1e-10
    assert np.linalg.norm(sa.v - sb.v) <= 1e-6 * np.linalg.norm(sa.v)
    assert np.linalg.norm(sa.w - sb.w) <= 1e-6 * np.linalg.norm(sa.w) + 1e-9
    tot_a = ra["lam"][:, 0].sum()
    tot_b = rb["lam"][:, 0].sum()
    assert tot_a == pytest.approx(tot_b, rel=1e-6)


def test_warm_start_restart_is_stationary(orc):
    """A converged step, re-solved from its own impulses with zero sweeps'
    worth of change, stays converged: warm start maps keys and tangent
    impulses correctly."""
    K, r = 3, 0.05
    x = [[0.0, 0.0, r + 2 * r * k] for k in range(K)]
    s = S.with_particles(S.base_params(hf=S.flat_heightfield(4, 4, -1, -1, 0.5), iters=300,
                                       tol=1e-12, residual_every=5), x, [r] * K)
    st, res = run(orc, s, 200)
    res2 = orc.step(s, st, iters=1, tol=0.0)
    assert res2["residual"] < 1e-8
    np.testing.assert_allclose(res2["lam"][:, 0], res["lam"][:, 0], rtol=1e-8)


# --------------------------------------------------------------------------
# learned warm start: features and targets of the oracle
# --------------------------------------------------------------------------

def test_learned_features_and_targets_of_a_resting_column(orc):
    """K equal spheres at rest on flat ground: pair contact j from the top
    carries j m g h, so its target Lambda_n/W with W = (m/2) g h is 2j, the
    ground contact's (W = m g h) is K; coordination numbers, depth below the
    column top, types and the predicted normal velocity follow from the
    geometry: pairs fall together (0), the ground contact approaches at g h
    (feature -1)."""
    K, r = 4, 0.05
    x = [[0.0, 0.0, r + 2 * r * k] for k in range(K)]
    s = S.with_particles(S.base_params(hf=S.flat_heightfield(4, 4, -1, -1, 0.5), mu_t=0.5,
                                       iters=400, tol=1e-12, residual_every=5), x, [r] * K)
    st, res = run(orc, s, 300)
    F, T, keys = res["features"], res["targets"], res["keys"]
    for j in range(1, K):
        a = K - 1 - j
        i = int(np.nonzero(keys == ((a << 32) | (a + 1)))[0][0])
        assert T[i, 0] == pytest.approx(2.0 * j, rel=1e-6)
        assert F[i, 2] == pytest.approx(2.0 * j, rel=1e-6)  # previous impulse, converged
        assert abs(F[i, 0]) < 1e-6 and F[i, 5] == 1.0 and F[i, 9] == 0.0
        assert F[i, 6] == 2 and F[i, 7] == (1 if a + 1 == K - 1 else 2)
        assert F[i, 8] == pytest.approx(K - a - 0.5, abs=0.01)  # (top - z_a) / 2r, top = 2 r K
        assert F[i, 1] == pytest.approx(res["delta"][i] / (2 * r), rel=1e-6)
        assert abs(T[i, 1]) < 1e-6 and abs(T[i, 2]) < 1e-6
    g = int(np.nonzero(keys == ((0 << 32) | S_BIT))[0][0])
    assert T[g, 0] == pytest.approx(K, rel=1e-6)
    assert F[g, 0] == pytest.approx(-1.0, rel=1e-6)
    assert F[g, 9] == 1.0 and F[g, 7] == 0.0 and F[g, 6] == 2
    assert F[g, 8] == pytest.approx(K - 0.5, abs=0.01)  # the column holds all spheres


def test_learned_friction_target_opposes_the_slip(orc):
    """A sphere sliding on flat ground (rolling locked): the friction impulse
    is mu Lambda_n against the slip, so target (Lambda_t . s)/W = -mu x target
    Lambda_n/W, and the normal target is 1 (W = m g h)."""
    r, mu = 0.05, 0.3
    s = S.with_particles(S.base_params(hf=S.flat_heightfield(100, 4, -1, -0.2, 0.1), mu_t=mu,
                                       mu_r=100.0, iters=60), [[0.0, 0.0, r]], [r])
    st = orc.State(s)
    for _ in range(60):
        orc.step(s, st)
    st.v[0, 0] = 2.0
    res = orc.step(s, st)
    res = orc.step(s, st)
    T, F = res["targets"][0], res["features"][0]
    assert T[0] == pytest.approx(1.0, rel=1e-3)
    assert T[1] == pytest.approx(-mu * T[0], rel=1e-6)
    assert abs(T[2]) < 1e-9
    assert F[4] == pytest.approx(-mu * F[2], rel=1e-6)  # previous friction also opposed the slip


def _mlp_params(seed):
    g = S.rng(seed)
    return {"W1": g.normal(0, 0.4, (64, 10)), "b1": g.normal(0, 0.1, 64),
            "W2": g.normal(0, 0.2, (64, 64)), "b2": g.normal(0, 0.1, 64),
            "W3": g.normal(0, 0.2, (3, 64)), "b3": g.normal(0, 0.1, 3)}


def test_mlp_backward_matches_finite_differences(orc):
    """The oracle's analytic FP64 gradients of the MSE loss against central
    differences (step 1e-6) on a 64-sample batch, for every parameter tensor."""
    g = S.rng(5)
    X = g.normal(0, 1, (64, 10))
    T = g.normal(0, 1, (64, 3))
    p = _mlp_params(6)
    loss, grads = orc.mlp_loss_grad(X, T, p)
    assert loss > 0
    for name, arr in p.items():
        flat = arr.reshape(-1)
        idx = S.rng(7).choice(flat.size, size=min(12, flat.size), replace=False)
        for i in idx:
            q = {k: v.copy() for k, v in p.items()}
            eps = 1e-6
            q[name].reshape(-1)[i] = flat[i] + eps
            lp, _ = orc.mlp_loss_grad(X, T, q)
            q[name].reshape(-1)[i] = flat[i] - eps
            lm, _ = orc.mlp_loss_grad(X, T, q)
            fd = (lp - lm) / (2 * eps)
            an = grads[name].reshape(-1)[i]
            assert abs(fd - an) <= 1e-7 * max(1.0, abs(an)) + 1e-9, (name, i, fd, an)


def test_mlp_forward_is_the_layer_formula(orc):
    """Forward pass against the three layers written with numpy matmuls."""
    g = S.rng(8)
    X = g.normal(0, 1, (32, 10))
    p = _mlp_params(9)
    Y = orc.mlp_forward(X, p)
    h1 = np.maximum(X @ p["W1"].T + p["b1"], 0)
    h2 = np.maximum(h1 @ p["W2"].T + p["b2"], 0)
    np.testing.assert_allclose(Y, h2 @ p["W3"].T + p["b3"], rtol=1e-12, atol=1e-12)


def test_threaded_colour_sweep_is_bitwise_the_serial_one(orc):
    """The CPU baseline's option of updating a colour's contacts on several
    threads changes nothing: those contacts share no particle, and the
    residual is summed in key order either way."""
    x, r, v, w = S.packed_block(600, 0.02, 0.03, 12)
    s = S.with_particles(S.base_params(iters=300, tol=1e-4, residual_every=5, cohesion=1000.0,
                                       hf=S.flat_heightfield(12, 12, 0, 0, 0.05, 0.05)), x, r, v, w)
    sa, sb = orc.State(s), orc.State(s)
    ra = orc.step(s, sa)
    rb = orc.step(s, sb, threads=4)
    assert ra["iterations"] == rb["iterations"] and ra["residual"] == rb["residual"]
    assert np.array_equal(ra["lam"], rb["lam"])
    assert np.array_equal(sa.x, sb.x) and np.array_equal(sa.v, sb.v) and np.array_equal(sa.w, sb.w)


def _greedy_violations(keys, col, prio, kept):
    """Checks of a colouring against its definition: proper, and every
    contact not kept has the smallest colour unused by its neighbours that
    are kept or of higher priority. Returns the number of violations."""
    a = (keys >> np.uint64(32)).astype(np.int64)
    lo = (keys & np.uint64(0xFFFFFFFF)).astype(np.int64)
    b = np.where(lo & S_BIT, -1, lo)
    inc = {}
    for c in range(len(keys)):
        for p in (a[c], b[c]):
            if p >= 0:
                inc.setdefault(int(p), []).append(c)
    bad = 0
    for c in range(len(keys)):
        nb = set()
        for p in (a[c], b[c]):
            if p >= 0:
                nb.update(inc[int(p)])
        nb.discard(c)
        bad += any(col[d] == col[c] for d in nb)
        if not kept[c]:
            used = {int(col[d]) for d in nb if kept[d] or prio[d] > prio[c]}
            smallest = next(k for k in range(len(nb) + 2) if k not in used)
            bad += int(col[c]) != smallest
    return bad


def test_incremental_colouring_keeps_colours_and_colours_new_contacts_greedily(orc):
    """With recolour_every = 4: steps 0 and 4 colour every contact greedily in
    priority order; steps 1-3 keep the previous colour of every persisting
    key and give each new contact the smallest colour that no kept neighbour
    and no new neighbour of higher priority uses."""
    x, r, v, w = S.packed_block(500, 0.02, 0.03, 14, vel_scale=0.3)
    s = S.with_particles(S.base_params(iters=10, cohesion=1000.0, recolour_every=4,
                                       hf=S.flat_heightfield(10, 10, 0, 0, 0.05, 0.05)), x, r, v, w)
    st = orc.State(s)
    prev = None
    new_total = 0
    for step in range(6):
        res = orc.step(s, st)
        keys, col = res["keys"], res["colour"]
        prio = np.array([orc.priority(int(k)) for k in keys], dtype=np.uint64)
        incremental = step % 4 != 0
        if incremental:
            pk, pc = prev
            pos = np.searchsorted(pk, keys)
            kept = (pos < len(pk)) & (pk[np.minimum(pos, len(pk) - 1)] == keys)
            assert np.array_equal(col[kept], pc[pos[kept]])  # persisting contacts keep their colour
            new_total += int((~kept).sum())
        else:
            kept = np.zeros(len(keys), bool)
        assert _greedy_violations(keys, col, prio, kept) == 0, step
        assert res["n_colours"] == col.max() + 1
        prev = (keys, col)
    assert new_total > 20  # the case does create new contacts in the incremental steps
