"""Seeded synthetic scene generators (inputs only; no arithmetic of the method).

Every workload is synthetic, seeded with NumPy ``PCG64(seed)``, and shaped like
the paper's bulldozing and excavation tests (section "Simulation tests"):
spherical pseudo-particles of 20-60 mm in a walled bed on a heightfield, cut
by a kinematic box tool. A scene is a plain dictionary of numpy arrays and
numbers, read identically by the CUDA binding and by the CPU oracle:

  x, v, w : (n, 3) float32   positions [m], velocities [m/s], spins [rad/s]
  r       : (n,) float32     radii [m]
  density, young, poisson, mu_t, mu_r, cohesion, mu_tool, dt, gravity(3)
  iters, tol, residual_every, warm_start
  hf      : {nx, ny, x0, y0, cell, h[(ny+1), (nx+1)] float32} or None
  walls   : (k, 10) float32  world boxes: centre(3), quaternion wxyz(4), half extents(3)
  tool_boxes : (m, 10) float32  boxes in the tool frame, same layout
  tool    : {pos, quat, vel, angvel} the tool's pose and motion this step

Particle material constants follow the paper's soil library section:
E = 1e9 Pa, nu = 0.15, restitution 0; the density is 2000 kg/m^3 for every
workload here.
"""
from __future__ import annotations

import math

import numpy as np

E_YOUNG = 1.0e9
NU = 0.15
RHO = 2000.0
G = (0.0, 0.0, -9.81)
DT = 1.0 / 60.0

WALL_T = 0.1  # wall thickness [m]


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def quat_axis_angle(axis, angle: float) -> tuple:
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    s = math.sin(0.5 * angle)
    return (math.cos(0.5 * angle), a[0] * s, a[1] * s, a[2] * s)


def box(center, half, quat=(1.0, 0.0, 0.0, 0.0)) -> np.ndarray:
    return np.array(list(center) + list(quat) + list(half), dtype=np.float32)


def base_params(**kw) -> dict:
    p = dict(density=RHO, young=E_YOUNG, poisson=NU, mu_t=0.6, mu_r=0.1, cohesion=0.0,
             dt=DT, gravity=G, iters=50, tol=0.0, residual_every=10, warm_start=1,
             hf=None, walls=np.zeros((0, 10), np.float32),
             tool_boxes=np.zeros((0, 10), np.float32),
             tool={"pos": (0.0, 0.0, 0.0), "quat": (1.0, 0.0, 0.0, 0.0),
                   "vel": (0.0, 0.0, 0.0), "angvel": (0.0, 0.0, 0.0)})
    p.update(kw)
    if "mu_tool" not in p:
        p["mu_tool"] = p["mu_t"]
    return p


def flat_heightfield(nx: int, ny: int, x0: float, y0: float, cell: float, z: float = 0.0) -> dict:
    return {"nx": nx, "ny": ny, "x0": x0, "y0": y0, "cell": cell,
            "h": np.full((ny + 1, nx + 1), z, dtype=np.float32)}


def gradient_noise(nx: int, ny: int, cell: float, wavelength: float, seed: int) -> np.ndarray:
    """2-D gradient noise on the (ny+1, nx+1) grid: unit gradients at lattice
    points of spacing ``wavelength``, quintic fade 6t^5 - 15t^4 + 10t^3
    (Perlin, "Improving noise", SIGGRAPH 2002). Values roughly in [-1, 1]."""
    g = rng(seed)
    gx = int(math.ceil(nx * cell / wavelength)) + 2
    gy = int(math.ceil(ny * cell / wavelength)) + 2
    ang = g.uniform(0.0, 2.0 * math.pi, size=(gy, gx))
    grad = np.stack([np.cos(ang), np.sin(ang)], axis=-1)
    X, Y = np.meshgrid(np.arange(nx + 1) * cell / wavelength,
                       np.arange(ny + 1) * cell / wavelength)
    i0 = np.floor(X).astype(int)
    j0 = np.floor(Y).astype(int)
    fx = X - i0
    fy = Y - j0

    def fade(t):
        return t * t * t * (t * (t * 6.0 - 15.0) + 10.0)

    def corner(di, dj):
        gr = grad[j0 + dj, i0 + di]
        return gr[..., 0] * (fx - di) + gr[..., 1] * (fy - dj)

    u, v = fade(fx), fade(fy)
    n00, n10, n01, n11 = corner(0, 0), corner(1, 0), corner(0, 1), corner(1, 1)
    nx0 = n00 + u * (n10 - n00)
    nx1 = n01 + u * (n11 - n01)
    return (nx0 + v * (nx1 - nx0)) * math.sqrt(2.0)


def rough_heightfield(nx, ny, x0, y0, cell, amplitude, wavelength, seed) -> dict:
    """Two octaves of gradient noise scaled so the largest |height| is ``amplitude``."""
    h = gradient_noise(nx, ny, cell, wavelength, seed) + 0.5 * gradient_noise(
        nx, ny, cell, 0.5 * wavelength, seed + 7919)
    h = h / max(1e-12, float(np.abs(h).max())) * amplitude
    return {"nx": nx, "ny": ny, "x0": x0, "y0": y0, "cell": cell, "h": h.astype(np.float32)}


def bed_walls(lx: float, ly: float, height: float, x0: float = 0.0, y0: float = 0.0) -> np.ndarray:
    """Four static boxes bounding the footprint [x0, x0+lx] x [y0, y0+ly]."""
    t = WALL_T
    hz = 0.5 * height
    return np.stack([
        box((x0 - 0.5 * t, y0 + 0.5 * ly, hz), (0.5 * t, 0.5 * ly + t, hz)),
        box((x0 + lx + 0.5 * t, y0 + 0.5 * ly, hz), (0.5 * t, 0.5 * ly + t, hz)),
        box((x0 + 0.5 * lx, y0 - 0.5 * t, hz), (0.5 * lx + t, 0.5 * t, hz)),
        box((x0 + 0.5 * lx, y0 + ly + 0.5 * t, hz), (0.5 * lx + t, 0.5 * t, hz)),
    ]).astype(np.float32)


def lattice_spawn(n: int, lx: float, ly: float, r_lo: float, r_hi: float, z0: float,
                  seed: int, x0: float = 0.0, y0: float = 0.0, jitter: float = 0.05):
    """n spheres with radii U[r_lo, r_hi] on a jittered cubic lattice of
    spacing 2.1 r_hi over the footprint, filled layer by layer upwards from
    z0; neighbouring spheres never touch (gap > the cohesive band)."""
    g = rng(seed)
    s = 2.1 * r_hi
    nxl = max(1, int((lx - 2.0 * r_hi) // s) + 1)
    nyl = max(1, int((ly - 2.0 * r_hi) // s) + 1)
    per = nxl * nyl
    layers = (n + per - 1) // per
    ii, jj, kk = np.meshgrid(np.arange(nxl), np.arange(nyl), np.arange(layers), indexing="ij")
    order = np.lexsort((ii.ravel(), jj.ravel(), kk.ravel()))
    ii, jj, kk = ii.ravel()[order][:n], jj.ravel()[order][:n], kk.ravel()[order][:n]
    off_x = x0 + 0.5 * (lx - (nxl - 1) * s)
    off_y = y0 + 0.5 * (ly - (nyl - 1) * s)
    x = np.stack([off_x + ii * s, off_y + jj * s, z0 + r_hi + kk * s], axis=1)
    x += g.uniform(-jitter * r_hi, jitter * r_hi, size=x.shape)
    r = g.uniform(r_lo, r_hi, size=n)
    return x.astype(np.float32), r.astype(np.float32)


def packed_block(n: int, r_lo: float, r_hi: float, seed: int, spacing: float | None = None,
                 x0=(0.0, 0.0, 0.0), shape=None, vel_scale: float = 0.2):
    """A jammed block: a jittered cubic lattice of spacing 2 r_mean, so that
    about half of the lattice neighbours overlap (by up to r_hi - r_lo) and
    the rest sit inside or outside the cohesive band. Random velocities and
    spins of magnitude ~vel_scale. Used as contact-rich one-step inputs."""
    g = rng(seed)
    s = spacing if spacing is not None else (r_lo + r_hi)
    if shape is None:
        side = int(round(n ** (1.0 / 3.0)))
        shape = (side, side, (n + side * side - 1) // (side * side))
    ii, jj, kk = np.meshgrid(*[np.arange(m) for m in shape], indexing="ij")
    pts = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=1)[:n]
    x = np.asarray(x0, dtype=np.float64) + (pts + 0.5) * s
    x += g.uniform(-0.08 * s, 0.08 * s, size=x.shape)
    r = g.uniform(r_lo, r_hi, size=n)
    v = g.normal(0.0, vel_scale, size=(n, 3))
    w = g.normal(0.0, vel_scale / r_hi, size=(n, 3))
    return (x.astype(np.float32), r.astype(np.float32), v.astype(np.float32),
            w.astype(np.float32))


def with_particles(params: dict, x, r, v=None, w=None) -> dict:
    s = dict(params)
    n = len(r)
    s["x"] = np.ascontiguousarray(np.asarray(x, np.float32).reshape(n, 3))
    s["r"] = np.ascontiguousarray(np.asarray(r, np.float32).reshape(n))
    s["v"] = np.zeros((n, 3), np.float32) if v is None else np.ascontiguousarray(
        np.asarray(v, np.float32).reshape(n, 3))
    s["w"] = np.zeros((n, 3), np.float32) if w is None else np.ascontiguousarray(
        np.asarray(w, np.float32).reshape(n, 3))
    return s


# ---------------------------------------------------------------------------
# tools and trajectories
# ---------------------------------------------------------------------------

def blade(width: float, height: float, thickness: float) -> np.ndarray:
    """A flat blade: one box, its frame at the box centre, normal along +x."""
    return box((0.0, 0.0, 0.0), (0.5 * thickness, 0.5 * width, 0.5 * height))[None, :]


def bucket(width: float = 1.2, depth: float = 1.2, height: float = 0.9) -> np.ndarray:
    """An excavator bucket from 12 boxes in its own frame (opening towards +x,
    cutting lip at the origin's front-bottom): 1 floor, 4 segments of a
    curved back, 2 sides, 1 lip and a bar of 4 teeth."""
    t = 0.03
    boxes = [box((0.5 * depth, 0.0, 0.0), (0.5 * depth, 0.5 * width, 0.5 * t))]  # floor
    # back: four plates on a quarter circle from the floor's rear up to the top
    rad = 0.5 * height
    for k in range(4):
        a0 = 0.5 * math.pi * (k + 0.5) / 4.0
        cx = -rad * math.sin(a0) + 0.0
        cz = rad - rad * math.cos(a0)
        seg = rad * math.pi / 8.0
        q = quat_axis_angle((0.0, 1.0, 0.0), -a0)
        boxes.append(box((cx, 0.0, cz + (height - rad) * (k == 3)), (0.5 * t, 0.5 * width, 0.5 * seg + 0.01), q))
    for sgn in (-1.0, 1.0):  # sides
        boxes.append(box((0.5 * depth - 0.25, sgn * 0.5 * width, 0.5 * height),
                         (0.5 * depth + 0.25, 0.5 * t, 0.5 * height)))
    boxes.append(box((depth + 0.05, 0.0, 0.0), (0.05, 0.5 * width, 0.5 * t),
                     quat_axis_angle((0.0, 1.0, 0.0), 0.3)))  # lip
    for k in range(4):  # teeth bar
        y = -0.5 * width + (k + 0.5) * width / 4.0
        boxes.append(box((depth + 0.14, y, -0.02), (0.06, 0.04, 0.02)))
    return np.stack(boxes).astype(np.float32)


def box_planes(centre, half, R=np.eye(3)) -> np.ndarray:
    """A box as 6 half-spaces (n_x, n_y, n_z, d), inside iff n . x <= d
    (centre, half extents, rotation R whose columns are the box axes)."""
    c = np.asarray(centre, np.float64)
    out = []
    for k in range(3):
        axis = np.asarray(R, np.float64)[:, k]
        for sgn in (1.0, -1.0):
            nrm = sgn * axis
            out.append([*nrm, float(nrm @ c + half[k])])
    return np.asarray(out, np.float32)


def surface_level(x: np.ndarray, r: np.ndarray, q: float = 0.95) -> float:
    """Bed surface height: the q-quantile of z + r."""
    return float(np.quantile(np.asarray(x, np.float64)[:, 2] + np.asarray(r, np.float64), q))


class BladeCycle:
    """Cut / lift / return cycle of a blade moving along +x: push ``push``
    metres at ``speed`` with the bottom ``depth`` below the surface, lift
    ``lift`` metres in ``t_lift`` s, return above the surface at ``speed``,
    lower in ``t_lift`` s, repeat."""

    def __init__(self, x_start: float, y_mid: float, surface: float, depth: float,
                 speed: float, height: float, push: float, lift: float = 0.6,
                 t_lift: float = 1.0):
        self.x_start, self.y, self.speed, self.push = x_start, y_mid, speed, push
        self.zc = surface - depth + 0.5 * height
        self.lift, self.t_lift = lift, t_lift
        t_push = push / speed
        self.phases = [t_push, t_lift, t_push, t_lift]
        self.period = sum(self.phases)

    def __call__(self, t: float) -> dict:
        tp = t % self.period
        p0, p1, p2, _ = self.phases
        if tp < p0:
            pos, vel = (self.x_start + self.speed * tp, self.y, self.zc), (self.speed, 0.0, 0.0)
        elif tp < p0 + p1:
            s = tp - p0
            pos = (self.x_start + self.push, self.y, self.zc + self.lift * s / p1)
            vel = (0.0, 0.0, self.lift / p1)
        elif tp < p0 + p1 + p2:
            s = tp - p0 - p1
            pos = (self.x_start + self.push - self.speed * s, self.y, self.zc + self.lift)
            vel = (-self.speed, 0.0, 0.0)
        else:
            s = tp - p0 - p1 - p2
            pos = (self.x_start, self.y, self.zc + self.lift - self.lift * s / self.t_lift)
            vel = (0.0, 0.0, -self.lift / self.t_lift)
        return {"pos": pos, "quat": (1.0, 0.0, 0.0, 0.0), "vel": vel, "angvel": (0.0, 0.0, 0.0)}


class SplineDig:
    """Seeded excavation path: a Catmull-Rom spline through 6 control points
    that enters the bed, drags at depth U[0.3, 0.6] m and leaves, traversed at
    a speed U[0.5, 1.2] m/s, with the bucket pitching (curling) about y as
    it goes. Loops back to the start when finished."""

    def __init__(self, x_lo: float, x_hi: float, y_mid: float, surface: float, seed: int):
        g = rng(seed)
        self.depth = float(g.uniform(0.3, 0.6))
        self.speed = float(g.uniform(0.5, 1.2))
        xs = np.linspace(x_lo, x_hi, 6)
        zs = np.array([surface + 0.4, surface - 0.3 * self.depth, surface - self.depth,
                       surface - self.depth, surface - 0.5 * self.depth, surface + 0.5])
        ys = y_mid + g.uniform(-0.2, 0.2, size=6)
        self.pts = np.stack([xs, ys, zs], axis=1)
        # arc-length table
        self.samples = self._sample(2000)
        seg = np.linalg.norm(np.diff(self.samples, axis=0), axis=1)
        self.s = np.concatenate([[0.0], np.cumsum(seg)])
        self.length = float(self.s[-1])
        self.pitch_total = 0.9  # rad of curl over the path

    def _point(self, u: float) -> np.ndarray:
        n = len(self.pts) - 1
        u = min(max(u, 0.0), n - 1e-9)
        i = int(u)
        t = u - i
        p0 = self.pts[max(i - 1, 0)]
        p1, p2 = self.pts[i], self.pts[i + 1]
        p3 = self.pts[min(i + 2, n)]
        t2, t3 = t * t, t * t * t
        return 0.5 * ((2 * p1) + (-p0 + p2) * t + (2 * p0 - 5 * p1 + 4 * p2 - p3) * t2 +
                      (-p0 + 3 * p1 - 3 * p2 + p3) * t3)

    def _sample(self, m: int) -> np.ndarray:
        n = len(self.pts) - 1
        return np.stack([self._point(n * k / (m - 1)) for k in range(m)])

    def __call__(self, t: float) -> dict:
        dist = (self.speed * t) % self.length
        k = int(np.searchsorted(self.s, dist, side="right") - 1)
        k = min(max(k, 0), len(self.samples) - 2)
        f = (dist - self.s[k]) / max(1e-12, self.s[k + 1] - self.s[k])
        pos = self.samples[k] + f * (self.samples[k + 1] - self.samples[k])
        tang = self.samples[k + 1] - self.samples[k]
        tang = tang / max(1e-12, np.linalg.norm(tang))
        frac = dist / self.length
        pitch = self.pitch_total * frac
        omega = self.pitch_total * self.speed / self.length
        return {"pos": tuple(pos), "quat": quat_axis_angle((0.0, 1.0, 0.0), -pitch),
                "vel": tuple(self.speed * tang), "angvel": (0.0, -omega, 0.0)}


# ---------------------------------------------------------------------------
# the workloads
# ---------------------------------------------------------------------------

def _spawned(params: dict, n: int, lx: float, ly: float, r_lo: float, r_hi: float,
             seed: int, z0: float) -> dict:
    x, r = lattice_spawn(n, lx, ly, r_lo, r_hi, z0, seed)
    return with_particles(params, x, r)


def small(seed: int = 0, n: int = 2000) -> dict:
    """2000 spheres, r ~ U[0.04, 0.06] m, over a walled 1 x 1 m footprint on a
    flat 32 x 32-cell heightfield (0.05 m cells), mu 0.6, mu_r 0.1, no
    cohesion, blade 0.8 x 0.3 x 0.02 m at 0.5 m/s and 0.1 m depth;
    dt = 1/60 s, 50 sweeps, 60 steps."""
    p = base_params(mu_t=0.6, mu_r=0.1, cohesion=0.0, iters=50,
                    hf=flat_heightfield(32, 32, -0.3, -0.3, 0.05),
                    walls=bed_walls(1.0, 1.0, 4.0), tool_boxes=blade(0.8, 0.3, 0.02))
    s = _spawned(p, n, 1.0, 1.0, 0.04, 0.06, seed, 0.0)
    s.update(name="small", steps=60, footprint=(1.0, 1.0), blade_speed=0.5, blade_depth=0.1,
             blade_height=0.3, tool_kind="blade", settle_steps=300)
    return s


def bulldozing(seed: int = 0, n: int = 50000) -> dict:
    """50 000 spheres, r ~ U[0.03, 0.05] m, in a walled 4 x 2 m bed on a
    128 x 64-cell heightfield (0.05 m) with +-2 cm two-octave gradient noise,
    mu 0.7, mu_r 0.1, c_p = 1 kPa, blade 2.0 x 0.37 x 0.02 m at 1 m/s and
    0.2 m depth; dt = 1/60 s, 100 sweeps, 600 steps."""
    p = base_params(mu_t=0.7, mu_r=0.1, cohesion=1000.0, iters=100,
                    hf=rough_heightfield(128, 64, -1.2, -0.6, 0.05, 0.02, 1.0, seed + 101),
                    walls=bed_walls(4.0, 2.0, 6.0), tool_boxes=blade(2.0, 0.37, 0.02))
    s = _spawned(p, n, 4.0, 2.0, 0.03, 0.05, seed, 0.05)
    s.update(name="bulldozing", steps=600, footprint=(4.0, 2.0), blade_speed=1.0,
             blade_depth=0.2, blade_height=0.37, tool_kind="blade", settle_steps=300)
    return s


def excavation(seed: int = 0, n: int = 200000) -> dict:
    """200 000 spheres, r ~ U[0.02, 0.04] m, in a walled 6 x 4 m bed on a
    256 x 256-cell heightfield (8 x 8 m), dirt-1 parameters (mu 0.4,
    mu_r 0.1, c_p 2.5 kPa), a 12-box bucket on a seeded spline dig."""
    p = base_params(mu_t=0.4, mu_r=0.1, cohesion=2500.0, iters=1000, tol=1e-4,
                    residual_every=10,
                    hf=flat_heightfield(256, 256, -1.0, -2.0, 0.03125),
                    walls=bed_walls(6.0, 4.0, 6.0), tool_boxes=bucket())
    s = _spawned(p, n, 6.0, 4.0, 0.02, 0.04, seed, 0.0)
    s.update(name="excavation", steps=300, footprint=(6.0, 4.0), tool_kind="bucket",
             settle_steps=300)
    return s


def large(seed: int = 0, n: int = 1000000) -> dict:
    """1 000 000 spheres, r ~ U[0.02, 0.03] m, in a walled 8 x 8 m bed on a
    1024 x 1024-cell heightfield over the same 8 x 8 m, excavation with the
    12-box bucket, mu 0.4, mu_r 0.1, c_p = 5 kPa, 100 sweeps."""
    p = base_params(mu_t=0.4, mu_r=0.1, cohesion=5000.0, iters=100,
                    hf=flat_heightfield(1024, 1024, 0.0, 0.0, 8.0 / 1024.0),
                    walls=bed_walls(8.0, 8.0, 8.0), tool_boxes=bucket())
    s = _spawned(p, n, 8.0, 8.0, 0.02, 0.03, seed, 0.0)
    s.update(name="large", steps=300, footprint=(8.0, 8.0), tool_kind="bucket",
             settle_steps=150)
    return s


def batched_bed(n: int, r_lo: float, r_hi: float, depth0: float, speed: float,
                blade_depth: float, mu_t: float, seed: int) -> dict:
    """One bed of a batch: n spheres on a 2:1 walled footprint sized so the
    spawn lattice is about depth0 deep, on a flat heightfield (0.05 m cells),
    mu_r 0.1, no cohesion, blade 0.8 ly x 0.3 x 0.02 m."""
    s_lat = 2.1 * r_hi
    area = n / (depth0 / s_lat) * s_lat * s_lat
    ly = max(math.sqrt(0.5 * area), 4.0 * s_lat)
    lx = 2.0 * ly
    nx = int(math.ceil((lx + 0.6) / 0.05))
    ny = int(math.ceil((ly + 0.6) / 0.05))
    p = base_params(mu_t=mu_t, mu_r=0.1, cohesion=0.0, iters=50,
                    hf=flat_heightfield(nx, ny, -0.3, -0.3, 0.05),
                    walls=bed_walls(lx, ly, 3.0 * depth0 + 2.0),
                    tool_boxes=blade(0.8 * ly, 0.3, 0.02))
    s = _spawned(p, n, lx, ly, r_lo, r_hi, seed, 0.0)
    s.update(name="batched-bed", footprint=(lx, ly), blade_speed=speed, blade_depth=blade_depth,
             blade_height=0.3, tool_kind="blade", settle_steps=300)
    return s


def batched(seed: int = 0, scenes: int = 256, n_lo: int = 1000, n_hi: int = 20000) -> list:
    """Independent beds for one batch: n ~ log-U[n_lo, n_hi] (mean ~6.3e3 for
    the defaults, ~1.6e6 spheres in 256 beds), r ~ U[0.03, 0.05] m, 2:1
    footprints 0.6 m deep before settling, blade speed U[0.2, 1.5] m/s,
    depth U[0.1, 0.4] m, mu_t U[0.4, 0.9]; dt = 1/60 s, 50 sweeps."""
    g = rng(seed)
    ns = np.exp(g.uniform(math.log(n_lo), math.log(n_hi), scenes)).astype(np.int64)
    speed = g.uniform(0.2, 1.5, scenes)
    depth = g.uniform(0.1, 0.4, scenes)
    mu = g.uniform(0.4, 0.9, scenes)
    return [batched_bed(int(ns[q]), 0.03, 0.05, 0.6, float(speed[q]), float(depth[q]), float(mu[q]),
                        1000 * seed + q + 1) for q in range(scenes)]


def bent_blade(width: float, height: float, thickness: float, angle_deg: float) -> np.ndarray:
    """A blade of two plates stacked vertically, each half the height: the
    lower one upright, the upper one turned by angle_deg about the blade's
    top edge of the lower plate, towards the pushing direction (+x)."""
    h2 = 0.5 * height
    lower = box((0.0, 0.0, -0.5 * h2), (0.5 * thickness, 0.5 * width, 0.5 * h2))
    a = math.radians(angle_deg)
    # centre of the upper plate: from the joint (0, 0, 0) along its own up axis
    up = (math.sin(a), 0.0, math.cos(a))
    upper = box((0.5 * h2 * up[0], 0.0, 0.5 * h2 * up[2]), (0.5 * thickness, 0.5 * width, 0.5 * h2),
                quat_axis_angle((0.0, 1.0, 0.0), a))
    return np.stack([lower, upper]).astype(np.float32)


def microscale(seed: int = 0, n: int = 50000) -> dict:
    """The paper's microscale reference configuration: 50 000 spheres of
    45-55 mm diameter and 2200 kg/m^3 (E 1 GPa, nu 0.15, restitution 0),
    sand-1 particle parameters (mu 0.3, mu_r 0.1, no cohesion), h = 1 ms and
    500 PGS sweeps, bulldozed by a 1.6 m wide, 0.37 m tall blade of two plates
    at 55 degrees cutting 0.05 m deep at 0.5 m/s over 5 m. The impact stage
    treats approaches faster than 0.5 m/s as impacts (20 sweeps)."""
    p = base_params(density=2200.0, young=1e9, poisson=0.15, mu_t=0.3, mu_r=0.1, cohesion=0.0,
                    dt=1e-3, iters=500, restitution=0.0, impact_speed=0.5, impact_iters=20,
                    hf=flat_heightfield(150, 50, -0.3, -0.3, 0.05),
                    walls=bed_walls(7.0, 2.0, 3.0), tool_boxes=bent_blade(1.6, 0.37, 0.02, 55.0))
    s = _spawned(p, n, 7.0, 2.0, 0.0225, 0.0275, seed, 0.0)
    s.update(name="microscale", steps=10000, footprint=(7.0, 2.0), blade_speed=0.5, blade_depth=0.05,
             blade_height=0.37, tool_kind="blade", settle_steps=600)
    return s


WORKLOADS = {"small": small, "bulldozing": bulldozing, "excavation": excavation,
             "large": large, "microscale": microscale}


def tool_path(scene: dict, surface: float, seed: int = 0):
    """The tool motion of a workload as a function of time, given the settled
    bed's surface height."""
    lx, ly = scene["footprint"]
    if scene.get("tool_kind") == "blade":
        return BladeCycle(0.1 * lx, 0.5 * ly, surface, scene["blade_depth"],
                          scene["blade_speed"], scene["blade_height"], push=0.75 * lx)
    return SplineDig(0.15 * lx, 0.85 * lx, 0.5 * ly, surface, seed)


def parked_tool(scene: dict) -> dict:
    """A tool pose far above the bed (used while the bed settles)."""
    lx, ly = scene["footprint"]
    return {"pos": (0.5 * lx, 0.5 * ly, 50.0), "quat": (1.0, 0.0, 0.0, 0.0),
            "vel": (0.0, 0.0, 0.0), "angvel": (0.0, 0.0, 0.0)}
