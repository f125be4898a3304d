"""Oracle of the active-zone cut (section "Mesoscale model": the co-moving
active zone of a cutting edge, Eq. failure_plane, and the conversion of the
overlapped terrain into particles), evaluated after each step.

TEST INFRASTRUCTURE ONLY (tests, smoke check); the product path never calls it.

The active zone of a cutting edge is a wedge: bounded by the separation plane
(the blade face), the failure surface from the edge to the free surface and
the two ends of the edge. The failure plane contains the edge and rises ahead
of the blade at theta = pi/2 - (phi + beta)/2 above the horizontal (Eq.
failure_plane), phi the soil's internal friction angle, beta the inclination
of the separation plane to the horizontal.

Readings:
* a heightfield node whose point on the failure plane lies ahead of the blade
  (at least the spawn radius) and within the edge's length, and whose height is
  above that point, is lowered onto the failure plane; the removed height times
  the cell area times the bank density is added to the node's pending mass (the
  surface then coincides with the failure plane, as the section states);
* a node cut this step places particles of one radius r_s in its liberated
  column, from its new height up to the highest it has been: the j-th position
  is z_f + r_s (1 + 2j), taken first fit while it stays below that top and the
  pending mass pays for a particle, unless it lies closer than r_s to the
  plane of a terrain triangle around the node (heights after the step's cut:
  every such plane passes through the node, so the distance is
  cell (z - z_f) / den, den the largest sqrt((cell^2 + A^2) + B^2) over those
  triangles, A and B a triangle's height steps along its legs; a sphere of
  radius r_s <= cell / 2 centred above the node reaches no other triangle) or
  an active particle overlaps it ((dx^2 + dy^2) + dz^2 < (r_s + r)^2 in FP32,
  positions after the step's update); nodes are at least 2 r_s apart, so new particles never overlap each
  other; they start at rest; the rest stays pending at the node;
* new particles take dormant particles (radius 0) of the scene in increasing id
  order, nodes in index order, each node's accepted positions in order; with
  no dormant slot left the mass stays pending;
* not modelled: fluidized mass, the reverse conversion (deposition, gap
  filling), compaction.
All per-node arithmetic is FP32 in the operation order below (the GPU's), the
wedge itself FP64 rounded to FP32.
"""
from __future__ import annotations

import math

import numpy as np

f32 = np.float32


def quat_matrix(q):
    """Rotation matrix (row-major) of a quaternion (w, x, y, z), FP64."""
    w, x, y, z = (float(c) for c in q)
    s = 1.0 / math.sqrt(((w * w + x * x) + y * y) + z * z)
    w, x, y, z = w * s, x * s, y * s, z * s
    return [1.0 - 2.0 * (y * y + z * z), 2.0 * (x * y - w * z), 2.0 * (x * z + w * y),
            2.0 * (x * y + w * z), 1.0 - 2.0 * (x * x + z * z), 2.0 * (y * z - w * x),
            2.0 * (x * z - w * y), 2.0 * (y * z + w * x), 1.0 - 2.0 * (x * x + y * y)]


def _rot(R, a):
    a = [float(c) for c in np.asarray(a, np.float32)]
    return [(R[3 * i] * a[0] + R[3 * i + 1] * a[1]) + R[3 * i + 2] * a[2] for i in range(3)]


def _unit(a):
    n = math.sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2])
    return [c / n for c in a]


def wedge(tool: dict, cutter: dict, density: float) -> dict | None:
    """The wedge of a cutter on a tool pose (FP32 coefficients), or None."""
    if not cutter or float(cutter["length"]) <= 0.0:
        return None
    R = quat_matrix(tool["quat"])
    e = _rot(R, cutter["edge"])
    e0 = [float(np.float32(tool["pos"][i])) + e[i] for i in range(3)]
    u = _unit(_rot(R, cutter["dir"]))
    ns = _unit(_rot(R, cutter["normal"]))
    beta = math.acos(min(1.0, abs(ns[2])))
    theta = 0.5 * math.pi - 0.5 * (float(np.float32(cutter["phi"])) + beta)
    fh = math.sqrt(ns[0] * ns[0] + ns[1] * ns[1])
    if fh < 1e-9:
        return None
    f = [ns[0] / fh, ns[1] / fh]
    d = [math.cos(theta) * f[0], math.cos(theta) * f[1], math.sin(theta)]
    nf = [d[1] * u[2] - d[2] * u[1], d[2] * u[0] - d[0] * u[2], d[0] * u[1] - d[1] * u[0]]
    if nf[2] < 0.0:
        nf = [-c for c in nf]
    nf = _unit(nf)
    if abs(nf[2]) < 1e-6:
        return None
    rs = float(np.float32(cutter["spawn_radius"]))
    m = density * 4.0 / 3.0 * math.pi * rs * rs * rs
    return {"e0": np.array(e0, np.float32), "u": np.array(u, np.float32), "ns": np.array(ns, np.float32),
            "nf": np.array(nf, np.float32), "L": f32(cutter["length"]), "rho_b": f32(cutter["bank_density"]),
            "rs": f32(rs), "ms": f32(m), "inv_m": f32(1.0 / m), "inv_I": f32(1.0 / (0.4 * m * rs * rs)),
            "theta": theta}


def _node_den(h, cell):
    """Per node, the largest FP32 sqrt((cell^2 + A^2) + B^2) over the
    heightfield triangles that have the node as a corner. Triangles of cell
    (a, b): lower with corners (a, b), (a+1, b), (a, b+1), A and B the height
    steps from the first corner to the second and third; upper with corners
    (a+1, b+1), (a, b+1), (a+1, b), likewise."""
    ny1, nx1 = h.shape
    c2 = cell * cell
    lo_a, lo_b = h[:-1, 1:] - h[:-1, :-1], h[1:, :-1] - h[:-1, :-1]  # lower triangle of each cell
    up_a, up_b = h[1:, :-1] - h[1:, 1:], h[:-1, 1:] - h[1:, 1:]  # upper triangle of each cell
    lo = np.sqrt((c2 + lo_a * lo_a) + lo_b * lo_b).astype(np.float32)
    up = np.sqrt((c2 + up_a * up_a) + up_b * up_b).astype(np.float32)
    den = np.full((ny1, nx1), cell, np.float32)
    # lower (a, b) has corners (a, b), (a+1, b), (a, b+1); upper (a, b) has
    # (a+1, b+1), (a, b+1), (a+1, b); offsets below are (row b, column a)
    for t, (dj, di) in ((lo, (0, 0)), (lo, (0, 1)), (lo, (1, 0)), (up, (1, 1)), (up, (1, 0)), (up, (0, 1))):
        sub = den[dj:dj + ny1 - 1, di:di + nx1 - 1]
        np.maximum(sub, t, out=sub)
    return den


def cut_and_spawn(hf: dict, pending, top, W: dict, x, r):
    """One step's cut and conversion. hf: the scene's heightfield dict (heights
    "h" as of this step); pending, top: per-node pending mass and highest
    height; x, r: particle positions after the step's update and radii
    (radius 0 = dormant). Returns (heights, pending, new ids, their positions
    (float32), liberated mass)."""
    shape = (hf["ny"] + 1, hf["nx"] + 1)
    h = np.asarray(hf["h"], np.float32).reshape(shape).copy()
    pend = np.asarray(pending, np.float32).reshape(shape).copy()
    top = np.asarray(top, np.float32).reshape(shape)
    if W is None:
        return h, pend, np.zeros(0, np.int64), np.zeros((0, 3), np.float32), 0.0
    ii = np.arange(hf["nx"] + 1, dtype=np.float32)[None, :]
    jj = np.arange(hf["ny"] + 1, dtype=np.float32)[:, None]
    xs = f32(hf["x0"]) + ii * f32(hf["cell"])
    ys = f32(hf["y0"]) + jj * f32(hf["cell"])
    e0, u, ns, nf = W["e0"], W["u"], W["ns"], W["nf"]
    dx = xs - e0[0]
    dy = ys - e0[1]
    zf = e0[2] - (nf[0] * dx + nf[1] * dy) / nf[2]
    dz = zf - e0[2]
    su = (u[0] * dx + u[1] * dy) + u[2] * dz
    ahead = (ns[0] * dx + ns[1] * dy) + ns[2] * dz
    inside = (su >= f32(0)) & (su <= W["L"]) & (ahead >= W["rs"]) & (h > zf)
    dh = np.where(inside, h - zf, f32(0)).astype(np.float32)
    cell = f32(hf["cell"])
    lib = ((W["rho_b"] * dh) * cell) * cell
    pend = np.where(inside, pend + lib, pend).astype(np.float32)
    h = np.where(inside, zf, h).astype(np.float32)
    # conversion at the nodes cut this step
    den = _node_den(h, f32(hf["cell"]))
    xf = np.asarray(x, np.float32).reshape(-1, 3)
    rf = np.asarray(r, np.float32).reshape(-1)
    active = np.nonzero(rf > 0)[0]
    from scipy.spatial import cKDTree

    tree = cKDTree(xf[active].astype(np.float64)) if len(active) else None
    reach = float(W["rs"]) + (float(rf.max()) if len(rf) else 0.0) + 1e-4
    dormant = np.nonzero(rf == 0)[0]
    rs, ms = W["rs"], W["ms"]
    two_rs = f32(2) * rs
    ids, pos = [], []
    rank = 0
    for j, i in zip(*np.nonzero(inside)):  # row-major: node index order
        x0, y0, z0 = xs[0, i], ys[j, 0], h[j, i]
        rem = pend[j, i]
        accepted = []
        for q in range(64):
            z = z0 + (rs + two_rs * f32(q))
            if z + rs > top[j, i] or rem < ms:
                break
            if (cell * (z - z0)) / den[j, i] < rs:  # too close to the terrain around the node
                continue
            blocked = False
            if tree is not None:
                for k in tree.query_ball_point((float(x0), float(y0), float(z)), reach):
                    P = xf[active[k]]
                    ddx, ddy, ddz = x0 - P[0], y0 - P[1], z - P[2]
                    rr = rs + rf[active[k]]
                    if (ddx * ddx + ddy * ddy) + ddz * ddz < rr * rr:
                        blocked = True
                        break
            if blocked:
                continue
            accepted.append(z)
            rem = rem - ms
        taken = 0
        for a, z in enumerate(accepted):
            if rank + a < len(dormant):
                ids.append(int(dormant[rank + a]))
                pos.append((x0, y0, z))
                taken += 1
        rank += len(accepted)
        pend[j, i] = pend[j, i] - f32(taken) * ms
    return (h, pend, np.asarray(ids, np.int64), np.asarray(pos, np.float32).reshape(-1, 3),
            float(lib.astype(np.float64).sum()))
