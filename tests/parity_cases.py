"""Seeded parity inputs shared by the GPU tests and the smoke check: contact-rich
packed blocks on a rough heightfield inside walls, cut by a moving and
turning blade (inputs only; no arithmetic of the method)."""
import math

import numpy as np

from paper_2011_00459_gb300 import scenes as S


def packed_scene(n: int, seed: int, cohesion: float = 1000.0, mu_t: float = 0.6,
                 mu_r: float = 0.1, iters: int = 50, tool: bool = True, r_lo: float = 0.02,
                 r_hi: float = 0.03, tol: float = 0.0, **extra) -> dict:
    x, r, v, w = S.packed_block(n, r_lo, r_hi, seed, vel_scale=0.1)
    lo = x.min(0) - r_hi
    hi = x.max(0) + r_hi
    lx, ly = float(hi[0] - lo[0]), float(hi[1] - lo[1])
    cell = 0.05
    nx = int(math.ceil(lx / cell)) + 2
    ny = int(math.ceil(ly / cell)) + 2
    hf = S.rough_heightfield(nx, ny, float(lo[0]) - cell, float(lo[1]) - cell, cell, 0.01, 0.4,
                             seed + 5)
    hf["h"] = hf["h"] + np.float32(lo[2] + 0.5 * r_hi)
    p = S.base_params(cohesion=cohesion, mu_t=mu_t, mu_r=mu_r, iters=iters, tol=tol,
                      residual_every=5, hf=hf,
                      walls=S.bed_walls(lx, ly, 2.0, float(lo[0]), float(lo[1])), **extra)
    if tool:
        p["tool_boxes"] = np.concatenate([S.blade(0.6 * ly, 0.2, 0.02),
                                          S.box((0.05, 0.0, 0.12), (0.04, 0.1, 0.02))[None]])
        p["tool"] = {"pos": (float(lo[0]) + 0.4 * lx, float(lo[1]) + 0.5 * ly, float(hi[2]) - 0.05),
                     "quat": S.quat_axis_angle((0.2, 1.0, 0.1), 0.35),
                     "vel": (0.6, 0.05, -0.1), "angvel": (0.1, -0.4, 0.2)}
    return S.with_particles(p, x, r, v, w)


def per_contact_impulse_error(scene: dict, keys, lam_gpu, lam_ref) -> np.ndarray:
    """|Lambda_gpu - Lambda_ref| of every contact (all 7 components) over its
    weight scale W = |g| h / (1/m_a + 1/m_b) (1/m_b = 0 for a static side)."""
    keys = np.asarray(keys, np.uint64)
    r = np.asarray(scene["r"], np.float64)
    m = scene["density"] * 4.0 / 3.0 * np.pi * r ** 3
    a = (keys >> np.uint64(32)).astype(np.int64)
    lo = (keys & np.uint64(0xFFFFFFFF)).astype(np.int64)
    static = (lo & 0x80000000) != 0
    inv = 1.0 / m[a] + np.where(static, 0.0, 1.0 / m[np.where(static, 0, lo)])
    W = np.linalg.norm(scene["gravity"]) * scene["dt"] / inv
    d = np.linalg.norm(np.asarray(lam_gpu, np.float64) - np.asarray(lam_ref, np.float64), axis=1)
    return d / W


def rel_impulse_error(lam_gpu, lam_ref) -> float:
    ref = np.asarray(lam_ref, np.float64)
    den = float(np.linalg.norm(ref))
    return float(np.linalg.norm(np.asarray(lam_gpu, np.float64) - ref)) / max(den, 1e-300)
