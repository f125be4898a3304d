"""ctypes wrapper of the FP64 CPU oracle (``tds_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the
benchmark's CPU-baseline leg call it; the product path never does. It imports
nothing from the CUDA package; scenes reach it as plain dictionaries of numpy
arrays (the layout written by ``paper_2011_00459_gb300.scenes``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "tds_oracle.c")

STATIC_BIT = 0x80000000


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction: the contact predicate
    is evaluated in plain IEEE float, operation by operation)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-fopenmp", "-o", _SO, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _SO


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("density", ctypes.c_double), ("young", ctypes.c_double), ("poisson", ctypes.c_double),
        ("mu_t", ctypes.c_double), ("mu_r", ctypes.c_double), ("cohesion", ctypes.c_double),
        ("mu_tool", ctypes.c_double), ("dt", ctypes.c_double), ("gravity", ctypes.c_double * 3),
        ("gamma_t", ctypes.c_double), ("gamma_r", ctypes.c_double),
        ("iters", ctypes.c_int32), ("residual_every", ctypes.c_int32), ("tol", ctypes.c_double),
        ("order", ctypes.c_int32), ("warm_start", ctypes.c_int32),
        ("shuffle_seed", ctypes.c_uint64),
        ("hf_nx", ctypes.c_int32), ("hf_ny", ctypes.c_int32),
        ("hf_x0", ctypes.c_float), ("hf_y0", ctypes.c_float), ("hf_cell", ctypes.c_float),
        ("hf_h", ctypes.POINTER(ctypes.c_float)),
        ("n_walls", ctypes.c_int32), ("walls", ctypes.POINTER(ctypes.c_float)),
        ("n_tool", ctypes.c_int32), ("tool_boxes", ctypes.POINTER(ctypes.c_float)),
        ("tool_pos", ctypes.c_float * 3), ("tool_quat", ctypes.c_float * 4),
        ("tool_vel", ctypes.c_float * 3), ("tool_angvel", ctypes.c_float * 3),
        ("restitution", ctypes.c_double), ("impact_speed", ctypes.c_double),
        ("impact_iters", ctypes.c_int32), ("threads", ctypes.c_int32),
        ("recolour_every", ctypes.c_int32),
    ]


class OrcStats(ctypes.Structure):
    _fields_ = [
        ("n_contacts", ctypes.c_int32), ("n_pp", ctypes.c_int32), ("n_static", ctypes.c_int32),
        ("n_colours", ctypes.c_int32), ("iterations", ctypes.c_int32),
        ("residual", ctypes.c_double),
        ("tool_force", ctypes.c_double * 3), ("tool_torque", ctypes.c_double * 3),
        ("impacts", ctypes.c_int32),
    ]


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        P = ctypes.POINTER
        L.orc_find_contacts.restype = ctypes.c_int32
        L.orc_find_contacts.argtypes = [P(OrcParams), ctypes.c_int32, P(ctypes.c_double),
                                        P(ctypes.c_double), ctypes.c_int32, ctypes.c_int32,
                                        P(ctypes.c_uint64)]
        L.orc_step.restype = ctypes.c_int32
        L.orc_step.argtypes = [P(OrcParams), ctypes.c_int32, P(ctypes.c_double),
                               P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double),
                               ctypes.c_int32, P(ctypes.c_uint64), P(ctypes.c_double),
                               P(ctypes.c_int32), ctypes.c_int32,
                               ctypes.c_int32, P(ctypes.c_uint64), P(ctypes.c_double),
                               P(ctypes.c_int32), P(ctypes.c_double), P(ctypes.c_double),
                               P(ctypes.c_double), P(OrcStats)]
        L.orc_priority.restype = ctypes.c_uint64
        L.orc_priority.argtypes = [ctypes.c_uint64]
        dp = P(ctypes.c_double)
        L.orc_mlp_forward.restype = None
        L.orc_mlp_forward.argtypes = [ctypes.c_int32] + [dp] * 8
        L.orc_mlp_loss_grad.restype = ctypes.c_double
        L.orc_mlp_loss_grad.argtypes = [ctypes.c_int32] + [dp] * 14
        _lib = L
    return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


class Params:
    """Marshals a scene dictionary into the C parameter struct (and keeps the
    arrays it points to alive)."""

    def __init__(self, scene: dict, tool: dict | None = None, **override):
        s = dict(scene)
        s.update(override)
        self._keep = []
        p = OrcParams()
        p.density = s["density"]; p.young = s["young"]; p.poisson = s["poisson"]
        p.mu_t = s["mu_t"]; p.mu_r = s["mu_r"]; p.cohesion = s["cohesion"]
        p.mu_tool = s.get("mu_tool", s["mu_t"])
        p.dt = s["dt"]
        for i in range(3):
            p.gravity[i] = s["gravity"][i]
        p.gamma_t = s.get("gamma_t", 1e-9); p.gamma_r = s.get("gamma_r", 1e-9)
        p.iters = int(s["iters"]); p.residual_every = int(s.get("residual_every", 1))
        p.tol = float(s.get("tol", 0.0))
        p.order = int(s.get("order", 0)); p.warm_start = int(s.get("warm_start", 1))
        p.shuffle_seed = int(s.get("shuffle_seed", 0))
        p.restitution = float(s.get("restitution", 0.0))
        p.impact_speed = float(s.get("impact_speed", 0.0))
        p.impact_iters = int(s.get("impact_iters", 0))
        p.threads = int(s.get("threads", 1))
        p.recolour_every = int(s.get("recolour_every", 1))
        hf = s.get("hf")
        if hf is not None:
            h = _f32(hf["h"]).reshape(-1)
            assert h.size == (hf["nx"] + 1) * (hf["ny"] + 1)
            self._keep.append(h)
            p.hf_nx = hf["nx"]; p.hf_ny = hf["ny"]
            p.hf_x0 = hf["x0"]; p.hf_y0 = hf["y0"]; p.hf_cell = hf["cell"]
            p.hf_h = _ptr(h, ctypes.c_float)
        walls = _f32(s.get("walls", np.zeros((0, 10))).reshape(-1, 10))
        boxes = _f32(s.get("tool_boxes", np.zeros((0, 10))).reshape(-1, 10))
        self._keep += [walls, boxes]
        p.n_walls = walls.shape[0]; p.walls = _ptr(walls, ctypes.c_float)
        p.n_tool = boxes.shape[0]; p.tool_boxes = _ptr(boxes, ctypes.c_float)
        t = tool if tool is not None else s.get("tool")
        if t is None:
            t = {"pos": (0, 0, 0), "quat": (1, 0, 0, 0), "vel": (0, 0, 0), "angvel": (0, 0, 0)}
        for i in range(3):
            p.tool_pos[i] = t["pos"][i]; p.tool_vel[i] = t["vel"][i]
            p.tool_angvel[i] = t["angvel"][i]
        for i in range(4):
            p.tool_quat[i] = t["quat"][i]
        self.c = p


def find_contacts(scene: dict, x=None, r=None, brute: bool = False, tool=None) -> np.ndarray:
    """Sorted uint64 contact keys of the current positions."""
    x = _f64(scene["x"] if x is None else x).reshape(-1, 3)
    r = _f64(scene["r"] if r is None else r)
    n = x.shape[0]
    P = Params(scene, tool)
    cap = max(64, 16 * n)
    while True:
        keys = np.zeros(cap, dtype=np.uint64)
        cnt = lib().orc_find_contacts(ctypes.byref(P.c), n, _ptr(x, ctypes.c_double),
                                      _ptr(r, ctypes.c_double), int(brute), cap,
                                      _ptr(keys, ctypes.c_uint64))
        if cnt == -1:
            cap *= 2
            continue
        if cnt < 0:
            raise RuntimeError(f"orc_find_contacts failed ({cnt})")
        return keys[:cnt].copy()


class State:
    """FP64 particle state plus the warm-start memory of the last step."""

    def __init__(self, scene: dict):
        self.x = _f64(scene["x"]).reshape(-1, 3).copy()
        self.v = _f64(scene["v"]).reshape(-1, 3).copy()
        self.w = _f64(scene["w"]).reshape(-1, 3).copy()
        self.r = _f64(scene["r"]).copy()
        self.prev_keys = np.zeros(0, dtype=np.uint64)
        self.prev_lam = np.zeros((0, 7), dtype=np.float64)
        self.prev_colour = np.zeros(0, dtype=np.int32)
        self.steps = 0  # steps taken


def step(scene: dict, state: State, tool=None, **override) -> dict:
    """Advance ``state`` by one step. Returns per-contact results in ascending
    key order (keys, lam[7], colour, delta) and the step statistics."""
    P = Params(scene, tool, **override)
    n = state.x.shape[0]
    cap = max(64, 16 * n)
    st = OrcStats()
    prev_colour = state.prev_colour
    if len(prev_colour) != len(state.prev_keys):  # colours unknown: every contact is coloured anew
        prev_colour = np.full(len(state.prev_keys), -1, np.int32)
    prev_colour = np.ascontiguousarray(prev_colour, np.int32)
    while True:
        keys = np.zeros(cap, dtype=np.uint64)
        lam = np.zeros((cap, 7), dtype=np.float64)
        col = np.zeros(cap, dtype=np.int32)
        dl = np.zeros(cap, dtype=np.float64)
        ft = np.zeros((cap, 10), dtype=np.float64)
        tg = np.zeros((cap, 3), dtype=np.float64)
        x0, v0, w0 = state.x.copy(), state.v.copy(), state.w.copy()
        rc = lib().orc_step(ctypes.byref(P.c), n, _ptr(x0, ctypes.c_double),
                            _ptr(v0, ctypes.c_double), _ptr(w0, ctypes.c_double),
                            _ptr(state.r, ctypes.c_double), len(state.prev_keys),
                            _ptr(state.prev_keys, ctypes.c_uint64),
                            _ptr(state.prev_lam, ctypes.c_double),
                            _ptr(prev_colour, ctypes.c_int32), int(state.steps), cap,
                            _ptr(keys, ctypes.c_uint64), _ptr(lam, ctypes.c_double),
                            _ptr(col, ctypes.c_int32), _ptr(dl, ctypes.c_double),
                            _ptr(ft, ctypes.c_double), _ptr(tg, ctypes.c_double),
                            ctypes.byref(st))
        if rc == -1:
            cap *= 2
            continue
        if rc != 0:
            raise RuntimeError(f"orc_step failed ({rc})")
        break
    nc = st.n_contacts
    state.x, state.v, state.w = x0, v0, w0
    state.prev_keys = keys[:nc].copy()
    state.prev_lam = lam[:nc].copy()
    state.prev_colour = col[:nc].copy()
    state.steps += 1
    return {
        "keys": keys[:nc].copy(), "lam": lam[:nc].copy(), "colour": col[:nc].copy(),
        "delta": dl[:nc].copy(), "features": ft[:nc].copy(), "targets": tg[:nc].copy(),
        "n_contacts": nc, "n_pp": st.n_pp, "n_static": st.n_static,
        "n_colours": st.n_colours, "iterations": st.iterations, "residual": st.residual,
        "tool_force": np.array(st.tool_force[:]), "tool_torque": np.array(st.tool_torque[:]),
        "impacts": st.impacts,
    }


def priority(key: int) -> int:
    return int(lib().orc_priority(ctypes.c_uint64(int(key))))


def mlp_forward(X, params: dict) -> np.ndarray:
    X = _f64(X).reshape(-1, 10)
    Y = np.zeros((X.shape[0], 3))
    w = [_f64(params[k]) for k in ("W1", "b1", "W2", "b2", "W3", "b3")]
    lib().orc_mlp_forward(X.shape[0], _ptr(X, ctypes.c_double),
                          *[_ptr(a, ctypes.c_double) for a in w], _ptr(Y, ctypes.c_double))
    return Y


def mlp_loss_grad(X, T, params: dict):
    X = _f64(X).reshape(-1, 10)
    T = _f64(T).reshape(-1, 3)
    w = [_f64(params[k]) for k in ("W1", "b1", "W2", "b2", "W3", "b3")]
    g = [np.zeros_like(a) for a in w]
    loss = lib().orc_mlp_loss_grad(X.shape[0], _ptr(X, ctypes.c_double),
                                   _ptr(T, ctypes.c_double),
                                   *[_ptr(a, ctypes.c_double) for a in w],
                                   *[_ptr(a, ctypes.c_double) for a in g])
    return loss, dict(zip(("W1", "b1", "W2", "b2", "W3", "b3"), g))
