"""Python binding of libtds (argument marshalling only).

Every step of the particle time step runs in the CUDA library behind the C ABI
of ``include/tds.h``; this module converts scene dictionaries (see
``scenes.py``) into ``tds_scene_desc``, provides device memory and the CUDA
stream through PyTorch, and copies results back. There is no CPU fallback:
without the built library (or without a GPU) every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libtds.so")

TDS_OK = 0
STATUS = {0: "TDS_OK", -1: "TDS_ERR_INVALID_ARG", -2: "TDS_ERR_CUDA", -3: "TDS_ERR_OOM",
          -4: "TDS_ERR_CAPACITY", -5: "TDS_ERR_NONFINITE", -6: "TDS_ERR_BARRIER_TIMEOUT",
          -7: "TDS_ERR_STATE"}
MAX_BOXES = 24
STATIC_BIT = 0x80000000

EXPORTED = ["tds_workspace_bytes", "tds_create_scene", "tds_set_tool_pose", "tds_step",
            "tds_synchronize", "tds_read_particles", "tds_read_tool_force", "tds_read_contacts",
            "tds_get_stats", "tds_set_timing", "tds_set_solver", "tds_destroy_scene",
            "tds_last_error", "tds_find_pair_contacts_noalloc", "tds_mlp_param_count",
            "tds_set_mlp_weights", "tds_set_recording", "tds_read_training_samples",
            "tds_mlp_workspace_bytes", "tds_mlp_forward", "tds_mlp_loss_grad", "tds_mlp_adam_step",
            "tds_set_warm_start", "tds_batch_workspace_bytes", "tds_create_batch",
            "tds_batch_set_tool_pose", "tds_batch_read_particles", "tds_batch_read_tool_forces",
            "tds_set_graph", "tds_batch_set_tool_poses", "tds_get_launch_config",
            "tds_set_launch_config", "tds_aggregate_bodies", "tds_coarse_grain", "tds_advect_fluid",
            "tds_set_impact", "tds_set_cutter", "tds_read_heightfield", "tds_read_radii",
            "tds_state_bytes", "tds_save_state", "tds_load_state", "tds_batch_read_solve",
            "tds_set_recolour_period"]

WARM_COLD, WARM_PREV, WARM_LEARNED = 0, 1, 2
SHAPES = ((416, 1), (768, 1), (512, 2), (640, 2), (512, 3), (256, 1))  # solver CTA shapes compiled (threads, contacts per thread)


class TdsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_f = ctypes.c_float
_fp = ctypes.POINTER(ctypes.c_float)


class SceneDesc(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_uint32),
        ("x", _fp), ("y", _fp), ("z", _fp),
        ("vx", _fp), ("vy", _fp), ("vz", _fp),
        ("wx", _fp), ("wy", _fp), ("wz", _fp),
        ("radius", _fp),
        ("density", _f), ("young", _f), ("poisson", _f),
        ("mu_t", _f), ("mu_r", _f), ("cohesion", _f), ("mu_tool", _f),
        ("hf_nx", ctypes.c_uint32), ("hf_ny", ctypes.c_uint32),
        ("hf_x0", _f), ("hf_y0", _f), ("hf_cell", _f), ("hf_heights", _fp),
        ("n_walls", ctypes.c_uint32), ("walls", _fp),
        ("n_tool_boxes", ctypes.c_uint32), ("tool_boxes", _fp),
        ("dt", _f), ("gravity", _f * 3),
        ("max_iters", ctypes.c_uint32), ("tol", _f), ("residual_every", ctypes.c_uint32),
        ("warm_start", ctypes.c_int32), ("contacts_per_particle", ctypes.c_uint32),
        ("domain_lo", _f * 3), ("domain_hi", _f * 3),
        ("restitution", _f), ("impact_speed", _f), ("impact_iters", ctypes.c_uint32),
    ]


class StepStats(ctypes.Structure):
    _fields_ = [("n_contacts", ctypes.c_uint32), ("n_pp", ctypes.c_uint32),
                ("n_static", ctypes.c_uint32), ("n_colours", ctypes.c_uint32),
                ("iterations", ctypes.c_uint32), ("residual", ctypes.c_float),
                ("steps", ctypes.c_uint64), ("kernel_launches", ctypes.c_uint64),
                ("timed_steps", ctypes.c_uint32), ("phase_ms", ctypes.c_float * 5),
                ("sweep_contacts_pp", ctypes.c_uint64), ("sweep_contacts_static", ctypes.c_uint64),
                ("sum_contacts", ctypes.c_uint64), ("solved_steps", ctypes.c_uint64),
                ("colour_rounds", ctypes.c_uint32), ("impacts", ctypes.c_uint32),
                ("spawned", ctypes.c_uint32)]

PHASES = ("broadphase", "narrowphase", "colouring", "pgs", "finish")


MAX_ZONES, ZONE_MAX_PLANES = 64, 8


class Zone(ctypes.Structure):
    _fields_ = [("scene", ctypes.c_uint32), ("n_planes", ctypes.c_uint32),
                ("planes", (ctypes.c_float * 4) * ZONE_MAX_PLANES)]


class Aggregate(ctypes.Structure):
    _fields_ = [("count", ctypes.c_uint32), ("pad", ctypes.c_uint32), ("mass", ctypes.c_double),
                ("com", ctypes.c_double * 3), ("vel", ctypes.c_double * 3), ("omega", ctypes.c_double * 3),
                ("inertia", ctypes.c_double * 6)]


class Grid(ctypes.Structure):
    _fields_ = [("origin", ctypes.c_float * 3), ("l0", ctypes.c_float), ("nx", ctypes.c_uint32),
                ("ny", ctypes.c_uint32), ("nz", ctypes.c_uint32), ("scene", ctypes.c_uint32)]


def make_grid(origin, l0: float, dims, scene: int = 0) -> Grid:
    g = Grid()
    for a in range(3):
        g.origin[a] = float(origin[a])
    g.l0 = float(l0)
    g.nx, g.ny, g.nz = (int(d) for d in dims)
    g.scene = int(scene)
    return g


def advect_fluid(grid: Grid, u, rho, dt: float, source=None, out=None, stream=None):
    """One conserved upwind step of the fluidized-mass density on device
    tensors (rho: nz x ny x nx, u: nz x ny x nx x 3); returns rho_out."""
    import torch

    out = torch.empty_like(rho) if out is None else out
    st = stream if stream is not None else torch.cuda.current_stream()
    src = ctypes.c_void_p(source.data_ptr()) if source is not None else None
    _check(lib().tds_advect_fluid(ctypes.byref(grid), ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(rho.data_ptr()),
                                  src, float(dt), ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(st.cuda_stream)))
    return out


class Cutter(ctypes.Structure):
    _fields_ = [("edge", ctypes.c_float * 3), ("dir", ctypes.c_float * 3), ("length", ctypes.c_float),
                ("normal", ctypes.c_float * 3), ("phi", ctypes.c_float), ("bank_density", ctypes.c_float),
                ("spawn_radius", ctypes.c_float)]


class LaunchConfig(ctypes.Structure):
    _fields_ = [("pgs_blocks", ctypes.c_int32), ("pgs_sync", ctypes.c_int32),
                ("colour_blocks", ctypes.c_int32), ("max_pgs_blocks", ctypes.c_int32),
                ("max_colour_blocks", ctypes.c_int32), ("pgs_threads", ctypes.c_int32),
                ("pgs_per_thread", ctypes.c_int32), ("wait_limit_us", ctypes.c_int32)]


_lib = None


def lib() -> ctypes.CDLL:
    """Load libtds.so (built in-tree by ``build.build()``); raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise TdsError(-2, f"{LIB_PATH} is missing: build it with paper_2011_00459_gb300.build")
        L = ctypes.CDLL(LIB_PATH)
        vp = ctypes.c_void_p
        L.tds_workspace_bytes.argtypes = [ctypes.POINTER(SceneDesc), ctypes.POINTER(ctypes.c_uint64)]
        L.tds_create_scene.argtypes = [ctypes.POINTER(SceneDesc), vp, ctypes.c_uint64, vp,
                                       ctypes.POINTER(vp)]
        L.tds_set_tool_pose.argtypes = [vp, _fp, _fp, _fp, _fp]
        L.tds_step.argtypes = [vp, ctypes.c_uint32]
        L.tds_state_bytes.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64)]
        L.tds_save_state.argtypes = [vp, vp, ctypes.c_uint64]
        L.tds_load_state.argtypes = [vp, vp, ctypes.c_uint64]
        L.tds_synchronize.argtypes = [vp]
        L.tds_read_particles.argtypes = [vp] + [vp] * 9 + [ctypes.c_uint32]
        L.tds_read_tool_force.argtypes = [vp, _fp, _fp]
        L.tds_read_contacts.argtypes = [vp, vp, vp, vp, ctypes.c_uint32,
                                        ctypes.POINTER(ctypes.c_uint32)]
        L.tds_get_stats.argtypes = [vp, ctypes.POINTER(StepStats)]
        L.tds_set_timing.argtypes = [vp, ctypes.c_int32]
        L.tds_set_solver.argtypes = [vp, ctypes.c_uint32, ctypes.c_float, ctypes.c_uint32]
        L.tds_find_pair_contacts_noalloc.argtypes = [vp, vp, vp, vp, ctypes.c_uint32, ctypes.c_int32,
                                                     vp, ctypes.c_uint32, vp, vp]
        L.tds_mlp_param_count.argtypes = []
        L.tds_set_mlp_weights.argtypes = [vp, vp, ctypes.c_uint32]
        L.tds_set_recording.argtypes = [vp, ctypes.c_int32]
        L.tds_set_warm_start.argtypes = [vp, ctypes.c_int32]
        L.tds_set_recolour_period.argtypes = [vp, ctypes.c_uint32]
        L.tds_set_impact.argtypes = [vp, ctypes.c_float, ctypes.c_float, ctypes.c_uint32]
        L.tds_set_cutter.argtypes = [vp, ctypes.c_uint32, ctypes.POINTER(Cutter)]
        L.tds_read_heightfield.argtypes = [vp, ctypes.c_uint32, vp, vp, ctypes.c_uint32]
        L.tds_read_radii.argtypes = [vp, vp, ctypes.c_uint32]
        L.tds_read_training_samples.argtypes = [vp, vp, vp, vp, ctypes.c_uint32,
                                                ctypes.POINTER(ctypes.c_uint32)]
        L.tds_mlp_workspace_bytes.argtypes = [ctypes.POINTER(ctypes.c_uint64)]
        L.tds_mlp_forward.argtypes = [vp, vp, ctypes.c_uint32, vp, vp, vp]
        L.tds_mlp_loss_grad.argtypes = [vp, vp, vp, ctypes.c_uint32, vp, vp, vp, vp]
        L.tds_mlp_adam_step.argtypes = [vp, vp, vp, vp, ctypes.c_uint32, ctypes.c_float, vp]
        L.tds_batch_workspace_bytes.argtypes = [ctypes.POINTER(SceneDesc), ctypes.c_uint32,
                                                ctypes.POINTER(ctypes.c_uint64)]
        L.tds_create_batch.argtypes = [ctypes.POINTER(SceneDesc), ctypes.c_uint32, vp, ctypes.c_uint64, vp,
                                       ctypes.POINTER(vp)]
        L.tds_batch_set_tool_pose.argtypes = [vp, ctypes.c_uint32, _fp, _fp, _fp, _fp]
        L.tds_batch_read_particles.argtypes = [vp, ctypes.c_uint32] + [vp] * 9 + [ctypes.c_uint32]
        L.tds_batch_read_tool_forces.argtypes = [vp, vp, ctypes.c_uint32]
        L.tds_batch_read_solve.argtypes = [vp, vp, vp, ctypes.c_uint32]
        L.tds_set_graph.argtypes = [vp, ctypes.c_int32]
        L.tds_batch_set_tool_poses.argtypes = [vp, vp, ctypes.c_uint32]
        L.tds_aggregate_bodies.argtypes = [vp, ctypes.POINTER(Zone), ctypes.c_uint32, ctypes.POINTER(Aggregate)]
        L.tds_coarse_grain.argtypes = [vp, ctypes.POINTER(Grid), ctypes.c_int32, ctypes.c_float, vp, vp, vp]
        L.tds_advect_fluid.argtypes = [ctypes.POINTER(Grid), vp, vp, vp, ctypes.c_float, vp, vp]
        L.tds_get_launch_config.argtypes = [vp, ctypes.POINTER(LaunchConfig)]
        L.tds_set_launch_config.argtypes = [vp, ctypes.POINTER(LaunchConfig)]
        L.tds_destroy_scene.argtypes = [vp]
        L.tds_destroy_scene.restype = None
        L.tds_last_error.restype = ctypes.c_char_p
        for name in EXPORTED:
            if name not in ("tds_destroy_scene", "tds_last_error"):
                getattr(L, name).restype = ctypes.c_int32
        L.tds_mlp_param_count.restype = ctypes.c_uint32
        _lib = L
    return _lib


def _check(status: int):
    if status != TDS_OK:
        raise TdsError(status, lib().tds_last_error().decode())


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def _fptr(a: np.ndarray):
    return a.ctypes.data_as(_fp)


def _vec(a, n):
    return (_f * n)(*[float(v) for v in a])


def _make_desc(s: dict, contacts_per_particle: int, domain):
    """tds_scene_desc of a scene dictionary; returns (desc, arrays to keep alive, n)."""
    x = _f32(s["x"]).reshape(-1, 3)
    n = x.shape[0]
    keep = []

    def col(a, k):
        c = np.ascontiguousarray(a[:, k])
        keep.append(c)
        return _fptr(c)

    v = _f32(s.get("v", np.zeros((n, 3)))).reshape(n, 3)
    w = _f32(s.get("w", np.zeros((n, 3)))).reshape(n, 3)
    r = _f32(s["r"]).reshape(n)
    keep.append(r)
    d = SceneDesc()
    d.n = n
    d.x, d.y, d.z = col(x, 0), col(x, 1), col(x, 2)
    d.vx, d.vy, d.vz = col(v, 0), col(v, 1), col(v, 2)
    d.wx, d.wy, d.wz = col(w, 0), col(w, 1), col(w, 2)
    d.radius = _fptr(r)
    d.density, d.young, d.poisson = s["density"], s["young"], s["poisson"]
    d.mu_t, d.mu_r, d.cohesion = s["mu_t"], s["mu_r"], s["cohesion"]
    d.mu_tool = s.get("mu_tool", s["mu_t"])
    hf = s.get("hf")
    if hf is not None:
        h = _f32(hf["h"]).reshape(-1)
        keep.append(h)
        d.hf_nx, d.hf_ny = hf["nx"], hf["ny"]
        d.hf_x0, d.hf_y0, d.hf_cell = hf["x0"], hf["y0"], hf["cell"]
        d.hf_heights = _fptr(h)
    walls = _f32(s.get("walls", np.zeros((0, 10)))).reshape(-1, 10)
    boxes = _f32(s.get("tool_boxes", np.zeros((0, 10)))).reshape(-1, 10)
    keep += [walls, boxes]
    d.n_walls, d.walls = walls.shape[0], _fptr(walls)
    d.n_tool_boxes, d.tool_boxes = boxes.shape[0], _fptr(boxes)
    d.dt = s["dt"]
    for i in range(3):
        d.gravity[i] = s["gravity"][i]
    d.max_iters = int(s["iters"])
    d.tol = float(s.get("tol", 0.0))
    d.residual_every = int(s.get("residual_every", 10))
    d.warm_start = int(s.get("warm_start", 1))
    d.contacts_per_particle = int(contacts_per_particle)
    d.restitution = float(s.get("restitution", 0.0))
    d.impact_speed = float(s.get("impact_speed", 0.0))
    d.impact_iters = int(s.get("impact_iters", 0))
    if domain is not None:
        for i in range(3):
            d.domain_lo[i], d.domain_hi[i] = domain[0][i], domain[1][i]
    return d, keep, n


class Scene:
    """One simulated bed on the current CUDA device.

    ``workspace="torch"`` carves all device memory from one torch uint8 tensor;
    ``"library"`` lets libtds cudaMalloc it. The CUDA stream is torch's current
    stream unless ``stream`` (a ``torch.cuda.Stream``) is given.
    """

    def __init__(self, scene: dict, stream=None, workspace: str = "torch",
                 contacts_per_particle: int = 0, domain=None, **override):
        s = dict(scene)
        s.update(override)
        self._create([s], stream, workspace, contacts_per_particle, [domain])
        if "tool" in s and s["tool"] is not None:
            self.set_tool_pose(s["tool"])

    def _create(self, scenes, stream, workspace, contacts_per_particle, domains):
        import torch

        if not torch.cuda.is_available():
            raise TdsError(-2, "no CUDA device")
        count = len(scenes)
        descs = (SceneDesc * count)()
        keep, sizes = [], []
        for q, s in enumerate(scenes):
            d, k, n = _make_desc(s, contacts_per_particle, domains[q])
            descs[q] = d
            keep += k
            sizes.append(n)
        self.sizes = sizes
        self.offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        self.n = int(self.offsets[-1])
        self.desc = descs[0]
        self.solver = (int(descs[0].max_iters), float(descs[0].tol), int(descs[0].residual_every))
        self._descs = descs
        self._keep = keep
        L = lib()
        self._torch = torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._ws = None
        ws_ptr, ws_bytes = None, 0
        if workspace == "torch":
            nb = ctypes.c_uint64()
            _check(L.tds_batch_workspace_bytes(descs, count, ctypes.byref(nb)))
            self._ws = torch.empty(int(nb.value) + 256, dtype=torch.uint8, device="cuda")
            base = self._ws.data_ptr()
            ws_ptr = (base + 255) & ~255
            ws_bytes = int(nb.value)
        h = ctypes.c_void_p()
        if count == 1:
            _check(L.tds_create_scene(ctypes.byref(descs[0]), ws_ptr, ws_bytes,
                                      ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        else:
            _check(L.tds_create_batch(descs, count, ws_ptr, ws_bytes,
                                      ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        self.h = h
        period = int(scenes[0].get("recolour_every", 1))
        if period != 1:
            self.set_recolour_period(period)

    # -- calls ---------------------------------------------------------------
    def set_tool_pose(self, tool: dict):
        _check(lib().tds_set_tool_pose(self.h, _vec(tool["pos"], 3), _vec(tool["quat"], 4),
                                       _vec(tool["vel"], 3), _vec(tool["angvel"], 3)))

    def step(self, nsteps: int = 1):
        _check(lib().tds_step(self.h, nsteps))

    def synchronize(self):
        _check(lib().tds_synchronize(self.h))

    def read_particles(self, out=None) -> dict:
        """x, v, w as (n, 3) float32 numpy arrays. ``out`` may give nine
        preallocated float32 host buffers (e.g. pinned torch tensors' numpy
        views) to copy into."""
        n = self.n
        bufs = out if out is not None else [np.empty(n, np.float32) for _ in range(9)]
        ptrs = [ctypes.c_void_p(b.ctypes.data) if b is not None else None for b in bufs]
        _check(lib().tds_read_particles(self.h, *ptrs, n))
        if out is not None:
            return {}
        return {"x": np.stack(bufs[0:3], 1), "v": np.stack(bufs[3:6], 1), "w": np.stack(bufs[6:9], 1)}

    def read_positions_into(self, x, y, z):
        _check(lib().tds_read_particles(self.h, ctypes.c_void_p(x.ctypes.data),
                                        ctypes.c_void_p(y.ctypes.data), ctypes.c_void_p(z.ctypes.data),
                                        None, None, None, None, None, None, self.n))

    def read_tool_force(self):
        f = (_f * 3)()
        t = (_f * 3)()
        _check(lib().tds_read_tool_force(self.h, f, t))
        return np.array(f[:], np.float64), np.array(t[:], np.float64)

    def read_contacts(self) -> dict:
        """The last step's contacts sorted by key: keys (uint64), lam (m, 7)
        float32 [normal, tangent world xyz, rolling xyz], colour (uint32)."""
        cnt = ctypes.c_uint32()
        _check(lib().tds_read_contacts(self.h, None, None, None, 0, ctypes.byref(cnt)))
        m = int(cnt.value)
        keys = np.zeros(m, np.uint64)
        lam = np.zeros((m, 7), np.float32)
        col = np.zeros(m, np.uint32)
        _check(lib().tds_read_contacts(self.h, ctypes.c_void_p(keys.ctypes.data),
                                       ctypes.c_void_p(lam.ctypes.data),
                                       ctypes.c_void_p(col.ctypes.data), m, ctypes.byref(cnt)))
        o = np.argsort(keys, kind="stable")
        return {"keys": keys[o], "lam": lam[o], "colour": col[o]}

    def stats(self) -> dict:
        st = StepStats()
        _check(lib().tds_get_stats(self.h, ctypes.byref(st)))
        out = {k: getattr(st, k) for k, _ in StepStats._fields_ if k != "phase_ms"}
        out["phase_ms"] = dict(zip(PHASES, st.phase_ms[:]))
        return out

    def set_solver(self, iters: int, tol: float = 0.0, residual_every: int = 10):
        _check(lib().tds_set_solver(self.h, int(iters), float(tol), int(residual_every)))
        self.solver = (int(iters), float(tol), int(residual_every))

    def set_timing(self, enable: bool = True):
        _check(lib().tds_set_timing(self.h, int(enable)))

    def set_mlp_weights(self, params: np.ndarray):
        p = np.ascontiguousarray(np.asarray(params, np.float32).reshape(-1))
        _check(lib().tds_set_mlp_weights(self.h, ctypes.c_void_p(p.ctypes.data), p.size))

    def set_impact(self, restitution: float, impact_speed: float, iters: int):
        """Impact stage settings (iters 0 disables it)."""
        _check(lib().tds_set_impact(self.h, float(restitution), float(impact_speed), int(iters)))

    def set_cutter(self, cutter: dict | None, scene: int = 0):
        """Active-zone cutter on the scene's tool (tool-frame edge point,
        edge direction, length, blade normal, phi [rad], bank density, spawn
        radius); None removes it."""
        c = Cutter()
        if cutter is not None:
            for k in ("edge", "dir", "normal"):
                for i in range(3):
                    getattr(c, k)[i] = float(cutter[k][i])
            c.length = float(cutter["length"])
            c.phi, c.bank_density = float(cutter["phi"]), float(cutter["bank_density"])
            c.spawn_radius = float(cutter["spawn_radius"])
        _check(lib().tds_set_cutter(self.h, int(scene), ctypes.byref(c)))

    def read_heightfield(self, scene: int = 0, shape=None):
        """Current heights and pending mass per node, (ny+1, nx+1) float32."""
        d = self._descs[scene]
        ny, nx = int(d.hf_ny) + 1, int(d.hf_nx) + 1
        h = np.empty(nx * ny, np.float32)
        p = np.empty(nx * ny, np.float32)
        _check(lib().tds_read_heightfield(self.h, int(scene), ctypes.c_void_p(h.ctypes.data),
                                          ctypes.c_void_p(p.ctypes.data), nx * ny))
        return h.reshape(ny, nx), p.reshape(ny, nx)

    def read_radii(self) -> np.ndarray:
        r = np.empty(self.n, np.float32)
        _check(lib().tds_read_radii(self.h, ctypes.c_void_p(r.ctypes.data), self.n))
        return r

    def save_state(self) -> np.ndarray:
        """The state of the last completed step as bytes (a checkpoint)."""
        n = ctypes.c_uint64()
        _check(lib().tds_state_bytes(self.h, ctypes.byref(n)))
        buf = np.empty(n.value, np.uint8)
        _check(lib().tds_save_state(self.h, ctypes.c_void_p(buf.ctypes.data), n.value))
        return buf

    def load_state(self, buf) -> None:
        """Continue from a checkpoint of a scene with the same layout."""
        buf = np.ascontiguousarray(buf, np.uint8)
        _check(lib().tds_load_state(self.h, ctypes.c_void_p(buf.ctypes.data), buf.size))

    def set_warm_start(self, mode: int):
        _check(lib().tds_set_warm_start(self.h, int(mode)))

    def set_recolour_period(self, period: int):
        """Colour every contact every ``period``-th step; in the steps between
        persisting contacts keep their colour and only new ones are coloured."""
        _check(lib().tds_set_recolour_period(self.h, int(period)))

    def set_recording(self, enable: bool = True):
        _check(lib().tds_set_recording(self.h, int(enable)))

    def aggregate_bodies(self, zones) -> list:
        """Aggregate bodies of the current state. ``zones``: dicts with
        "planes" ((k, 4) half-spaces n . x <= d) and optionally "scene".
        Returns per zone a dict of count, mass, com, vel, omega and the 3x3
        inertia about com."""
        arr = (Zone * max(1, len(zones)))()
        for q, z in enumerate(zones):
            pl = np.asarray(z["planes"], np.float32).reshape(-1, 4)
            arr[q].scene, arr[q].n_planes = int(z.get("scene", 0)), pl.shape[0]
            for k in range(min(pl.shape[0], ZONE_MAX_PLANES)):
                for c in range(4):
                    arr[q].planes[k][c] = float(pl[k, c])
        out = (Aggregate * max(1, len(zones)))()
        _check(lib().tds_aggregate_bodies(self.h, arr, len(zones), out))
        res = []
        for q in range(len(zones)):
            a = out[q]
            I = np.array(a.inertia[:])
            res.append({"count": a.count, "mass": a.mass, "com": np.array(a.com[:]), "vel": np.array(a.vel[:]),
                        "omega": np.array(a.omega[:]),
                        "inertia": np.array([[I[0], I[3], I[4]], [I[3], I[1], I[5]], [I[4], I[5], I[2]]])})
        return res

    def coarse_grain(self, grid: Grid, kernel: int = 0, R: float = 0.0):
        """Mass density, momentum density and velocity fields of the current
        state on ``grid`` (torch device tensors: rho (nz, ny, nx), p and u
        (nz, ny, nx, 3)), computed on the scene's stream."""
        torch = self._torch
        shape = (grid.nz, grid.ny, grid.nx)
        rho = torch.empty(shape, dtype=torch.float32, device="cuda")
        p = torch.empty(shape + (3,), dtype=torch.float32, device="cuda")
        u = torch.empty_like(p)
        _check(lib().tds_coarse_grain(self.h, ctypes.byref(grid), int(kernel), float(R),
                                      ctypes.c_void_p(rho.data_ptr()), ctypes.c_void_p(p.data_ptr()),
                                      ctypes.c_void_p(u.data_ptr())))
        return rho, p, u

    def launch_config(self) -> dict:
        c = LaunchConfig()
        _check(lib().tds_get_launch_config(self.h, ctypes.byref(c)))
        return {k: getattr(c, k) for k, _ in LaunchConfig._fields_}

    def set_launch_config(self, pgs_blocks: int = 0, pgs_sync: int | None = None, colour_blocks: int = 0,
                          pgs_threads: int = 0, pgs_per_thread: int = 0, wait_limit_us: int = 0):
        """Solver CTAs, solver sync mode (1 neighbour, 0 grid barrier),
        colouring CTAs, the solver CTA shape (threads x contacts per
        thread, one of SHAPES) and the limit of a wait on other CTAs [us];
        0 (or None for the mode) keeps the current value."""
        c = LaunchConfig()
        _check(lib().tds_get_launch_config(self.h, ctypes.byref(c)))
        c.pgs_blocks, c.colour_blocks = int(pgs_blocks), int(colour_blocks)
        c.wait_limit_us = int(wait_limit_us)
        if pgs_sync is not None:
            c.pgs_sync = int(pgs_sync)
        if pgs_threads or pgs_per_thread:
            c.pgs_threads, c.pgs_per_thread = int(pgs_threads), int(pgs_per_thread)
        _check(lib().tds_set_launch_config(self.h, ctypes.byref(c)))

    def set_graph(self, enable: bool = True):
        """Replay each step from a CUDA graph (needs a non-default stream)."""
        _check(lib().tds_set_graph(self.h, int(enable)))

    def read_training_samples(self) -> dict:
        """Features (m, 10), targets (m, 3) and keys of the last recorded step,
        sorted by key."""
        cnt = ctypes.c_uint32()
        _check(lib().tds_read_training_samples(self.h, None, None, None, 0, ctypes.byref(cnt)))
        m = int(cnt.value)
        feat = np.zeros((m, 10), np.float32)
        targ = np.zeros((m, 3), np.float32)
        keys = np.zeros(m, np.uint64)
        _check(lib().tds_read_training_samples(self.h, ctypes.c_void_p(feat.ctypes.data),
                                               ctypes.c_void_p(targ.ctypes.data),
                                               ctypes.c_void_p(keys.ctypes.data), m, ctypes.byref(cnt)))
        o = np.argsort(keys, kind="stable")
        return {"features": feat[o], "targets": targ[o], "keys": keys[o]}

    def close(self):
        if getattr(self, "h", None):
            lib().tds_destroy_scene(self.h)
            self.h = None
        self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch(Scene):
    """Independent scenes advanced together by the same launches: each scene
    keeps its particles, heightfield, walls, tool and friction coefficients
    and steps exactly as it would alone. Particle ids are global (scene q owns
    ``offsets[q]:offsets[q + 1]``)."""

    def __init__(self, scenes, stream=None, workspace: str = "torch",
                 contacts_per_particle: int = 0, domains=None):
        scenes = [dict(s) for s in scenes]
        if domains is None:
            domains = [None] * len(scenes)
        self._create(scenes, stream, workspace, contacts_per_particle, domains)
        for q, s in enumerate(scenes):
            if s.get("tool") is not None:
                self.set_scene_tool_pose(q, s["tool"])

    def __len__(self):
        return len(self.sizes)

    def set_scene_tool_pose(self, q: int, tool: dict):
        _check(lib().tds_batch_set_tool_pose(self.h, int(q), _vec(tool["pos"], 3), _vec(tool["quat"], 4),
                                             _vec(tool["vel"], 3), _vec(tool["angvel"], 3)))

    def set_tool_poses(self, tools):
        """Every scene's tool pose in one call (a sequence of pose dicts)."""
        P = np.empty((len(self.sizes), 13), np.float32)
        for q, t in enumerate(tools):
            P[q, 0:3], P[q, 3:7], P[q, 7:10], P[q, 10:13] = t["pos"], t["quat"], t["vel"], t["angvel"]
        _check(lib().tds_batch_set_tool_poses(self.h, ctypes.c_void_p(P.ctypes.data), len(self.sizes)))

    def read_scene(self, q: int) -> dict:
        """x, v, w of scene q as (n_q, 3) float32 arrays."""
        n = self.sizes[q]
        bufs = [np.empty(n, np.float32) for _ in range(9)]
        ptrs = [ctypes.c_void_p(b.ctypes.data) for b in bufs]
        _check(lib().tds_batch_read_particles(self.h, int(q), *ptrs, n))
        return {"x": np.stack(bufs[0:3], 1), "v": np.stack(bufs[3:6], 1), "w": np.stack(bufs[6:9], 1)}

    def read_tool_forces(self) -> np.ndarray:
        """(scenes, 6) float64: force and torque on each scene's tool."""
        out = np.zeros((len(self.sizes), 6), np.float32)
        _check(lib().tds_batch_read_tool_forces(self.h, ctypes.c_void_p(out.ctypes.data), len(self.sizes)))
        return out.astype(np.float64)

    def read_solve(self) -> dict:
        """Each scene's solve in the last step: residual (float32) at its last
        check and sweeps (uint32)."""
        res = np.zeros(len(self.sizes), np.float32)
        sw = np.zeros(len(self.sizes), np.uint32)
        _check(lib().tds_batch_read_solve(self.h, ctypes.c_void_p(res.ctypes.data), ctypes.c_void_p(sw.ctypes.data),
                                          len(self.sizes)))
        return {"residual": res, "sweeps": sw}


# ---------------------------------------------------------------------------
# the learned warm start's network on device buffers (torch tensors)
# ---------------------------------------------------------------------------
PARAM_SHAPES = (("W1", (64, 10)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)),
                ("W3", (3, 64)), ("b3", (3,)))


def param_count() -> int:
    return int(lib().tds_mlp_param_count())


def flatten_params(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[k], np.float32).reshape(-1) for k, _ in PARAM_SHAPES])


def unflatten_params(v) -> dict:
    v = np.asarray(v, np.float64).reshape(-1)
    out, o = {}, 0
    for k, shp in PARAM_SHAPES:
        sz = int(np.prod(shp))
        out[k] = v[o:o + sz].reshape(shp)
        o += sz
    return out


def init_params(seed: int = 0) -> np.ndarray:
    """He-style initial weights (seeded), zero biases."""
    g = np.random.Generator(np.random.PCG64(seed))
    p = {"W1": g.normal(0, np.sqrt(2 / 10), (64, 10)), "b1": np.zeros(64),
         "W2": g.normal(0, np.sqrt(2 / 64), (64, 64)), "b2": np.zeros(64),
         "W3": g.normal(0, np.sqrt(1 / 64), (3, 64)), "b3": np.zeros(3)}
    return flatten_params(p)


class Net:
    """FP32 master parameters and Adam moments on the GPU; the forward,
    loss/gradient and update run in libtds's tensor-core kernels."""

    def __init__(self, params=None, seed: int = 0):
        import torch

        self.torch = torch
        p = init_params(seed) if params is None else np.asarray(params, np.float32)
        self.params = torch.tensor(p, device="cuda")
        self.grad = torch.zeros_like(self.params)
        self.mom = torch.zeros_like(self.params)
        self.vel = torch.zeros_like(self.params)
        nb = ctypes.c_uint64()
        _check(lib().tds_mlp_workspace_bytes(ctypes.byref(nb)))
        self.ws = torch.empty(int(nb.value) + 256, dtype=torch.uint8, device="cuda")
        self.loss = torch.zeros(1, device="cuda")
        self.step_count = 0

    def _ws(self):
        return ctypes.c_void_p((self.ws.data_ptr() + 255) & ~255)

    def _stream(self):
        return ctypes.c_void_p(self.torch.cuda.current_stream().cuda_stream)

    def forward(self, X):
        X = self.torch.as_tensor(X, dtype=self.torch.float32, device="cuda").contiguous()
        Y = self.torch.empty((X.shape[0], 3), device="cuda")
        _check(lib().tds_mlp_forward(ctypes.c_void_p(self.params.data_ptr()), ctypes.c_void_p(X.data_ptr()),
                                     X.shape[0], ctypes.c_void_p(Y.data_ptr()), self._ws(), self._stream()))
        return Y

    def loss_grad(self, X, T):
        X = self.torch.as_tensor(X, dtype=self.torch.float32, device="cuda").contiguous()
        T = self.torch.as_tensor(T, dtype=self.torch.float32, device="cuda").contiguous()
        _check(lib().tds_mlp_loss_grad(ctypes.c_void_p(self.params.data_ptr()), ctypes.c_void_p(X.data_ptr()),
                                       ctypes.c_void_p(T.data_ptr()), X.shape[0],
                                       ctypes.c_void_p(self.grad.data_ptr()),
                                       ctypes.c_void_p(self.loss.data_ptr()), self._ws(), self._stream()))
        return self.loss, self.grad

    def train_step(self, X, T, lr: float = 1e-3) -> float:
        self.loss_grad(X, T)
        self.step_count += 1
        _check(lib().tds_mlp_adam_step(ctypes.c_void_p(self.params.data_ptr()),
                                       ctypes.c_void_p(self.grad.data_ptr()),
                                       ctypes.c_void_p(self.mom.data_ptr()),
                                       ctypes.c_void_p(self.vel.data_ptr()), self.step_count, float(lr),
                                       self._stream()))
        return self.loss

    def host_params(self) -> np.ndarray:
        return self.params.detach().cpu().numpy().astype(np.float32)
