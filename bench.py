"""Benchmark of the active-soil particle step (particle-steps/s) on GB300.

Default workload: the 1 000 000-sphere excavation bed (r ~ U[0.02, 0.03] m,
8 x 8 m, 1024^2 heightfield, 12-box bucket on a seeded spline dig, c_p 5 kPa,
previous-step warm start), each step's PGS solved to the 1e-4 residual (cap
2000 sweeps, adaptive check schedule). The bed is spawned on a jittered lattice and
settled untimed on the GPU; the bucket then approaches its deepest cut
untimed, and the timed steps dig. ``--workload batched`` times 256
independent beds in one batch (graph replay); ``--unbatched`` the same beds
as separate scenes.

  value   = particles x timed steps / device time of those steps (CUDA events
            on the scene's stream, state resident in HBM)
  e2e     = the same through the C ABI with host buffers: every step sets the
            tool pose from the host and reads positions and tool force back
            into pinned host memory
  fixed_sweeps / roofline: a second timed region on the same bed with the
            workload's fixed sweep count (100 for the large bed); the
            roofline is the persistent PGS kernel's algorithmic bytes (204 B
            per particle-pair contact and 160 B per static contact per sweep)
            over its CUDA-event time there, against the measured HBM copy peak
  cpu_baseline: the FP64 CPU oracle on a bounded column of the same bed

``--impl reference`` times the oracle alone (the slow baseline arm).
Multi-GPU (torchrun): independent replicas, one per rank, no collective on
the data path; value sums the particles of all ranks over the slowest rank.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s at fixed PGS residual; plain vs batched/learned on 1 GB300"
UNIT = "particle-steps/s"
SETTLE_SWEEPS = 30   # PGS sweeps per untimed settle step
TUNE_RESERVE = 80    # last settle steps available to the launch-shape autotuner
BYTES_PP = 204.0      # per particle-pair contact per sweep
BYTES_STATIC = 160.0  # per static contact per sweep


def reduce_max(value: float, world: int, device: str = "cuda") -> float:
    """The largest value over the ranks (the slowest rank's time)."""
    if world <= 1:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(value: float, world: int, device: str = "cuda") -> float:
    """The sum over the ranks (particles of all replicas)."""
    if world <= 1:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t)
    return float(t.item())


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tds", choices=["tds", "reference"])
    ap.add_argument("--workload", default="large")
    ap.add_argument("--n", type=int, default=0, help="override the particle count")
    ap.add_argument("--scenes", type=int, default=0, help="batched workload: override the bed count")
    ap.add_argument("--pgs-sync", type=int, default=-1, choices=[-1, 0, 1],
                    help="solver sync between colours: 1 neighbour, 0 grid barrier (-1: library default)")
    ap.add_argument("--pgs-blocks", type=int, default=0, help="solver CTAs (0: library default)")
    ap.add_argument("--pgs-shape", default="", help="solver CTA shape THREADSxPER_THREAD (e.g. 416x1)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the library's default launch shapes (no untimed tuning before warm-up)")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the learned and batched comparison forms of the default run")
    ap.add_argument("--unbatched", action="store_true",
                    help="batched workload: step the beds as separate scenes (the plain form)")
    ap.add_argument("--iters", type=int, default=0, help="override the sweeps per step")
    ap.add_argument("--settle", type=int, default=-1)
    ap.add_argument("--approach", type=float, default=0.3,
                    help="fraction of the dig path covered untimed before timing")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--tol", type=float, default=1e-4,
                    help="stop each step's solve at this residual (cap --max-iters); 0: fixed sweeps")
    ap.add_argument("--roofline-sweeps", type=int, default=-1,
                    help="sweeps per step of the second timed region that gives the PGS roofline "
                         "(-1: the workload's fixed sweep count, 0: no second region)")
    ap.add_argument("--max-iters", type=int, default=2000)
    ap.add_argument("--cold", action="store_true", help="cold start instead of previous-step impulses")
    ap.add_argument("--recolour-period", type=int, default=16,
                    help="colour every contact every k-th step, only the new contacts in between (1: every step)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--verbose", action="store_true")
    return ap.parse_args()


def log(args, *a):
    if args.verbose:
        print(*a, file=sys.stderr, flush=True)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(rows)}


# ---------------------------------------------------------------------------
# roofline inputs
# ---------------------------------------------------------------------------
def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


def pgs_source_sha() -> str:
    """Hash of the solver's code (tds_solve.cu and tds_internal.cuh with
    comments and blank lines removed): the ncu counters stay valid while it
    is unchanged."""
    h = hashlib.sha256()
    for f in ("tds_solve.cu", "tds_internal.cuh"):
        src = open(os.path.join(ROOT, "paper_2011_00459_gb300", "csrc", f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update("\n".join(line.rstrip() for line in src.splitlines() if line.strip()).encode())
    return h.hexdigest()[:16]


def ncu_traffic(workload: str) -> float | None:
    """DRAM bytes per PGS launch per (sweep x contact) from the committed ncu
    summary, if it was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", f"k_pgs_{workload}.md")
    if not os.path.exists(p):
        return None
    text = open(p).read()
    sha = re.search(r"source_sha:\s*([0-9a-f]+)", text)
    per = re.search(r"dram_bytes_per_sweep_contact:\s*([0-9.eE+-]+)", text)
    if not sha or not per or sha.group(1) != pgs_source_sha():
        return None
    return float(per.group(1))


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
def _apply_args(scene: dict, args) -> dict:
    if args.iters:
        scene["iters"] = args.iters
    scene["fixed_iters"] = int(scene["iters"] if args.roofline_sweeps < 0 else args.roofline_sweeps)
    if args.tol > 0:
        scene["tol"] = args.tol
        scene["iters"] = args.max_iters
        scene["residual_every"] = 0  # adaptive check schedule (same stopping criterion)
    if args.cold:
        scene["warm_start"] = 0
    scene["recolour_every"] = args.recolour_period
    return scene


def make_workload(args, rank: int):
    """One scene dict, or for the batched workload a list of them."""
    from paper_2011_00459_gb300 import scenes as S

    if args.workload == "batched":
        kw = {"scenes": args.scenes} if args.scenes else {}
        return [_apply_args(s, args) for s in S.batched(seed=args.seed + rank, **kw)]
    gen = S.WORKLOADS[args.workload]
    kw = {"n": args.n} if args.n else {}
    return _apply_args(gen(seed=args.seed + rank, **kw), args)


def _solve_desc(scene: dict) -> str:
    k = int(scene.get("recolour_every", 1))
    colouring = (", every contact coloured every step" if k <= 1 else
                 f", every contact coloured every {k}th step and only the new contacts in between")
    return (f"residual <= {scene['tol']:g} (cap {scene['iters']} sweeps)" if scene.get("tol", 0) > 0
            else f"{scene['iters']} sweeps") + colouring


def describe(work, args) -> dict:
    if isinstance(work, list):
        ns = np.array([len(s["r"]) for s in work])
        s0 = work[0]
        return {
            "workload": f"batched: {len(work)} independent walled beds, {int(ns.sum())} spheres "
                        f"(n per bed log-U[1e3, 2e4]: min {ns.min()}, mean {ns.mean():.0f}, max {ns.max()}), "
                        f"r~U[0.03,0.05] m, 2:1 footprints 0.6 m deep, flat heightfields, blade speed "
                        f"U[0.2,1.5] m/s, depth U[0.1,0.4] m, mu_t U[0.4,0.9], PGS to {_solve_desc(s0)} per step, "
                        + ("each bed its own scene and launch sequence per step (unbatched)"
                           if args.unbatched else
                           "one launch sequence per step replayed from a CUDA graph"),
            "particles": int(ns.sum()), "scenes": len(work), "max_sweeps": int(s0["iters"]), "dt": s0["dt"],
            "solve": _solve_desc(s0),
            "warm_start": "previous step" if s0.get("warm_start", 1) else "cold",
            "seed": args.seed, "l2": "inputs larger than L2 (contact rows and impulses > 129 MB)",
        }
    scene = work
    return {
        "workload": f"{scene['name']}: {len(scene['r'])} spheres r~U[{scene['r'].min():.3f},"
                    f"{scene['r'].max():.3f}] m, {scene['footprint'][0]:g}x{scene['footprint'][1]:g} m "
                    f"walled bed, {scene['hf']['nx']}x{scene['hf']['ny']} heightfield, "
                    f"{len(scene['tool_boxes'])}-box {scene['tool_kind']}, c_p {scene['cohesion']:g} Pa, "
                    f"PGS to {_solve_desc(scene)} per step, previous-step warm start",
        "particles": int(len(scene["r"])), "max_sweeps": int(scene["iters"]), "dt": scene["dt"],
        "solve": _solve_desc(scene),
        "warm_start": "previous step" if scene.get("warm_start", 1) else "cold",
        "seed": args.seed, "l2": "inputs larger than L2 (contact rows and impulses > 129 MB)",
    }


class PlainSim:
    """One bed: settle with the tool parked, approach untimed, then dig."""

    def __init__(self, tds, S, scene, stream, args):
        self.g = tds.Scene(scene, stream=stream)
        self.scene, self.S, self.args = scene, S, args
        self.n = len(scene["r"])
        self.dt = scene["dt"]

    def settle_and_approach(self, between=None):
        S, scene, args, g = self.S, self.scene, self.args, self.g
        settle = scene["settle_steps"] if args.settle < 0 else args.settle
        g.set_tool_pose(S.parked_tool(scene))
        g.set_solver(SETTLE_SWEEPS)
        reserve = min(settle, TUNE_RESERVE)
        g.step(settle - reserve)
        # the last settle steps host the launch-shape choice: its timed steps
        # are settle steps (same sweeps, tool parked) and launch shapes do not
        # change results, so the trajectory is the one an untuned run takes
        taken = between() if between else 0
        g.step(max(0, reserve - taken))
        g.set_solver(int(scene["iters"]), float(scene.get("tol", 0.0)), int(scene.get("residual_every", 10)))
        parts = g.read_particles()
        self.surface = S.surface_level(parts["x"], scene["r"])
        self.path = S.tool_path(scene, self.surface, seed=args.seed)
        length = getattr(self.path, "length", None)
        t0 = args.approach * (length if length is not None else self.path.push) / self.path.speed
        self.k = 0
        while self.k * self.dt < t0:
            self.advance()

    def advance(self):
        self.g.set_tool_pose(self.path(self.k * self.dt))
        self.g.step(1)
        self.k += 1

    def read_back(self, xs):
        self.g.read_positions_into(*xs)
        self.g.read_tool_force()

    def d2h_bytes(self):
        return 3 * 4 * self.n + 6 * 4

    def h2d_bytes(self):
        return 13 * 4


class BatchedSim(PlainSim):
    """Independent beds in one batch, stepped by replayed CUDA graphs; every
    bed settles with its blade parked, then all blades cut along their own
    cycles (speed and depth per bed)."""

    def __init__(self, tds, S, scenes, stream, args):
        self.g = tds.Batch(scenes, stream=stream)
        self.g.set_graph(True)
        self.scenes, self.S, self.args = scenes, S, args
        self.n = int(self.g.n)
        self.dt = scenes[0]["dt"]

    def settle_and_approach(self, between=None):
        S, args, g = self.S, self.args, self.g
        s0 = self.scenes[0]
        settle = s0["settle_steps"] if args.settle < 0 else args.settle
        g.set_tool_poses([S.parked_tool(s) for s in self.scenes])
        g.set_solver(SETTLE_SWEEPS)
        reserve = min(settle, TUNE_RESERVE)
        g.step(settle - reserve)
        taken = between() if between else 0  # launch shapes chosen on settle steps (see PlainSim)
        g.step(max(0, reserve - taken))
        g.set_solver(int(s0["iters"]), float(s0.get("tol", 0.0)), int(s0.get("residual_every", 10)))
        self.paths = []
        for q, s in enumerate(self.scenes):
            surface = S.surface_level(g.read_scene(q)["x"], s["r"])
            self.paths.append(S.tool_path(s, surface, seed=args.seed))
        self.surface = float("nan")
        self.k = 0
        t0 = args.approach * float(np.median([p.push / p.speed for p in self.paths]))
        while self.k * self.dt < t0:
            self.advance()

    def advance(self):
        t = self.k * self.dt
        self.g.set_tool_poses([p(t) for p in self.paths])
        self.g.step(1)
        self.k += 1

    def read_back(self, xs):
        self.g.read_positions_into(*xs)
        self.g.read_tool_forces()

    def d2h_bytes(self):
        return 3 * 4 * self.n + 6 * 4 * len(self.scenes)

    def h2d_bytes(self):
        return 13 * 4 * len(self.scenes)


class SceneGroup:
    """Separate scenes on one stream, driven like one: the unbatched form of
    a batch (each scene its own launch sequence every step)."""

    def __init__(self, scenes):
        self.scenes = scenes
        self.n = sum(s.n for s in scenes)

    def synchronize(self):
        for s in self.scenes:
            s.synchronize()

    def set_timing(self, on=True):
        for s in self.scenes:
            s.set_timing(on)

    def set_solver(self, iters, tol=0.0, every=10):
        for s in self.scenes:
            s.set_solver(iters, tol, every)

    def stats(self) -> dict:
        out = None
        for s in self.scenes:
            st = s.stats()
            if out is None:
                out = st
                out["n_colours"] = [st["n_colours"]]
                out["colour_rounds"] = [st["colour_rounds"]]
                out["residual"] = [st["residual"]]
                continue
            for k in ("n_contacts", "n_pp", "n_static", "kernel_launches", "sweep_contacts_pp",
                      "sweep_contacts_static", "sum_contacts", "solved_steps"):
                out[k] += st[k]
            out["n_colours"].append(st["n_colours"])
            out["colour_rounds"].append(st["colour_rounds"])
            out["residual"].append(st["residual"])
            for k in out["phase_ms"]:
                out["phase_ms"][k] += st["phase_ms"][k]
        out["n_colours"] = max(out["n_colours"])
        out["colour_rounds"] = max(out["colour_rounds"])
        out["residual"] = max(out["residual"])
        out["solved_steps"] //= len(self.scenes)
        return out

    def close(self):
        for s in self.scenes:
            s.close()


class UnbatchedSim(BatchedSim):
    """The batch's beds settled and approached in the batch (untimed), then
    stepped as separate scenes, one launch sequence per bed and step."""

    def __init__(self, tds, S, scenes, stream, args):
        super().__init__(tds, S, scenes, stream, args)
        self.tds, self.stream = tds, stream

    def settle_and_approach(self, between=None):
        super().settle_and_approach(None)  # the separate scenes keep the default shapes
        parts = []
        for q, s in enumerate(self.scenes):
            st = self.g.read_scene(q)
            sc = dict(s)
            sc["x"], sc["v"], sc["w"] = st["x"], st["v"], st["w"]
            sc["tool"] = self.paths[q](self.k * self.dt)
            parts.append(sc)
        self.g.close()
        self.g = SceneGroup([self.tds.Scene(sc, stream=self.stream) for sc in parts])

    def advance(self):
        if not isinstance(self.g, SceneGroup):  # settling and approach run in the batch
            return BatchedSim.advance(self)
        t = self.k * self.dt
        for p, g in zip(self.paths, self.g.scenes):
            g.set_tool_pose(p(t))
            g.step(1)
        self.k += 1

    def read_back(self, xs):
        o = 0
        for g in self.g.scenes:
            g.read_positions_into(xs[0][o:o + g.n], xs[1][o:o + g.n], xs[2][o:o + g.n])
            g.read_tool_force()
            o += g.n


def time_aggregates(g, work, stream, reps: int) -> dict:
    """Aggregate bodies of four zones per scene (quarters of each bed's
    footprint, full height) on the current state: CUDA-event time per call
    (kernels, the zone upload and the result read-back)."""
    import torch

    from paper_2011_00459_gb300 import scenes as S

    beds = work if isinstance(work, list) else [work]
    zones = []
    for q, sc in enumerate(beds[:16]):
        lx, ly = sc["footprint"]
        for i in range(2):
            for j in range(2):
                zones.append({"scene": q, "planes": S.box_planes(((i + 0.5) * lx / 2, (j + 0.5) * ly / 2, 5.0),
                                                                 (lx / 4, ly / 4, 10.0))})
    out = g.aggregate_bodies(zones)  # warm
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        out = g.aggregate_bodies(zones)
    e1.record(stream)
    e1.synchronize()
    return {"zones": len(zones), "particles_in_zones": int(sum(o["count"] for o in out)),
            "ms_per_call": e0.elapsed_time(e1) / reps}


def time_fields(g, work, stream, reps: int, tds) -> dict:
    """Coarse-grained fields of the first bed on 0.1 m voxels (voxel kernel and
    Gaussian with R = l0) and one advection step on that grid: CUDA-event
    time per call."""
    import torch

    sc = work[0] if isinstance(work, list) else work
    lx, ly = sc["footprint"]
    l0 = 0.1
    dims = (int(np.ceil(lx / l0)) + 2, int(np.ceil(ly / l0)) + 2, 20)
    grid = tds.make_grid((-l0, -l0, -0.2), l0, dims, 0)
    out = {"voxels": int(np.prod(dims)), "l0": l0}
    for name, kernel, R in (("voxel_kernel_ms", 0, 0.0), ("gaussian_kernel_ms", 1, l0)):
        g.coarse_grain(grid, kernel, R)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            rho, p, u = g.coarse_grain(grid, kernel, R)
        e1.record(stream)
        e1.synchronize()
        out[name] = e0.elapsed_time(e1) / reps
    dt = float(l0 / (3.0 * max(float(u.abs().max()), 1e-6)))
    a = rho.clone()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        a = tds.advect_fluid(grid, u, a, dt, stream=stream)
    e1.record(stream)
    e1.synchronize()
    out["advect_ms"] = e0.elapsed_time(e1) / reps
    return out


class _Parked:
    """A sim whose steps keep the tools where they are (parked): what the
    autotuner steps while it times launch shapes."""

    def __init__(self, sim):
        self.g = sim.g

    def advance(self):
        self.g.step(1)


def prepare(args, work, tds, S, stream, replay=None):
    """Creates the sim, settles it, picks the launch shapes (autotuned on the
    settled bed, tools parked; or ``replay``'s shape with the same number of
    parked steps, so the trajectory repeats), approaches and warms up."""
    if isinstance(work, list):
        sim = (UnbatchedSim if args.unbatched else BatchedSim)(tds, S, work, stream, args)
    else:
        sim = PlainSim(tds, S, work, stream, args)
    tuned = {}

    def between() -> int:
        """Sets the launch shapes during the settle; returns the settle steps taken."""
        g = sim.g
        if args.pgs_sync >= 0 or args.pgs_blocks or args.pgs_shape:
            t, per = (int(v) for v in args.pgs_shape.split("x")) if args.pgs_shape else (0, 0)
            g.set_launch_config(pgs_blocks=args.pgs_blocks, pgs_sync=None if args.pgs_sync < 0 else args.pgs_sync,
                                pgs_threads=t, pgs_per_thread=per)
        elif replay is not None:
            g.set_launch_config(**replay["shape"])
            tuned.update(replay)
        elif not args.no_autotune:
            from paper_2011_00459_gb300 import autotune

            tuned.update(autotune.tune(_Parked(sim), sweeps=SETTLE_SWEEPS, use_cache=False,
                                       log=lambda m: log(args, m)))
            log(args, f"autotune: {tuned}")
            return int(tuned["steps"])
        return 0

    sim.settle_and_approach(between)
    for _ in range(args.warmup):
        sim.advance()
    sim.g.synchronize()
    sim.g.stats()  # reset the accumulators
    return sim, (tuned or None)


def run_tds(args, rank: int, world: int, local_rank: int):
    import torch

    from paper_2011_00459_gb300 import build as B
    from paper_2011_00459_gb300 import scenes as S
    from paper_2011_00459_gb300 import tds

    torch.cuda.set_device(local_rank)
    if rank == 0:
        B.build()
    if world > 1:
        torch.distributed.barrier()
        B.build()
    work = make_workload(args, rank)
    first = work[0] if isinstance(work, list) else work
    stream = torch.cuda.Stream()
    t_setup = time.time()
    with torch.cuda.stream(stream):
        sim, tuned = prepare(args, work, tds, S, stream)
        g, n = sim.g, sim.n
        log(args, f"setup {time.time() - t_setup:.1f}s, surface {sim.surface:.3f}")
        # ---- device-timed region ------------------------------------------------
        g.set_timing(True)
        clocks = Clocks(local_rank)
        clocks.start()
        time.sleep(0.3)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        launches0 = g.stats()["kernel_launches"]
        torch.cuda.nvtx.range_push("timed")
        e0.record(stream)
        for _ in range(args.steps):
            sim.advance()
        e1.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        clk = clocks.stop()
        st = g.stats()
        launches = st["kernel_launches"] - launches0
        ms = reduce_max(ms, world)
        n_all = reduce_sum(n, world)
        g.set_timing(False)
        # ---- fixed sweeps (the roofline region), same bed continuing its dig ----
        fixed = None
        if first.get("tol", 0) > 0 and first["fixed_iters"] > 0:
            g.set_solver(int(first["fixed_iters"]), 0.0, 10)
            for _ in range(2):
                sim.advance()
            g.synchronize()
            g.stats()
            g.set_timing(True)
            torch.cuda.synchronize()
            f0 = torch.cuda.Event(enable_timing=True)
            f1 = torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            for _ in range(args.steps):
                sim.advance()
            f1.record(stream)
            torch.cuda.synchronize()
            fms = f0.elapsed_time(f1)
            fst = g.stats()
            g.set_timing(False)
            fms = reduce_max(fms, world)
            fixed = {"ms": fms, "st": fst, "sweeps": int(first["fixed_iters"])}
        agg = fields = None
        if not isinstance(g, SceneGroup):
            agg = time_aggregates(g, work, stream, args.steps)
            fields = time_fields(g, work, stream, args.steps, tds)
        one = g.scenes[0] if isinstance(g, SceneGroup) else g
        launch_cfg = one.launch_config()
        if isinstance(work, list) and not isinstance(g, SceneGroup):
            sv = g.read_solve()  # each bed's own solve in the last timed step
            r, k = sv["residual"].astype(np.float64), sv["sweeps"].astype(np.int64)
            launch_cfg["per_bed"] = {
                "beds": int(len(r)), "max_final_residual": float(r.max()),
                "beds_above_tol": int((r > first.get("tol", 0.0)).sum()) if first.get("tol", 0) > 0 else None,
                "beds_at_sweep_cap": int((k >= int(first["iters"])).sum()),
                "sweeps_min_median_max": [int(k.min()), float(np.median(k)), int(k.max())]}
        if tuned:
            launch_cfg["autotune"] = {k: tuned[k] for k in ("source", "ms", "default_ms", "steps") if k in tuned}
        g.close()
        # ---- end-to-end through the C ABI with host buffers ---------------------
        # a second, identical preparation: the same settled bed, launch shapes,
        # approach and warm-up, so the e2e loop times the same steps as above
        e2e = None
        if not args.no_e2e:
            sim, _ = prepare(args, work, tds, S, stream, replay=tuned)
            g = sim.g
            xs = [torch.empty(n, dtype=torch.float32).pin_memory().numpy() for _ in range(3)]
            if world > 1:
                torch.distributed.barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(args.steps):
                sim.advance()
                sim.read_back(xs)
            t_e2e = time.perf_counter() - t0
            est = g.stats()
            t_e2e = reduce_max(t_e2e, world)
            e2e = {"value": n_all * args.steps / t_e2e, "unit": UNIT,
                   "h2d_bytes_per_step": sim.h2d_bytes(), "d2h_bytes_per_step": sim.d2h_bytes(),
                   "mean_sweeps": (est["sweep_contacts_pp"] + est["sweep_contacts_static"])
                   / max(1, est["sum_contacts"]),
                   "steps": "the same steps as the device-timed region (identical preparation)"}
            g.close()
    launch_cfg["aggregate_bodies"] = agg
    launch_cfg["fields"] = fields
    return work, n_all, ms, st, launches, clk, e2e, fixed, launch_cfg


# ---------------------------------------------------------------------------
# the oracle on a bounded sample of the same workload
# ---------------------------------------------------------------------------
def cpu_model() -> str:
    """The host CPU's model name (/proc/cpuinfo, else lscpu on Arm hosts)."""
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform

    return platform.processor() or platform.machine()


def oracle_sample(scene: dict, seconds: float, seed: int, steps: int | None = None, warmup: int = 0,
                  threads: int = 1):
    """A column of the same bed (same radii, material, sweeps), spawned by the
    same lattice generator over a 0.5 x 0.5 m footprint of the same height,
    settled by the oracle itself (untimed), ``warmup`` untimed steps of the
    full solve, then timed for steps of the full solve; ``threads`` > 1
    updates the contacts of each colour on that many threads (the same
    results bit for bit). Returns (particle-steps/s, description, steps timed,
    mean sweeps per timed step)."""
    from oracle import oracle
    from paper_2011_00459_gb300 import scenes as S

    n_full = len(scene["r"])
    lx, ly = scene["footprint"]
    frac = (0.5 * 0.5) / (lx * ly)
    n = max(200, int(round(n_full * frac)))
    r_lo, r_hi = float(scene["r"].min()), float(scene["r"].max())
    x, r = S.lattice_spawn(n, 0.5, 0.5, r_lo, r_hi, 0.0, seed)
    p = dict(scene)
    if p.get("tol", 0) > 0 and not p.get("residual_every"):
        p["residual_every"] = 5  # the oracle checks at a fixed period
    p["walls"] = S.bed_walls(0.5, 0.5, 6.0)
    p["hf"] = S.flat_heightfield(12, 12, -0.05, -0.05, 0.05)
    p["tool_boxes"] = np.zeros((0, 10), np.float32)
    col = S.with_particles(p, x, r)
    st = oracle.State(col)
    for _ in range(60):  # settle (untimed) with fewer sweeps
        oracle.step(col, st, iters=20)
    for _ in range(warmup):  # untimed steps of the full solve
        oracle.step(col, st)
    t0 = time.perf_counter()
    k = 0
    sweeps = 0
    while True:
        sweeps += oracle.step(col, st, threads=threads)["iterations"]
        k += 1
        el = time.perf_counter() - t0
        if (steps is not None and k >= steps) or (steps is None and el >= seconds):
            break
    who = "1 thread" if threads <= 1 else f"{threads} threads (each colour's contacts split among them)"
    desc = (f"FP64 oracle, {who}: {n}-sphere column (0.5x0.5 m footprint) of the same bed, "
            f"oracle-settled 60 steps and {warmup} full steps untimed, then {k} steps timed, "
            f"PGS to {_solve_desc(scene)} ({sweeps / k:.1f} sweeps per step)")
    return n * k / el, desc, k, sweeps / k


def cpu_baseline(scene: dict, seconds: float, seed: int, warmup: int, gpu_sweeps: float | None) -> dict:
    """The oracle on one thread for about ``seconds``, then on all host cores
    (the reported baseline) over exactly the same steps from the same state
    (the same results bit for bit, so the same sweeps), with the CPU model,
    the oracle's sweeps per step and the GPU's."""
    cores = os.cpu_count() or 1
    v1, d1, k, sw1 = oracle_sample(scene, seconds, seed, warmup=warmup, threads=1)
    val, desc, _, sw = oracle_sample(scene, 0.0, seed, steps=k, warmup=warmup, threads=cores)
    return {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc,
            "sweeps_per_step": sw, "gpu_sweeps_per_step": gpu_sweeps, "cpu_model": cpu_model(),
            "single_thread": {"value": v1, "unit": UNIT, "cores": 1, "sample": d1, "sweeps_per_step": sw1}}


def learned_form(args, launch_cfg, stream, same_as: str = "the headline", cold: bool = False) -> dict:
    """The learned warm start on the workload of ``args``: an identical
    preparation (same settle, launch shapes, approach and warm-up with the
    previous-step warm start), then the same timed steps with the network
    trained on plain solves of the small and bulldozing beds (weights shipped
    with the package). ``cold``: the same steps started from zero impulses
    instead (plain PGS without any warm start)."""
    import torch

    from paper_2011_00459_gb300 import learned as LR
    from paper_2011_00459_gb300 import scenes as S
    from paper_2011_00459_gb300 import tds

    work = make_workload(args, 0)
    replay = {"shape": {k: launch_cfg[k] for k in ("pgs_blocks", "pgs_sync", "colour_blocks", "pgs_threads",
                                                   "pgs_per_thread")}}
    with torch.cuda.stream(stream):
        sim, _ = prepare(args, work, tds, S, stream, replay=replay)
        g = sim.g
        if cold:
            g.set_warm_start(tds.WARM_COLD)
        else:
            g.set_mlp_weights(LR.load_weights())
            g.set_warm_start(tds.WARM_LEARNED)
        g.stats()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            sim.advance()
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        st = g.stats()
        g.close()
    return {"warm_start": "cold (zero impulses)" if cold else "learned (10-64-64-3 BF16 network)",
            "value": sim.n * args.steps / (ms * 1e-3),
            "unit": UNIT, "ms_per_step": ms / args.steps,
            "mean_sweeps": (st["sweep_contacts_pp"] + st["sweep_contacts_static"]) / max(1, st["sum_contacts"]),
            "final_residual": st["residual"], "steps": f"the same steps as {same_as} (identical preparation)"}


def paired_learned(args, launch_cfg, stream, same_as: str = "the headline") -> dict:
    """The learned warm start against the previous-step one from identical
    states: at every step of the trajectory the state is saved, the step is
    taken with the network's initial impulses (its sweeps recorded), the state
    is restored and the step is taken with the previous-step ones (the
    trajectory continues from there). Untimed: sweeps only."""
    import torch

    from paper_2011_00459_gb300 import learned as LR
    from paper_2011_00459_gb300 import scenes as S
    from paper_2011_00459_gb300 import tds

    work = make_workload(args, 0)
    replay = {"shape": {k: launch_cfg[k] for k in ("pgs_blocks", "pgs_sync", "colour_blocks", "pgs_threads",
                                                   "pgs_per_thread")}}
    sweeps = lambda st: (st["sweep_contacts_pp"] + st["sweep_contacts_static"]) / max(1, st["sum_contacts"])
    with torch.cuda.stream(stream):
        sim, _ = prepare(args, work, tds, S, stream, replay=replay)
        g = sim.g
        g.set_mlp_weights(LR.load_weights())
        prev, learned = [], []
        for _ in range(args.steps):
            saved = g.save_state()
            g.set_warm_start(tds.WARM_LEARNED)
            g.stats()
            sim.advance()
            learned.append(sweeps(g.stats()))
            g.load_state(saved)
            sim.k -= 1
            g.set_warm_start(tds.WARM_PREV)
            sim.advance()
            prev.append(sweeps(g.stats()))
        g.close()
    p, l = np.array(prev), np.array(learned)
    return {"steps": f"{args.steps} steps of {same_as}'s trajectory, each solved from the same state both ways",
            "mean_sweeps_previous_step": float(p.mean()), "mean_sweeps_learned": float(l.mean()),
            "sweeps_saved": float(1.0 - l.sum() / p.sum()),
            "steps_fewer": int((l < p).sum()), "steps_more": int((l > p).sum())}


def batched_args(args):
    import copy

    a = copy.copy(args)
    a.workload, a.no_e2e, a.roofline_sweeps, a.no_cpu_baseline = "batched", True, 0, True
    return a


def batched_form(args, rank: int, world: int, local_rank: int) -> tuple:
    """The batched workload (256 beds in one graph-replayed batch) at the same
    residual, timed like the headline; also returns its launch shape."""
    a = batched_args(args)
    work, n_all, ms, st, launches, clk, e2e, fixed, launch_cfg = run_tds(a, rank, world, local_rank)
    beds = launch_cfg.pop("per_bed", None)
    return ({"workload": describe(work, a)["workload"], "value": n_all * a.steps / (ms * 1e-3), "unit": UNIT,
             "ms_per_step": ms / a.steps, "warm_start": "previous step",
             "mean_sweeps": (st["sweep_contacts_pp"] + st["sweep_contacts_static"]) / max(1, st["sum_contacts"]),
             "final_residual": st["residual"], "per_bed_last_step": beds, "gpu_launches": int(launches)},
            launch_cfg)


def unbatched_form(args, rank: int, world: int, local_rank: int, steps: int = 3) -> dict:
    """The batch's beds stepped one scene at a time (each bed its own launch
    sequence every step) against the batch itself, on identical preparations
    and the same steps; each form stops at its own residual test (the batch:
    one norm over all beds; a separate bed: its own)."""
    out = {}
    for unb in (False, True):
        a = batched_args(args)
        a.steps, a.unbatched = min(args.steps, steps), unb
        work, n_all, ms, st, launches, clk, e2e, fixed, launch_cfg = run_tds(a, rank, world, local_rank)
        out["unbatched" if unb else "batched"] = {
            "value": n_all * a.steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / a.steps,
            "mean_sweeps": (st["sweep_contacts_pp"] + st["sweep_contacts_static"]) / max(1, st["sum_contacts"]),
            "gpu_launches": int(launches)}
    out["steps"] = min(args.steps, steps)
    out["scenes"] = len(work)
    out["speedup"] = out["batched"]["value"] / out["unbatched"]["value"]
    return out


CONFIG_FORMS = (("small", 1), ("bulldozing", 2), ("excavation", 3))


def config_form(args, name: str, rank: int, world: int, local_rank: int, steps: int = 10) -> dict:
    """Another of the workload's configurations, timed like the headline: the
    same metric (every step solved to the residual of ``args``, previous-step
    warm start) and, where the configuration fixes a sweep count, a second
    region at that count. The excavation configuration adds the same steps
    from a cold start and with the learned warm start, and the learned warm
    start paired with the previous-step one from identical states."""
    import copy

    import torch

    a = copy.copy(args)
    a.workload, a.n, a.scenes, a.no_e2e, a.no_cpu_baseline = name, 0, 0, True, True
    a.steps = min(args.steps, steps)
    a.roofline_sweeps = 0 if name == "excavation" else -1
    work, n_all, ms, st, launches, clk, e2e, fixed, launch_cfg = run_tds(a, rank, world, local_rank)
    msw = lambda q: (q["sweep_contacts_pp"] + q["sweep_contacts_static"]) / max(1, q["sum_contacts"])
    out = {"workload": describe(work, a)["workload"], "particles": int(n_all), "steps": a.steps,
           "warm_start": "previous step", "value": n_all * a.steps / (ms * 1e-3), "unit": UNIT,
           "ms_per_step": ms / a.steps, "mean_sweeps": msw(st), "final_residual": st["residual"],
           "contacts_per_step": st["sum_contacts"] / max(1, st["solved_steps"]), "colours": st["n_colours"],
           "gpu_launches": int(launches)}
    if fixed:
        out["fixed_sweeps"] = {"sweeps": fixed["sweeps"], "value": n_all * a.steps / (fixed["ms"] * 1e-3),
                               "unit": UNIT, "ms_per_step": fixed["ms"] / a.steps}
    if name == "excavation":
        out["cold"] = learned_form(a, launch_cfg, torch.cuda.Stream(), "the excavation configuration", cold=True)
        out["learned"] = learned_form(a, launch_cfg, torch.cuda.Stream(), "the excavation configuration")
        out["learned_paired"] = paired_learned(a, launch_cfg, torch.cuda.Stream(), "the excavation configuration")
    return out


def sample_scene(work) -> dict:
    """The scene the oracle samples: the bed itself, or the batch's bed of
    median size."""
    if not isinstance(work, list):
        return work
    ns = [len(s["r"]) for s in work]
    return work[int(np.argsort(ns)[len(ns) // 2])]


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return 0
    from oracle import oracle

    oracle.build()
    work = make_workload(args, 0)
    scene = sample_scene(work)
    steps = max(1, args.steps)
    cores = os.cpu_count() or 1
    val, desc, k, sw = oracle_sample(scene, 0.0, args.seed, steps=steps, warmup=args.warmup, threads=cores)
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT,
           "n_gpus": args.gpus, "steps": k, "warmup": args.warmup, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": describe(work, args),
           "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": desc, "sweeps_per_step": sw, "cpu_model": cpu_model()},
           "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    import torch

    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    work, n_all, ms, st, launches, clk, e2e, fixed, launch_cfg = run_tds(args, rank, world, local_rank)
    peaks = measured_peaks()
    # roofline of k_pgs: over the fixed-sweep region when there is one (every
    # launch then does the same sweeps), else over the headline region
    rst = fixed["st"] if fixed else st
    pgs_ms = rst["phase_ms"]["pgs"]
    alg_bytes = BYTES_PP * rst["sweep_contacts_pp"] + BYTES_STATIC * rst["sweep_contacts_static"]
    achieved = alg_bytes / (pgs_ms * 1e-3) / 1e9 if pgs_ms > 0 else 0.0
    per = ncu_traffic(args.workload)
    sweeps_contacts = rst["sweep_contacts_pp"] + rst["sweep_contacts_static"]
    traffic = per * sweeps_contacts / max(1, rst["solved_steps"]) if per is not None else None
    phase = lambda q: {k: v / max(1, q["timed_steps"]) for k, v in q["phase_ms"].items()}
    result = {
        "metric": METRIC, "value": n_all * args.steps / (ms * 1e-3), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {**describe(work, args), "parallelism": f"replicas{world}" if world > 1 else "single",
                   "contacts_per_step": st["sum_contacts"] / max(1, st["solved_steps"]),
                   "colours": st["n_colours"], "colour_rounds": st["colour_rounds"],
                   "mean_sweeps": (st["sweep_contacts_pp"] + st["sweep_contacts_static"]) / max(1, st["sum_contacts"]),
                   "final_residual": st["residual"],
                   "launch": launch_cfg,
                   "phase_ms_per_step": phase(st)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                     "kernel": "k_pgs (persistent colour-sweep PGS)",
                     "region": (f"second timed region: {fixed['sweeps']} fixed sweeps per step, {args.steps} "
                                f"steps of the same bed continuing its dig" if fixed else "the headline region"),
                     "peak_source": peaks["source"] + " HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"},
        "gpu_launches": int(launches),
        "clocks": clk,
        "e2e": e2e,
    }
    if fixed:
        fs = fixed["st"]
        result["fixed_sweeps"] = {
            "sweeps": fixed["sweeps"], "value": n_all * args.steps / (fixed["ms"] * 1e-3), "unit": UNIT,
            "ms_per_step": fixed["ms"] / args.steps,
            "contacts_per_step": fs["sum_contacts"] / max(1, fs["solved_steps"]),
            "phase_ms_per_step": phase(fs)}
    if world == 1 and not args.no_forms and args.workload != "batched" and args.tol > 0:
        import torch

        result["forms"] = {"plain": {"warm_start": "previous step", "value": result["value"],
                                     "ms_per_step": result["ms_per_step"],
                                     "mean_sweeps": result["config"]["mean_sweeps"]}}
        try:
            result["forms"]["learned"] = learned_form(args, launch_cfg, torch.cuda.Stream())
        except Exception as exc:  # a form that cannot run is reported, not fatal
            result["forms"]["learned"] = {"error": repr(exc)}
        try:
            result["forms"]["learned_paired"] = paired_learned(args, launch_cfg, torch.cuda.Stream())
        except Exception as exc:
            result["forms"]["learned_paired"] = {"error": repr(exc)}
        if args.workload == "large":
            try:
                result["forms"]["batched"], bcfg = batched_form(args, rank, world, local_rank)
                result["forms"]["batched_learned"] = learned_form(batched_args(args), bcfg, torch.cuda.Stream(),
                                                                  "the batched form")
            except Exception as exc:
                result["forms"].setdefault("batched", {"error": repr(exc)})
                result["forms"].setdefault("batched_learned", {"error": repr(exc)})
            try:
                result["forms"]["batched_learned_paired"] = paired_learned(batched_args(args), bcfg,
                                                                           torch.cuda.Stream(), "the batched form")
            except Exception as exc:
                result["forms"]["batched_learned_paired"] = {"error": repr(exc)}
            try:
                result["forms"]["batched_vs_unbatched"] = unbatched_form(args, rank, world, local_rank)
            except Exception as exc:
                result["forms"]["batched_vs_unbatched"] = {"error": repr(exc)}
            result["configs"] = {}
            for name, num in CONFIG_FORMS:
                try:
                    result["configs"][name] = {"config": num, **config_form(args, name, rank, world, local_rank)}
                except Exception as exc:
                    result["configs"][name] = {"config": num, "error": repr(exc)}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import oracle

        oracle.build()
        result["cpu_baseline"] = cpu_baseline(sample_scene(work), args.cpu_seconds, args.seed, args.warmup,
                                              result["config"]["mean_sweeps"])
    if rank == 0:
        print(json.dumps(result))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
