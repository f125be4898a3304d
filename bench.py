"""Benchmark of the active-soil particle step (particle-steps/s) on GB300.

Default workload: the 1 000 000-sphere excavation bed (r ~ U[0.02, 0.03] m,
8 x 8 m, 1024^2 heightfield, 12-box bucket on a seeded spline dig, c_p 5 kPa,
100 PGS sweeps per step, previous-step warm start). The bed is spawned on a
jittered lattice and settled untimed on the GPU; the bucket then approaches
its deepest cut untimed, and the timed steps dig.

  value   = particles x timed steps / device time of those steps (CUDA events
            on the scene's stream, state resident in HBM)
  e2e     = the same through the C ABI with host buffers: every step sets the
            tool pose from the host and reads positions and tool force back
            into pinned host memory
  roofline: the persistent PGS kernel, algorithmic bytes (204 B per
            particle-pair contact and 160 B per static contact per sweep)
            over its CUDA-event time, against the measured HBM copy peak
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
BYTES_PP = 204.0      # per particle-pair contact per sweep
BYTES_STATIC = 160.0  # per static contact per sweep


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tds", choices=["tds", "reference"])
    ap.add_argument("--workload", default="large")
    ap.add_argument("--n", type=int, default=0, help="override the particle count")
    ap.add_argument("--iters", type=int, default=0, help="override the sweeps per step")
    ap.add_argument("--settle", type=int, default=-1)
    ap.add_argument("--approach", type=float, default=0.3,
                    help="fraction of the dig path covered untimed before timing")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--tol", type=float, default=0.0,
                    help="residual mode: stop each step's solve at this residual (cap --max-iters)")
    ap.add_argument("--max-iters", type=int, default=2000)
    ap.add_argument("--cold", action="store_true", help="cold start instead of previous-step impulses")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
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
    h = hashlib.sha256()
    for f in ("tds_solve.cu", "tds_internal.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2011_00459_gb300", "csrc", f), "rb").read())
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
def make_workload(args, rank: int) -> dict:
    from paper_2011_00459_gb300 import scenes as S

    gen = S.WORKLOADS[args.workload]
    kw = {"n": args.n} if args.n else {}
    scene = gen(seed=args.seed + rank, **kw)
    if args.iters:
        scene["iters"] = args.iters
    if args.tol > 0:
        scene["tol"] = args.tol
        scene["iters"] = args.max_iters
        scene["residual_every"] = 5
    if args.cold:
        scene["warm_start"] = 0
    return scene


def describe(scene: dict, args) -> dict:
    return {
        "workload": f"{scene['name']}: {len(scene['r'])} spheres r~U[{scene['r'].min():.3f},"
                    f"{scene['r'].max():.3f}] m, {scene['footprint'][0]:g}x{scene['footprint'][1]:g} m "
                    f"walled bed, {scene['hf']['nx']}x{scene['hf']['ny']} heightfield, "
                    f"{len(scene['tool_boxes'])}-box {scene['tool_kind']}, c_p {scene['cohesion']:g} Pa, "
                    f"{scene['iters']} PGS sweeps/step, previous-step warm start",
        "particles": int(len(scene["r"])), "sweeps": int(scene["iters"]), "dt": scene["dt"],
        "solve": (f"residual <= {scene['tol']:g} (cap {scene['iters']} sweeps)" if scene.get("tol", 0) > 0
                  else f"{scene['iters']} sweeps"),
        "warm_start": "previous step" if scene.get("warm_start", 1) else "cold",
        "seed": args.seed, "l2": "inputs larger than L2 (contact rows and impulses > 129 MB)",
    }


def settle_and_approach(g, scene, args, S):
    """Untimed: settle the spawned bed with the tool parked, then move the
    tool along its path up to the start of the timed region."""
    settle = scene["settle_steps"] if args.settle < 0 else args.settle
    g.set_tool_pose(S.parked_tool(scene))
    g.set_solver(30)
    for _ in range(settle):
        g.step(1)
    g.set_solver(int(scene["iters"]), float(scene.get("tol", 0.0)), int(scene.get("residual_every", 10)))
    parts = g.read_particles()
    surface = S.surface_level(parts["x"], scene["r"])
    path = S.tool_path(scene, surface, seed=args.seed)
    dt = scene["dt"]
    length = getattr(path, "length", None)
    t0 = 0.0
    if length is not None:
        t0 = args.approach * length / path.speed
    else:
        t0 = args.approach * path.push / path.speed
    k = 0
    while k * dt < t0:
        g.set_tool_pose(path(k * dt))
        g.step(1)
        k += 1
    return path, k, surface


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
    scene = make_workload(args, rank)
    n = len(scene["r"])
    stream = torch.cuda.Stream()
    t_setup = time.time()
    with torch.cuda.stream(stream):
        g = tds.Scene(scene, stream=stream)
        path, k, surface = settle_and_approach(g, scene, args, S)
        dt = scene["dt"]
        for _ in range(args.warmup):
            g.set_tool_pose(path(k * dt))
            g.step(1)
            k += 1
        g.synchronize()
        g.stats()  # reset the accumulators
        log(args, f"setup {time.time() - t_setup:.1f}s, surface {surface:.3f}")
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
            g.set_tool_pose(path(k * dt))
            g.step(1)
            k += 1
        e1.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        clk = clocks.stop()
        st = g.stats()
        launches = st["kernel_launches"] - launches0
        if world > 1:
            t = torch.tensor([ms], device="cuda")
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            ms = float(t.item())
            tot = torch.tensor([float(n)], device="cuda")
            torch.distributed.all_reduce(tot)
            n_all = float(tot.item())
        else:
            n_all = float(n)
        g.set_timing(False)
        # ---- end-to-end through the C ABI with host buffers ---------------------
        e2e = None
        if not args.no_e2e:
            xs = [torch.empty(n, dtype=torch.float32).pin_memory().numpy() for _ in range(3)]
            for _ in range(2):  # warm the read path
                g.set_tool_pose(path(k * dt)); g.step(1); k += 1
                g.read_positions_into(*xs); g.read_tool_force()
            if world > 1:
                torch.distributed.barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(args.steps):
                g.set_tool_pose(path(k * dt))
                g.step(1)
                k += 1
                g.read_positions_into(*xs)
                g.read_tool_force()
            t_e2e = time.perf_counter() - t0
            if world > 1:
                t = torch.tensor([t_e2e], device="cuda")
                torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
                t_e2e = float(t.item())
            e2e = {"value": n_all * args.steps / t_e2e, "unit": UNIT,
                   "h2d_bytes_per_step": 13 * 4, "d2h_bytes_per_step": 3 * 4 * n + 6 * 4}
        g.close()
    return scene, n_all, ms, st, launches, clk, e2e


# ---------------------------------------------------------------------------
# the oracle on a bounded sample of the same workload
# ---------------------------------------------------------------------------
def oracle_sample(scene: dict, seconds: float, seed: int, steps: int | None = None):
    """A column of the same bed (same radii, material, sweeps), spawned by the
    same lattice generator over a 0.5 x 0.5 m footprint of the same height,
    settled by the oracle itself (untimed), then timed for steps of the full
    sweep count. Returns (particle-steps/s, description, steps timed)."""
    from oracle import oracle
    from paper_2011_00459_gb300 import scenes as S

    n_full = len(scene["r"])
    lx, ly = scene["footprint"]
    frac = (0.5 * 0.5) / (lx * ly)
    n = max(200, int(round(n_full * frac)))
    r_lo, r_hi = float(scene["r"].min()), float(scene["r"].max())
    x, r = S.lattice_spawn(n, 0.5, 0.5, r_lo, r_hi, 0.0, seed)
    p = dict(scene)
    p["walls"] = S.bed_walls(0.5, 0.5, 6.0)
    p["hf"] = S.flat_heightfield(12, 12, -0.05, -0.05, 0.05)
    p["tool_boxes"] = np.zeros((0, 10), np.float32)
    col = S.with_particles(p, x, r)
    st = oracle.State(col)
    for _ in range(60):  # settle (untimed) with fewer sweeps
        oracle.step(col, st, iters=20)
    t0 = time.perf_counter()
    k = 0
    while True:
        oracle.step(col, st)
        k += 1
        el = time.perf_counter() - t0
        if (steps is not None and k >= steps) or (steps is None and el >= seconds):
            break
    desc = (f"FP64 oracle, 1 thread: {n}-sphere column (0.5x0.5 m footprint) of the same bed, "
            f"oracle-settled 60 steps untimed, then {k} steps of {scene['iters']} sweeps timed")
    return n * k / el, desc, k


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return 0
    from oracle import oracle

    oracle.build()
    scene = make_workload(args, 0)
    steps = max(1, args.steps)
    val, desc, k = oracle_sample(scene, 0.0, args.seed, steps=steps)
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT,
           "n_gpus": args.gpus, "steps": k, "warmup": args.warmup, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": describe(scene, args),
           "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": desc},
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
    scene, n_all, ms, st, launches, clk, e2e = run_tds(args, rank, world, local_rank)
    peaks = measured_peaks()
    pgs_ms = st["phase_ms"]["pgs"]
    alg_bytes = BYTES_PP * st["sweep_contacts_pp"] + BYTES_STATIC * st["sweep_contacts_static"]
    achieved = alg_bytes / (pgs_ms * 1e-3) / 1e9 if pgs_ms > 0 else 0.0
    per = ncu_traffic(args.workload)
    sweeps_contacts = st["sweep_contacts_pp"] + st["sweep_contacts_static"]
    traffic = per * sweeps_contacts / max(1, st["solved_steps"]) if per is not None else None
    result = {
        "metric": METRIC, "value": n_all * args.steps / (ms * 1e-3), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {**describe(scene, args), "parallelism": f"replicas{world}" if world > 1 else "single",
                   "contacts_per_step": st["sum_contacts"] / max(1, st["solved_steps"]),
                   "colours": st["n_colours"], "colour_rounds": st["colour_rounds"],
                   "mean_sweeps": (st["sweep_contacts_pp"] + st["sweep_contacts_static"]) / max(1, st["sum_contacts"]),
                   "final_residual": st["residual"],
                   "phase_ms_per_step": {k: v / max(1, st["timed_steps"]) for k, v in st["phase_ms"].items()}},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                     "kernel": "k_pgs (persistent colour-sweep PGS)",
                     "peak_source": peaks["source"] + " HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"},
        "gpu_launches": int(launches),
        "clocks": clk,
        "e2e": e2e,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import oracle

        oracle.build()
        val, desc, _ = oracle_sample(scene, args.cpu_seconds, args.seed)
        result["cpu_baseline"] = {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                                  "sample": desc}
    if rank == 0:
        print(json.dumps(result))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
