"""Launch-shape autotuner (host-side search; the timed work is the library's
own step).

The knobs are the runtime launch shapes of ``tds_set_launch_config``: the
persistent solver's CTA count and its synchronisation between colours
(neighbour flags or a grid barrier) and the persistent colouring's CTA count.
Every setting gives bit-identical results, so the tuner only picks the
fastest: it times a few steps of the caller's own scene (continuing its
motion) per candidate with CUDA events on the scene's stream and keeps the
best. Choices are cached as JSON per GPU model and workload shape (particles
rounded to two significant digits, and scenes), so a later run with the same
shape reuses them without timing.
"""
from __future__ import annotations

import json
import math
import os
import tempfile

CACHE_ENV = "TDS_AUTOTUNE_CACHE"


def cache_path() -> str:
    p = os.environ.get(CACHE_ENV)
    if p:
        return p
    base = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    return os.path.join(base, "tds", "autotune.json")


def _round2(x: float) -> int:
    """x rounded to two significant digits (0 stays 0)."""
    if x <= 0:
        return 0
    e = int(math.floor(math.log10(x))) - 1
    return int(round(x / 10 ** e) * 10 ** e)


def shape_key(gpu: str, particles: int, scenes: int) -> str:
    return f"{gpu}|n={_round2(particles)}|scenes={scenes}"


def load_cache(path: str | None = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}  # missing or unreadable cache: tune again


def store_cache(key: str, entry: dict, path: str | None = None) -> None:
    """Adds one entry; written atomically (temporary file, then rename)."""
    path = path or cache_path()
    data = load_cache(path)
    data[key] = entry
    d = os.path.dirname(path) or "."
    os.makedirs(d, exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=d, prefix=".autotune.")
    with os.fdopen(fd, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


SYNC_MODES = (1, 0)  # neighbour synchronisation, grid barrier
# solver CTA shapes the library compiles: (threads, contacts per thread, CTAs per SM)
SHAPES = ((416, 1, 2), (768, 1, 1), (512, 2, 1), (640, 2, 1), (512, 3, 1), (256, 1, 3))
KEYS = ("pgs_blocks", "pgs_sync", "colour_blocks", "pgs_threads", "pgs_per_thread")


def candidates(cfg: dict, sms: int) -> list:
    """Solver shapes to time first (sync mode x solver CTA shape), the
    library's defaults first. A shape keeps the default's share of the
    machine: its CTAs scale with its CTAs per SM."""
    base = {k: cfg[k] for k in KEYS}
    per_sm = {(t, p): k for t, p, k in SHAPES}
    k0 = per_sm.get((base["pgs_threads"], base["pgs_per_thread"]), 1)
    out = [base]
    for sync in SYNC_MODES:
        for t, per, k in SHAPES:
            blocks = max(1, min(sms * k, (base["pgs_blocks"] * k) // k0))
            shape = dict(base, pgs_sync=sync, pgs_threads=t, pgs_per_thread=per, pgs_blocks=blocks)
            if shape not in out:
                out.append(shape)
    return out


def block_candidates(cfg: dict, best: dict) -> list:
    """Fewer solver CTAs on the chosen solver shape."""
    p = max(1, (3 * best["pgs_blocks"]) // 4)
    return [dict(best, pgs_blocks=p)] if p != best["pgs_blocks"] else []


def colour_candidates(cfg: dict, best: dict, sms: int) -> list:
    """Colouring CTAs to time on the chosen solver shape (the colouring and
    the solver are separate kernels, so the two choices do not interact)."""
    maxc = cfg["max_colour_blocks"]
    col = sorted({min(maxc, c) for c in (cfg["colour_blocks"], sms, 2 * sms, maxc) if c >= 1}, reverse=True)
    return [dict(best, colour_blocks=c) for c in col if c != best["colour_blocks"]]


def time_steps(sim, steps: int) -> float:
    """Milliseconds per step of ``sim.advance()`` (device time on its stream)."""
    import torch

    stream = sim.g.stream
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        sim.advance()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / steps


def tune(sim, steps: int = 3, sweeps: int = 50, use_cache: bool = True, path: str | None = None,
         log=None) -> dict:
    """Picks the fastest launch shape for ``sim`` (an object with ``g`` — a
    tds.Scene or tds.Batch — and ``advance()`` taking one step of its
    motion), applies it and returns {"shape", "ms", "source", "key"}.
    Candidates are timed at ``sweeps`` fixed sweeps per step, so that every
    timed step does the same solver work; the solver settings are restored
    afterwards."""
    import torch

    g = sim.g
    cfg = g.launch_config()
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    key = shape_key(props.name, g.n, len(g.sizes))
    if use_cache:
        hit = load_cache(path).get(key)
        if hit and all(k in hit.get("shape", {}) for k in KEYS):
            shape = hit["shape"]
            if shape["colour_blocks"] <= cfg["max_colour_blocks"]:
                try:
                    g.set_launch_config(**shape)  # the library checks the solver CTAs against the shape
                    return {"shape": shape, "ms": hit.get("ms"), "source": "cache", "key": key, "sweeps": sweeps,
                            "steps": 0}
                except Exception:
                    g.set_launch_config(**{k: cfg[k] for k in KEYS})
    saved = g.solver
    g.set_solver(sweeps, 0.0, 10)
    results = []

    def timed(shapes):
        for shape in shapes:
            g.set_launch_config(**shape)
            sim.advance()  # first step of a shape (graph capture, if any) is not timed
            ms = time_steps(sim, steps)
            results.append((ms, shape))
            if log:
                log(f"autotune: {shape} {ms:.3f} ms/step")
        return min(results, key=lambda r: r[0])[1]

    sms = props.multi_processor_count
    try:
        best = timed(candidates(cfg, sms))
        best = timed(block_candidates(cfg, best)) if block_candidates(cfg, best) else best
        timed(colour_candidates(cfg, best, sms))
    finally:
        g.set_solver(*saved)
    ms, best = min(results, key=lambda r: r[0])
    g.set_launch_config(**best)
    entry = {"shape": best, "ms": ms, "default_ms": results[0][0], "tried": len(results), "sweeps": sweeps}
    if use_cache:
        store_cache(key, entry, path)
    return {"shape": best, "ms": ms, "source": "timed", "key": key, "default_ms": results[0][0],
            "sweeps": sweeps, "steps": len(results) * (1 + steps)}
