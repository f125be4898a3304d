"""Training of the learned warm start on the GPU (argument marshalling and
bookkeeping only: the features, targets, forward and backward passes and Adam
run in libtds's kernels).

Training data come from plain solves (previous-step warm start, tight
residual) of seeded beds being dug by their tools; the network starts only the
contacts that have no previous-step impulses, so those are the samples kept.
"""
from __future__ import annotations

import os

import numpy as np

from . import scenes as S


def dig_samples(tds, scene: dict, steps: int, tol: float = 1e-5, max_iters: int = 2000,
                settle: int | None = None, seed: int = 0, approach: float = 0.1):
    """Settle a bed with its tool parked, then dig for ``steps`` steps solving
    each to ``tol``; returns features and targets of the new contacts."""
    g = tds.Scene(scene)
    try:
        g.set_tool_pose(S.parked_tool(scene))
        g.set_solver(30)
        g.step(scene["settle_steps"] if settle is None else settle)
        parts = g.read_particles()
        path = S.tool_path(scene, S.surface_level(parts["x"], scene["r"]), seed=seed)
        dt = scene["dt"]
        length = getattr(path, "length", None)
        t0 = approach * (length if length is not None else path.push) / path.speed
        g.set_solver(max_iters, tol, 10)
        g.set_recording(True)
        X, T = [], []
        for k in range(steps):
            g.set_tool_pose(path(t0 + k * dt))
            g.step(1)
            s = g.read_training_samples()
            new = s["features"][:, 5] == 0
            X.append(s["features"][new])
            T.append(s["targets"][new])
        return np.concatenate(X), np.concatenate(T)
    finally:
        g.close()


def collect(tds, samples: int = 2_000_000, seed: int = 0, steps: int = 480, log=None):
    """About ``samples`` new-contact samples, half from the small workload and
    half from the bulldozing workload: each bed is settled once and dug for
    ``steps`` steps (one blade cycle of the bulldozing bed), solved to 1e-5;
    further seeds until the quota is met."""
    X, T = [], []
    plan = ["small", "bulldozing"]
    quota = samples // len(plan)
    for name in plan:
        got, k = 0, 0
        while got < quota:
            scene = S.WORKLOADS[name](seed=seed + 100 * k)
            x, t = dig_samples(tds, scene, steps, seed=seed + k, max_iters=1000)
            X.append(x)
            T.append(t)
            got += len(x)
            k += 1
            if log:
                log(f"learned: {name} seed {seed + 100 * (k - 1)}: {len(x)} samples ({got}/{quota})")
    X, T = np.concatenate(X), np.concatenate(T)
    return X[:samples], T[:samples]


def standardise(X, T):
    """Per-column mean and spread of inputs and targets (spread 1 where a
    column is constant)."""
    X, T = np.asarray(X, np.float64), np.asarray(T, np.float64)
    mx, sx = X.mean(0), X.std(0)
    mt, st = T.mean(0), T.std(0)
    sx = np.where(sx > 1e-6 * np.maximum(1.0, np.abs(mx)), sx, 1.0)
    st = np.where(st > 1e-12, st, 1.0)
    return mx, sx, mt, st


def fold(params: np.ndarray, mx, sx, mt, st, tds_module) -> np.ndarray:
    """Parameters of the network on raw inputs and outputs equal to a network
    trained on standardised ones: y = mt + st * f((x - mx) / sx). The input
    affine map folds into the first layer (W1 / sx, b1 - W1 mx / sx), the
    output one into the last (st W3, st b3 + mt)."""
    p = {k: np.asarray(v, np.float64) for k, v in tds_module.unflatten_params(params).items()}
    W1 = p["W1"] / sx[None, :]
    b1 = p["b1"] - W1 @ mx
    W3 = p["W3"] * st[:, None]
    b3 = p["b3"] * st + mt
    return tds_module.flatten_params({"W1": W1, "b1": b1, "W2": p["W2"], "b2": p["b2"], "W3": W3, "b3": b3})


def train(tds, X, T, epochs: int = 30, batch: int = 8192, lr: float = 2e-3, seed: int = 0,
          log=None) -> np.ndarray:
    """Adam on minibatches of shuffled, standardised samples; returns FP32
    parameters for raw features (the standardisation folded in)."""
    mx, sx, mt, st = standardise(X, T)
    order = np.random.Generator(np.random.PCG64(seed)).permutation(len(X))
    Xn = ((np.asarray(X, np.float64)[order] - mx) / sx).astype(np.float32)
    Tn = ((np.asarray(T, np.float64)[order] - mt) / st).astype(np.float32)
    import torch

    Xd = torch.from_numpy(np.ascontiguousarray(Xn)).cuda()
    Td = torch.from_numpy(np.ascontiguousarray(Tn)).cuda()
    net = tds.Net(seed=seed)
    for e in range(epochs):
        report = log is not None and (e == 0 or e == epochs - 1)
        loss = 0.0
        for b in range(0, len(X), batch):
            l = net.train_step(Xd[b:b + batch], Td[b:b + batch], lr=lr)
            if report:
                loss += float(l) * min(batch, len(X) - b)
        if report:
            log(f"learned: epoch {e}: standardised loss {loss / len(X):.4g}")
    return fold(net.host_params(), mx, sx, mt, st, tds).astype(np.float32)


WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "warmstart_mlp.npz")


def load_weights(path: str = WEIGHTS) -> np.ndarray:
    """Trained parameters shipped with the package (written by ``main``)."""
    with np.load(path) as f:
        return np.asarray(f["params"], np.float32)


def main(argv=None) -> int:
    """Collect samples, train on the GPU and write the parameters:
    ``python -m paper_2011_00459_gb300.learned --samples 400000 --out PATH``."""
    import argparse
    import time

    from . import build, tds

    ap = argparse.ArgumentParser()
    ap.add_argument("--samples", type=int, default=400_000)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default=WEIGHTS)
    a = ap.parse_args(argv)
    build.build()
    t0 = time.time()
    X, T = collect(tds, samples=a.samples, seed=a.seed, log=print)
    params = train(tds, X, T, epochs=a.epochs, seed=a.seed, log=print)
    os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
    np.savez(a.out, params=params, samples=len(X), epochs=a.epochs, seed=a.seed,
             sources="new contacts of plain solves (residual 1e-5) of the small and bulldozing beds dug by "
                     "their blades")
    print(f"wrote {a.out}: {len(X)} samples, {time.time() - t0:.0f} s")
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
