"""Training of the per-leaf warm-start network (not in the paper).

The network (``include/octfuse.h``, "learned warm start") maps a leaf's
sorted Eq. 1 samples, level and neighbour means to an initial u.  Training
data come from the plain solver itself: for each seeded scan the octree is
built (``ofu_integrate_frames``), the features of every observed leaf are
taken from the median initialisation (``ofu_features``), and the target is
the field the solver reaches after ``target_iters`` primal-dual iterations on
that same structure (``ofu_iterate``).  Every observed leaf weighs the same
in the loss.  Every arithmetic step runs in the library's kernels; PyTorch only
holds device memory.

    python -m paper_1608_07411_gb300.warm_start --scenes 24 --out params.npy
"""
from __future__ import annotations

import argparse
import os
import time

import numpy as np

from . import octfuse as of
from .scenes import make_scene

DEFAULT_PARAMS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "warm_start_params.npy")
TRAIN_SEED0 = 100          # training scans use seeds 100, 101, ...; evaluation uses others


def init_params(seed: int) -> np.ndarray:
    """He-style initial weights (sqrt(2 / fan_in)), zero biases, packed."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = [rng.normal(0, np.sqrt(2.0 / 39), (64, 39)), np.zeros(64),
             rng.normal(0, np.sqrt(2.0 / 64), (64, 64)), np.zeros(64),
             rng.normal(0, np.sqrt(1.0 / 64), 64), np.zeros(1)]
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


def scan_data(scene, target_iters, stream, torch):
    """(X [n][39], t [n], w [n]) on the device for the observed leaves of one scan."""
    dev = torch.device("cuda", torch.cuda.current_device())
    ctx = of.ofu_create_octree(of.params_for(scene), stream)
    try:
        depth = torch.from_numpy(scene.depth).to(dev)
        intr = torch.from_numpy(scene.intr.copy()).to(dev)
        pose = torch.from_numpy(scene.pose.reshape(-1, 16).copy()).to(dev)
        F, H, W = scene.depth.shape
        of.ofu_integrate_frames(ctx, F, H, W, depth.data_ptr(), intr.data_ptr(), pose.data_ptr())
        n = of.ofu_num_leaves(ctx)
        X = torch.empty((n, 39), dtype=torch.float32, device=dev)
        of.ofu_features(ctx, X.data_ptr(), n)
        of.ofu_iterate(ctx, target_iters)
        t = torch.empty(n, dtype=torch.float32, device=dev)
        lv = torch.empty(n, dtype=torch.uint8, device=dev)
        of.ofu_export_leaves(ctx, None, lv.data_ptr(), t.data_ptr(), n)
        Wn = torch.empty(n, dtype=torch.int32, device=dev)
        of.ofu_export_field(ctx, of.FIELD_W, Wn.data_ptr(), n)
    finally:
        of.ofu_destroy(ctx)
    keep = Wn > 0
    # every observed leaf counts once: the band of finest leaves around the
    # surface, where the energy's TV term lives, must not be outweighed by the
    # volume of a few saturated coarse leaves
    w = torch.ones(n, dtype=torch.float32, device=dev)
    return X[keep].contiguous(), t[keep].contiguous(), w[keep].contiguous()


def train(n_scenes=24, target_iters=300, steps=3000, batch=65536, lr=2e-3, seed=0,
          scene_kw=None, log=print):
    import torch
    torch.cuda.init()
    stream = torch.cuda.current_stream().cuda_stream
    Xs, ts, ws = [], [], []
    t0 = time.time()
    for k in range(n_scenes):
        sc = make_scene("torus_box", TRAIN_SEED0 + k, **(scene_kw or {}))
        X, t, w = scan_data(sc, target_iters, stream, torch)
        Xs.append(X)
        ts.append(t)
        ws.append(w)
        log(f"scan {k}: {len(t)} observed leaves ({time.time() - t0:.0f} s)")
    X = torch.cat(Xs).contiguous()
    t = torch.cat(ts).contiguous()
    w = torch.cat(ws).contiguous()
    n = len(t)
    net = of.ofu_mlp_create(stream)
    try:
        of.ofu_mlp_set_params(net, init_params(seed))
        rng = np.random.Generator(np.random.PCG64(seed + 1))
        dev = X.device
        losses = []
        for s in range(steps):
            rows = torch.from_numpy(rng.integers(0, n, batch, dtype=np.int32)).to(dev)
            want = (s % 100 == 0) or s == steps - 1
            l = of.ofu_mlp_train_step(net, X.data_ptr(), t.data_ptr(), w.data_ptr(), rows.data_ptr(),
                                      batch, lr * (0.1 if s > 0.8 * steps else 1.0), want)
            if want:
                losses.append((s, l))
                log(f"step {s}: loss {l:.5f}")
        params = np.empty(of.ofu_mlp_num_params(), np.float32)
        of.ofu_mlp_get_params(net, params)
    finally:
        of.ofu_mlp_destroy(net)
    return params, losses


def load_params(path=DEFAULT_PARAMS):
    if not os.path.exists(path):
        raise FileNotFoundError(f"no trained warm-start parameters at {path}")
    p = np.load(path).astype(np.float32)
    if p.shape != (of.ofu_mlp_num_params(),):
        raise ValueError(f"{path}: expected {of.ofu_mlp_num_params()} parameters, got {p.shape}")
    return p


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--scenes", type=int, default=24)
    ap.add_argument("--target-iters", type=int, default=300)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--batch", type=int, default=65536)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default=DEFAULT_PARAMS)
    a = ap.parse_args()
    of.load()
    params, losses = train(a.scenes, a.target_iters, a.steps, a.batch, a.lr, a.seed)
    np.save(a.out, params)
    print(f"saved {a.out}: final loss {losses[-1][1]:.5f}")


if __name__ == "__main__":
    main()
