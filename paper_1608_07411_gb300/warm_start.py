"""Training and evaluation of the per-leaf warm-start network (not in the paper).

The network (``include/octfuse.h``, "learned warm start") maps a leaf's
sorted Eq. 1 samples, level and neighbour means to an initial u.  Training
data come from the plain solver itself: for each seeded torus/box scan the
octree is built (``ofu_integrate_frames``), the features of the observed
leaves are taken from the median initialisation (``ofu_features``), and the
target is the field the plain solver converges to on that same structure: its
iterations run until the relative primal-dual gap is below ``gap_tol``
(``ofu_solve``; or a fixed ``target_iters`` when ``gap_tol`` is 0).  Every
observed leaf weighs the same in the loss; at most ``rows_per_scan`` of them
per scan, drawn with a seeded generator.  Every arithmetic step runs in the
library's kernels; PyTorch only holds device memory.  Scans are rendered by a
pool of host processes (started with spawn) while the GPU works.

Evaluation (``--evaluate``) runs held-out scans of another workload (the
5-primitive D_max 9 scene by default) and reports, per scan and form (plain
float32, float16 samples, warm start, both), the iterations and device time to
the plain solver's converged energy within 1e-4, under the workload's own
schedule (split/join every 10 iterations during the first 500, then the
structure kept).

    python -m paper_1608_07411_gb300.warm_start --scenes 200 --gap-tol 1e-5 \
        --out params.npy --evaluate 1000:1010
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


_THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def _render(args):
    name, seed = args
    return make_scene(name, seed)


def scenes(name, seeds, workers=None):
    """Rendered scans in seed order, from a spawn pool of host processes."""
    import multiprocessing as mp
    workers = workers or max(1, min(len(seeds), (os.cpu_count() or 2) - 1))
    ctx = mp.get_context("spawn")
    # one BLAS / OpenMP thread per worker (children inherit the environment at
    # spawn; many workers with a thread per core each would oversubscribe)
    saved = {k: os.environ.get(k) for k in _THREAD_VARS}
    os.environ.update({k: "1" for k in _THREAD_VARS})
    try:
        pool = ctx.Pool(workers)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    with pool:
        for sc in pool.imap(_render, [(name, s) for s in seeds]):
            yield sc


def scan_data(scene, target_iters, stream, torch, gap_tol=0.0, rows=0, seed=0):
    """(X [n][39], t [n], w [n]) on the device for the observed leaves of one
    scan (at most `rows` of them when rows > 0) and the iterations run."""
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
        if gap_tol > 0:
            done, _, _ = of.ofu_solve(ctx, target_iters, 0, 50, gap_tol)
        else:
            of.ofu_iterate(ctx, target_iters)
            done = target_iters
        t = torch.empty(n, dtype=torch.float32, device=dev)
        lv = torch.empty(n, dtype=torch.uint8, device=dev)
        of.ofu_export_leaves(ctx, None, lv.data_ptr(), t.data_ptr(), n)
        Wn = torch.empty(n, dtype=torch.int32, device=dev)
        of.ofu_export_field(ctx, of.FIELD_W, Wn.data_ptr(), n)
    finally:
        of.ofu_destroy(ctx)
    keep = torch.nonzero(Wn > 0).flatten()
    if rows and len(keep) > rows:
        pick = np.random.Generator(np.random.PCG64(seed)).choice(len(keep), rows, replace=False)
        keep = keep[torch.from_numpy(np.sort(pick)).to(dev)]
    # every observed leaf counts once: the band of finest leaves around the
    # surface, where the energy's TV term lives, must not be outweighed by the
    # volume of a few saturated coarse leaves
    w = torch.ones(len(keep), dtype=torch.float32, device=dev)
    return X[keep].contiguous(), t[keep].contiguous(), w, done


def train(n_scenes=24, target_iters=300, steps=3000, batch=65536, lr=2e-3, seed=0,
          scene_kw=None, log=print, gap_tol=0.0, rows_per_scan=0, scan_iter=None):
    import torch
    torch.cuda.init()
    stream = torch.cuda.current_stream().cuda_stream
    Xs, ts, ws = [], [], []
    t0 = time.time()
    if scan_iter is None:
        scan_iter = (make_scene("torus_box", TRAIN_SEED0 + k, **(scene_kw or {})) for k in range(n_scenes))
    for k, sc in enumerate(scan_iter):
        X, t, w, done = scan_data(sc, target_iters, stream, torch, gap_tol, rows_per_scan, seed + k)
        Xs.append(X)
        ts.append(t)
        ws.append(w)
        log(f"scan {k}: {len(t)} training leaves, target after {done} iterations ({time.time() - t0:.0f} s)")
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


def evaluate(params, scans, torch, log=print):
    """Per held-out scan: iterations and device time of each form to the plain
    float32 solver's converged energy (relative gap < 1e-5) within 1e-4."""
    stream = torch.cuda.current_stream()
    dev = torch.device("cuda", torch.cuda.current_device())
    net = of.ofu_mlp_create(stream.cuda_stream)
    of.ofu_mlp_set_params(net, params)
    rows = []
    try:
        for sc in scans:
            depth = torch.from_numpy(sc.depth).to(dev)
            intr = torch.from_numpy(sc.intr.copy()).to(dev)
            pose = torch.from_numpy(sc.pose.reshape(-1, 16).copy()).to(dev)
            F, H, W = sc.depth.shape
            R = sc.restructure_every
            refine = sc.refine_iters or sc.iters
            limit = 20000

            def start(fp16, warm):
                c = of.ofu_create_octree(of.params_for(sc, sample_fp16=fp16), stream.cuda_stream)
                of.ofu_integrate_frames(c, F, H, W, depth.data_ptr(), intr.data_ptr(), pose.data_ptr())
                if warm:
                    of.ofu_warm_start(c, net)
                return c

            def run(c, stop):
                it, e = 0, None
                while it < limit:
                    n = R if it < refine else 50
                    _, _, e = of.ofu_solve(c, n, 0, n, 0.0)
                    it += n
                    if stop(it, e):
                        return it, e, True
                    if it < refine:
                        of.ofu_restructure(c)
                return it, e, False

            c = start(False, False)
            it, e, conv = run(c, lambda it, e: it >= refine and e[2] / max(abs(e[0]), 1.0) < 1e-5)
            of.ofu_destroy(c)
            target = e[0] * (1 + 1e-4)
            row = {"seed": sc.seed, "workload": sc.name, "reference_iters": it,
                   "reference_energy": e[0], "converged": conv}
            for name, fp16, warm in (("plain_f32", False, False), ("f16_samples", True, False),
                                     ("f32_warm_start", False, True), ("f16_warm_start", True, True)):
                torch.cuda.synchronize()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                c = start(fp16, warm)
                it, e, ok = run(c, lambda it, e: e[0] <= target)
                b.record(stream)
                b.synchronize()
                row[name] = {"iters": it, "ms": a.elapsed_time(b), "reached": ok}
                of.ofu_destroy(c)
            log(f"eval seed {sc.seed}: " + ", ".join(f"{k} {row[k]['iters']} it {row[k]['ms']:.1f} ms"
                                                    for k in ("plain_f32", "f16_samples", "f32_warm_start",
                                                              "f16_warm_start")))
            rows.append(row)
    finally:
        of.ofu_mlp_destroy(net)
    return rows


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
    ap.add_argument("--target-iters", type=int, default=300,
                    help="fixed-structure iterations of the targets (the cap with --gap-tol)")
    ap.add_argument("--gap-tol", type=float, default=0.0,
                    help="converge the targets to this relative gap (0: --target-iters iterations)")
    ap.add_argument("--rows-per-scan", type=int, default=0)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--batch", type=int, default=65536)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default=DEFAULT_PARAMS)
    ap.add_argument("--evaluate", default="", help="held-out seeds a:b of --eval-workload")
    ap.add_argument("--eval-workload", default="at_scale")
    ap.add_argument("--eval-out", default="")
    a = ap.parse_args()
    import json

    import torch
    # the host pools are started before the first GPU call
    train_scans = scenes("torus_box", [TRAIN_SEED0 + k for k in range(a.scenes)])
    eval_scans = None
    if a.evaluate:
        lo, hi = (int(x) for x in a.evaluate.split(":"))
        eval_scans = scenes(a.eval_workload, list(range(lo, hi)))
    of.load()
    params = None
    if a.scenes > 0:
        params, losses = train(a.scenes, a.target_iters, a.steps, a.batch, a.lr, a.seed,
                               gap_tol=a.gap_tol, rows_per_scan=a.rows_per_scan, scan_iter=train_scans)
        np.save(a.out, params)
        print(f"saved {a.out}: final loss {losses[-1][1]:.5f}")
    if eval_scans is not None:
        rows = evaluate(params if params is not None else load_params(a.out), eval_scans, torch)
        if a.eval_out:
            with open(a.eval_out, "w") as fh:
                json.dump(rows, fh, indent=1)


if __name__ == "__main__":
    main()
