#!/usr/bin/env python
"""Benchmark: octree TV-L1 fusion of the torus/box workload on GB300.

One step = the whole hot path on one scan: Eq. 1/2 construction and leaf
integration from device-resident frames (ofu_integrate_frames), then the
workload's primal-dual iterations with split/join every 10 iterations and a
final float64 energy (ofu_solve).  The metric is leaf-iterations per second
(sum over iterations of the leaf count, divided by the step time).

Prints one JSON line.  Under torchrun every rank fuses its own seeded scan
(independent problems: weak scaling, no collective on the data path); the
step time is the maximum over ranks and the value sums all ranks' work.

--impl reference times the FP64 CPU oracle on the host cores instead (rank 0
only), on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "leaf-iterations/s"
WORKLOAD_TEXT = {
    "torus_box": "torus R=0.3 r=0.08 united with an axis-aligned 0.3^3 box, 32 depth maps 640x480 "
                 "(seeded Fibonacci sphere of cameras at 1.2 m, fx=fy=600), noise 2 mm + 1% outliers, "
                 "D_max=8 (256^3), 500 primal-dual iterations, split/join every 10",
    "sphere": "sphere r=0.4, 8 depth maps 160x120 on a ring at 1.5 m, noise 1 mm, D_max=6, "
              "200 iterations, split/join every 10",
    "at_scale": "5 seeded spheres/tori/boxes in a 2 m scene, 100 depth maps 640x480, D_max=9",
}
# world point whose level-2 octree node is the oracle's bounded sample
CROP_POINT = {"torus_box": (0.3, 0.0, 0.0), "sphere": (0.4, 0.0, 0.0), "at_scale": (0.0, 0.0, 0.0)}


def args_():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--workload", default="torus_box", choices=tuple(WORKLOAD_TEXT))
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--fp16", action="store_true", help="store Eq. 1 samples as float16")
    ap.add_argument("--iters", type=int, default=0, help="override the workload's iteration count")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-tte", action="store_true", help="skip the time-to-energy measurement")
    return ap.parse_args()


# ----------------------------------------------------------------------------
# oracle legs (host cores)


def oracle_crop(scene):
    """The level-2 node (1/64 of the domain, 64^3 finest voxels at D_max=8)
    around a surface point, as a scene of its own: the oracle builds that
    node's subtree with its own construction and iterates on it."""
    from oracle import solver
    sub = 2
    node = scene.extent / (1 << sub)
    pt = np.asarray(CROP_POINT[scene.name])
    idx = np.clip(np.floor((pt - scene.origin) / node), 0, (1 << sub) - 1)
    crop = dataclasses.replace(scene, origin=scene.origin + idx * node, extent=node,
                               max_depth=scene.max_depth - sub)
    st = solver.initial_state(crop)
    return crop, st


def cpu_rate(scene, seconds):
    from oracle import solver
    t0 = time.perf_counter()
    crop, st = oracle_crop(scene)
    setup = time.perf_counter() - t0
    it = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        solver.step(st, 5)
        it += 5
    dt = time.perf_counter() - t0
    return len(st.keys) * it / dt, len(st.keys), it, dt, setup


def run_reference(a, scene):
    from oracle import solver
    crop, st = oracle_crop(scene)
    per_step = 10
    for _ in range(a.warmup):
        solver.step(st, per_step)
    times = []
    for _ in range(a.steps):
        t0 = time.perf_counter()
        solver.step(st, per_step)
        times.append(time.perf_counter() - t0)
    value = len(st.keys) * per_step * a.steps / sum(times)
    sample = (f"oracle (float64 NumPy/SciPy, single thread) on the level-2 node around "
              f"{CROP_POINT[scene.name]} of the {scene.name} scan ({len(st.keys)} leaves of its own "
              f"construction), {per_step} iterations per step")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * statistics.mean(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_of(a, scene, extra={"sample": sample}),
        "cpu_baseline": {"value": value, "unit": METRIC, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_of(a, scene, extra=None):
    cfg = {"workload": f"{scene.name}: {WORKLOAD_TEXT[scene.name]}", "seed": a.seed,
           "iterations": a.iters or scene.iters, "restructure_every": scene.restructure_every,
           "samples": "float16" if a.fp16 else "float32",
           "l2": "flushed before every step (256 MiB write)",
           "parallelism": f"replicas x{a.gpus} (independent scans)"}
    if extra:
        cfg.update(extra)
    return cfg


# ----------------------------------------------------------------------------
# clocks


class Clocks:
    """Samples nvidia-smi every 200 ms while the timed region runs; rows are
    matched to the benchmarked GPU by UUID."""
    Q = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = (uuid or "").lower().replace("gpu-", "")
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=subprocess.PIPE,
                                      stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        rows = [[x.strip() for x in ln.split(",")] for ln in out.strip().splitlines()]
        rows = [r for r in rows if len(r) >= 9]
        mine = [r for r in rows if self.uuid and r[0].lower().replace("gpu-", "") == self.uuid]
        rows = mine or rows
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for f in rows:
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "matched_by_uuid": bool(mine)}


# ----------------------------------------------------------------------------


def kernel_source_sha():
    h = hashlib.sha256()
    for f in ("solve.cu", "ofu_internal.cuh"):
        with open(os.path.join(ROOT, "paper_1608_07411_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel, alg_bytes_per_launch):
    """DRAM bytes per launch from the committed ncu summary, scaled to this
    launch by algorithmic bytes; None when absent or the kernel changed."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            t = json.load(fh)
    except (OSError, ValueError):
        return None
    rec = t.get(kernel)
    if not rec or rec.get("source_sha") != kernel_source_sha():
        return None
    return rec["dram_bytes_per_launch"] * alg_bytes_per_launch / rec["alg_bytes_per_launch"]


def peak_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


def time_to_energy(a, scene, of, stream, depth_d, intr_d, pose_d):
    """Reference energy E* = primal energy of the plain float32 solve at the
    workload's iteration count; then, per form, the device time (from the
    frames, construction included) and iterations until the primal energy
    first drops to E* (1 + 1e-4), checked after every restructure window."""
    import torch
    F, H, W = scene.depth.shape
    R = scene.restructure_every
    iters = a.iters or scene.iters

    from paper_1608_07411_gb300 import warm_start
    try:
        net = of.ofu_mlp_create(stream.cuda_stream)
        of.ofu_mlp_set_params(net, warm_start.load_params())
    except (OSError, ValueError):
        net = None

    def ctx_for(fp16, warm=False):
        c = of.ofu_create_octree(of.params_for(scene, sample_fp16=fp16), stream.cuda_stream)
        of.ofu_integrate_frames(c, F, H, W, depth_d.data_ptr(), intr_d.data_ptr(), pose_d.data_ptr())
        if warm:
            of.ofu_warm_start(c, net)
        return c

    c = ctx_for(False)
    done, li, (Pr, Dr, Gr) = of.ofu_solve(c, iters, R, 0, 0.0)
    of.ofu_destroy(c)
    target = Pr * (1 + 1e-4)
    out = {"reference": f"plain float32 energy after {iters} iterations", "reference_energy": Pr,
           "reference_gap": Gr, "target": target, "check_every": R}
    forms = [("plain_f32", False, False), ("f16_samples", True, False)]
    if net is not None:
        forms += [("f32_warm_start", False, True), ("f16_warm_start", True, True)]
    for name, fp16, warm in forms:
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        c = ctx_for(fp16, warm)
        it, reached, P = 0, False, float("inf")
        while it < 4 * iters:
            _, _, (P, _, _) = of.ofu_solve(c, R, 0, R, 0.0)
            it += R
            if P <= target:
                reached = True
                break
            of.ofu_restructure(c)
        ev1.record(stream)
        ev1.synchronize()
        out[name] = {"ms": ev0.elapsed_time(ev1), "iters": it, "reached": reached, "energy": P}
        of.ofu_destroy(c)
    if net is not None:
        of.ofu_mlp_destroy(net)
    return out


def aggregate(dist, total_ms, work, device):
    """Whole-job figures of a multi-rank run: the step time is the slowest
    rank's, the work (leaf-iterations) the sum over ranks.  Without a process
    group the rank's own values are returned."""
    if dist is None:
        return float(total_ms), float(work)
    import torch
    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    w = torch.tensor([work], dtype=torch.float64, device=device)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t.item()), float(w.item())


def main():
    a = args_()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    from paper_1608_07411_gb300.scenes import make_scene

    if a.impl == "reference":
        if rank == 0:
            run_reference(a, make_scene(a.workload, a.seed))
        return

    import torch

    import __graft_entry__
    from paper_1608_07411_gb300 import octfuse as of

    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    if rank == 0:
        __graft_entry__.build()
    if dist:
        dist.barrier()
    of.load()

    scene = make_scene(a.workload, a.seed + rank)
    iters = a.iters or scene.iters
    R = scene.restructure_every
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    depth_d = torch.from_numpy(scene.depth).to(dev)
    intr_d = torch.from_numpy(scene.intr.copy()).to(dev)
    pose_d = torch.from_numpy(scene.pose.reshape(-1, 16).copy()).to(dev)
    F, H, W = scene.depth.shape
    ctx = of.ofu_create_octree(of.params_for(scene, sample_fp16=a.fp16), stream.cuda_stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    s0s = []
    cons_ev = []

    def step(timed=False):
        if timed:
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c0.record(stream)
        of.ofu_integrate_frames(ctx, F, H, W, depth_d.data_ptr(), intr_d.data_ptr(), pose_d.data_ptr())
        if timed:
            c1.record(stream)
            cons_ev.append((c0, c1))
        n0 = of.ofu_num_leaves(ctx)
        s0s.append(of.ofu_export_field(ctx, of.FIELD_SAMPLES, None, 0))
        done, li, e = of.ofu_solve(ctx, iters, R, 0, 0.0)
        return n0, li, e

    for _ in range(max(a.warmup, 0)):
        step()
    torch.cuda.synchronize()

    # ---- device-timed steps (inputs resident in HBM) ----
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        uuid = ""
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(uuid)
    of.ofu_profile(ctx, True)
    l0 = of.ofu_kernel_launches()
    times, leaf_iters, n0s, energies = [], 0, [], None
    for _ in range(a.steps):
        flush.zero_()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        n0, li, energies = step(timed=True)
        ev1.record(stream)
        ev1.synchronize()
        times.append(ev0.elapsed_time(ev1))
        leaf_iters += li
        n0s.append(n0)
    torch.cuda.synchronize()
    launches = of.ofu_kernel_launches() - l0
    ms, nl, ab = of.ofu_profile_read(ctx)
    of.ofu_profile(ctx, False)
    clk = clocks.stop()
    n_final = of.ofu_num_leaves(ctx)
    n_samples = of.ofu_export_field(ctx, of.FIELD_SAMPLES, None, 0)
    total_ms, leaf_iters_all = aggregate(dist, sum(times), leaf_iters, dev)
    value = leaf_iters_all / (total_ms / 1e3)

    # ---- end to end through the C ABI with pinned host buffers ----
    depth_h = torch.from_numpy(scene.depth).pin_memory()
    intr_h = torch.from_numpy(scene.intr.copy()).pin_memory()
    pose_h = torch.from_numpy(scene.pose.reshape(-1, 16).copy()).pin_memory()
    cap = 4 * max(n0s + [n_final])
    keys_h = torch.empty(cap, dtype=torch.int64).pin_memory()
    lev_h = torch.empty(cap, dtype=torch.uint8).pin_memory()
    u_h = torch.empty(cap, dtype=torch.float32).pin_memory()
    e2e_t, e2e_li, d2h = [], 0, 0
    if dist:
        dist.barrier()
    for _ in range(a.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        of.ofu_integrate_frames(ctx, F, H, W, depth_h.data_ptr(), intr_h.data_ptr(), pose_h.data_ptr())
        done, li, e = of.ofu_solve(ctx, iters, R, 0, 0.0)
        n = of.ofu_export_leaves(ctx, keys_h.data_ptr(), lev_h.data_ptr(), u_h.data_ptr(), cap)
        e2e_t.append(time.perf_counter() - t0)
        e2e_li += li
        d2h = n * (8 + 1 + 4) + 24
    e2e_total, e2e_li = aggregate(dist, sum(e2e_t), e2e_li, dev)
    e2e_val = e2e_li / e2e_total
    h2d = scene.depth.nbytes + scene.intr.nbytes + scene.pose.nbytes

    # ---- roofline of the dominant iteration kernel ----
    names = ("k_dual", "k_primal")
    dom = 0 if ms[0] > ms[1] else 1
    achieved = ab[dom] / (ms[dom] * 1e-3) / 1e9 if ms[dom] > 0 else 0.0
    peak, peak_kind = peak_hbm()
    alg_per_launch = ab[dom] / max(nl[dom], 1)
    traffic = measured_traffic(names[dom], alg_per_launch)
    roof = {"kernel": names[dom], "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_kind": peak_kind, "traffic": traffic,
            "alg_bytes_per_launch": alg_per_launch, "launches": int(nl[dom]),
            "avg_launch_us": 1e3 * ms[dom] / max(nl[dom], 1),
            "other": {"kernel": names[1 - dom], "achieved": (ab[1 - dom] / (ms[1 - dom] * 1e-3) / 1e9)
                      if ms[1 - dom] > 0 else 0.0, "avg_launch_us": 1e3 * ms[1 - dom] / max(nl[1 - dom], 1)},
            "iteration_share_of_step": (ms[0] + ms[1]) / sum(times)}

    # iteration kernels alone, and the construction (Eq. 1 at every finest voxel for the
    # median field, then count and fill passes over the leaves) on its own
    iterate_only = {"value": leaf_iters / ((ms[0] + ms[1]) * 1e-3) if ms[0] + ms[1] > 0 else 0.0,
                    "unit": METRIC, "kernels": list(names), "scope": "rank 0"}
    cons_ms = statistics.median(c0.elapsed_time(c1) for c0, c1 in cons_ev)
    evals = (8 ** scene.max_depth + 2 * int(statistics.median(n0s))) * F
    construction = {"ms": cons_ms, "eq1_evaluations": evals,
                    "eq1_evaluations_per_s": evals / (cons_ms * 1e-3), "finest_voxels": 8 ** scene.max_depth,
                    "frames": F, "share_of_step": cons_ms * a.steps / sum(times)}

    tte = None if a.no_tte else time_to_energy(a, scene, of, stream, depth_d, intr_d, pose_d)

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        rate, nleaf, it, dt, setup = cpu_rate(scene, a.cpu_seconds)
        cpu = {"value": rate, "unit": METRIC, "cores": 1, "kind": "oracle",
               "sample": f"float64 NumPy/SciPy oracle, single thread: {it} iterations on the {nleaf} "
                         f"leaves of the level-2 node around {CROP_POINT[scene.name]} ({dt:.1f} s timed, "
                         f"{setup:.1f} s construction untimed)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": total_ms / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f16-samples/f32" if a.fp16 else "f32",
            "data": "synthetic", "config": config_of(a, scene, extra={
                "leaves_initial": int(statistics.median(n0s)), "leaves_final": n_final,
                "samples_initial": int(statistics.median(s0s)),
                "samples_final": n_samples, "final_energy": energies}),
            "e2e": {"value": e2e_val, "unit": METRIC, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(launches),
            "roofline": roof, "clocks": clk, "cpu_baseline": cpu, "time_to_energy": tte,
            "iterate_only": iterate_only, "construction": construction,
        }
        print(json.dumps(line), flush=True)
    of.ofu_destroy(ctx)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
