#!/usr/bin/env python
"""Benchmark: octree TV-L1 fusion on GB300.

One step = the whole hot path on one scan: Eq. 1/2 construction and leaf
integration from device-resident frames (ofu_integrate_frames), then the
primal-dual iterations with split/join every 10 iterations until the
workload's stopping rule (ofu_solve), which for the default workload (5
seeded primitives, 100 views 640x480, D_max = 9) is a relative primal-dual gap
below 1e-5 checked in float64 every 10 iterations, with an iteration cap.  The
metric is leaf-iterations per second (sum over iterations of the leaf count,
divided by the step time).

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
import platform
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "leaf-iterations/s"
WORKLOAD_TEXT = {
    "at_scale": "5 seeded spheres/tori/boxes in a 2 m scene, 100 depth maps 640x480 (Fibonacci sphere "
                "of cameras at 3 m, fx=fy=600), noise 0.0015 z^2 m, D_max=9 (512^3), primal-dual "
                "iterations with split/join every 10 during the first 500, then on that structure until "
                "the relative gap < 1e-5 (checked every 50, cap 20000)",
    "torus_box": "torus R=0.3 r=0.08 united with an axis-aligned 0.3^3 box, 32 depth maps 640x480 "
                 "(seeded Fibonacci sphere of cameras at 1.2 m, fx=fy=600), noise 2 mm + 1% outliers, "
                 "D_max=8 (256^3), 500 primal-dual iterations, split/join every 10",
    "sphere": "sphere r=0.4, 8 depth maps 160x120 on a ring at 1.5 m, noise 1 mm, D_max=6, "
              "200 iterations, split/join every 10",
}
# the oracle's bounded sample: the octree node (level, around a world point)
# that the oracle builds and iterates on its own
CROP = {"torus_box": ((0.3, 0.0, 0.0), 2), "sphere": ((0.4, 0.0, 0.0), 2),
        "at_scale": ((0.0, 0.0, 0.0), 3)}


def args_():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--workload", default="at_scale", choices=tuple(WORKLOAD_TEXT))
    ap.add_argument("--second", default="torus_box", choices=tuple(WORKLOAD_TEXT) + ("none",),
                    help="a second workload measured the same way and reported inside the line")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--fp16", action="store_true", help="store Eq. 1 samples as float16")
    ap.add_argument("--iters", type=int, default=0, help="override the workload's iteration cap")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-tte", action="store_true", help="skip the time-to-energy measurement")
    ap.add_argument("--no-precision", action="store_true", help="skip the float16/float32 field errors")
    ap.add_argument("--no-study", action="store_true", help="skip the Eq. 7 quantisation-error study")
    ap.add_argument("--no-descent", action="store_true", help="skip the eps-L1 descent line")
    return ap.parse_args()


def stop_rule(a, scene):
    """The workload's solve: (iteration cap, restructure period, refinement
    iterations, gap check period, gap tolerance).  With a gap tolerance the
    solve splits/joins every `R` iterations during the first `refine`
    iterations, then keeps that structure and iterates until the relative
    gap is below the tolerance (checked every `check` iterations) or the cap."""
    R = scene.restructure_every
    tol = scene.gap_tol
    refine = scene.refine_iters if tol > 0 else 0
    check = scene.gap_check_every if tol > 0 else 0
    return (a.iters or scene.iters), R, refine, check, tol


def run_solve(of, ctx, rule):
    """One solve by the rule of stop_rule: (iterations, leaf-iterations, energies)."""
    cap, R, refine, check, tol = rule
    if tol <= 0:
        return of.ofu_solve(ctx, cap, R, 0, 0.0)
    d1, l1, e = of.ofu_solve(ctx, min(refine, cap), R, 0, 0.0)
    if cap <= refine:
        return d1, l1, e
    d2, l2, e = of.ofu_solve(ctx, cap - refine, 0, check, tol)
    return d1 + d2, l1 + l2, e


# ----------------------------------------------------------------------------
# oracle legs (host cores)


def oracle_crop(scene):
    """A node of the octree (CROP: level and a world point inside it) as a
    scene of its own: the oracle builds that node's subtree with its own
    construction and iterates on it."""
    from oracle import solver
    pt, sub = CROP[scene.name]
    node = scene.extent / (1 << sub)
    idx = np.clip(np.floor((np.asarray(pt) - scene.origin) / node), 0, (1 << sub) - 1)
    crop = dataclasses.replace(scene, origin=scene.origin + idx * node, extent=node,
                               max_depth=scene.max_depth - sub)
    return crop, solver.initial_state(crop)


def _oracle_worker(args):
    """Runs the oracle on a crop for `seconds` (one host process)."""
    crop, seconds = args
    from oracle import solver
    st = solver.initial_state(crop)
    it, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        solver.step(st, 5)
        it += 5
    return len(st.keys) * it, time.perf_counter() - t0


def cpu_model():
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                low = ln.lower()
                if low.startswith("model name") or low.startswith("cpu part") or low.startswith("hardware"):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def cpu_rate(scene, seconds):
    """Oracle throughput on the crop: one process, then one process per host
    core (independent copies, summed), started with spawn."""
    import multiprocessing as mp
    t0 = time.perf_counter()
    crop, st = oracle_crop(scene)
    setup = time.perf_counter() - t0
    work, dt = _oracle_worker((crop, seconds))
    one = work / dt
    cores = os.cpu_count() or 1
    allc = None
    if cores > 1:
        # one BLAS / OpenMP thread per process (children inherit the environment)
        names = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
        saved = {k: os.environ.get(k) for k in names}
        os.environ.update({k: "1" for k in names})
        try:
            pool = mp.get_context("spawn").Pool(cores)
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        with pool:
            res = pool.map(_oracle_worker, [(crop, seconds)] * cores)
        allc = sum(w / t for w, t in res)
    return {"one_core": one, "all_cores": allc, "cores": cores, "leaves": len(st.keys),
            "setup_s": setup, "seconds": seconds}


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
    pt, sub = CROP[scene.name]
    sample = (f"oracle (float64 NumPy/SciPy, single thread) on the level-{sub} node around {pt} of the "
              f"{scene.name} scan ({len(st.keys)} leaves of its own construction), {per_step} iterations "
              f"per step")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * statistics.mean(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_of(a, scene, extra={"sample": sample}),
        "cpu_baseline": {"value": value, "unit": METRIC, "cores": 1, "kind": "oracle", "sample": sample,
                         "host_cores": os.cpu_count(), "cpu_model": cpu_model()},
        "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_of(a, scene, extra=None):
    cap, R, refine, check, tol = stop_rule(a, scene)
    cfg = {"workload": f"{scene.name}: {WORKLOAD_TEXT[scene.name]}", "seed": a.seed,
           "iteration_cap": cap, "restructure_every": R, "restructure_until": refine or cap,
           "gap_check_every": check, "gap_tol": tol,
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
# roofline inputs


def kernel_source_sha():
    h = hashlib.sha256()
    for f in ("solve.cu", "stencil.cuh", "ofu_internal.cuh"):
        with open(os.path.join(ROOT, "paper_1608_07411_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel, workload, alg_bytes_per_launch):
    """DRAM bytes per launch from the committed ncu summary of this kernel on
    this workload, scaled to this launch by algorithmic bytes; None when
    absent or when the kernel source changed since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            t = json.load(fh)
    except (OSError, ValueError):
        return None
    rec = t.get(workload, {}).get(kernel)
    if not rec or rec.get("source_sha") != kernel_source_sha():
        return None
    return rec["dram_bytes_per_launch"] * alg_bytes_per_launch / rec["alg_bytes_per_launch"]


def peak_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


# ----------------------------------------------------------------------------
# GPU legs


class Gpu:
    """Device copies of one scan and the stream the library runs on."""

    def __init__(self, scene, of, torch, dev):
        self.scene, self.of, self.torch = scene, of, torch
        self.stream = torch.cuda.current_stream()
        self.depth = torch.from_numpy(scene.depth).to(dev)
        self.intr = torch.from_numpy(scene.intr.copy()).to(dev)
        self.pose = torch.from_numpy(scene.pose.reshape(-1, 16).copy()).to(dev)
        self.F, self.H, self.W = scene.depth.shape

    def ctx(self, fp16):
        return self.of.ofu_create_octree(self.of.params_for(self.scene, sample_fp16=fp16),
                                         self.stream.cuda_stream)

    def integrate(self, c):
        self.of.ofu_integrate_frames(c, self.F, self.H, self.W, self.depth.data_ptr(),
                                     self.intr.data_ptr(), self.pose.data_ptr())

    def event(self):
        e = self.torch.cuda.Event(enable_timing=True)
        e.record(self.stream)
        return e


def rel_gap(e):
    return e[2] / max(abs(e[0]), 1.0)


def measure(a, scene, of, torch, dev, flush, dist, fp16, with_e2e):
    """Timed steps of one workload; returns the figures of the JSON line."""
    g = Gpu(scene, of, torch, dev)
    rule = stop_rule(a, scene)
    tol = rule[4]
    ctx = g.ctx(fp16)
    info = []

    def step():
        c0 = g.event()
        g.integrate(ctx)
        c1 = g.event()
        n0 = of.ofu_num_leaves(ctx)
        s0 = of.ofu_export_field(ctx, of.FIELD_SAMPLES, None, 0)
        done, li, e = run_solve(of, ctx, rule)
        info.append({"n0": n0, "s0": s0, "iters": done, "li": li, "energy": e, "cons": (c0, c1)})
        return li

    for _ in range(max(a.warmup, 0)):
        step()
    torch.cuda.synchronize()
    info.clear()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = of.ofu_kernel_launches()
    times, leaf_iters = [], 0
    for _ in range(a.steps):
        flush.zero_()
        ev0 = g.event()
        leaf_iters += step()
        ev1 = g.event()
        ev1.synchronize()
        times.append(ev0.elapsed_time(ev1))
    torch.cuda.synchronize()
    launches = of.ofu_kernel_launches() - l0
    total_ms, work = aggregate(dist, sum(times), leaf_iters, dev)
    last = info[-1]
    out = {
        "value": work / (total_ms / 1e3), "ms_per_step": total_ms / a.steps, "gpu_launches": launches,
        "leaf_iterations_per_step": leaf_iters / a.steps,
        "iterations": last["iters"], "final_energy": last["energy"], "rel_gap": rel_gap(last["energy"]),
        "gap_tol": tol, "gap_reached": bool(tol > 0 and rel_gap(last["energy"]) < tol),
        "leaves_initial": int(statistics.median(i["n0"] for i in info)),
        "leaves_final": of.ofu_num_leaves(ctx),
        "samples_initial": int(statistics.median(i["s0"] for i in info)),
        "samples_final": of.ofu_export_field(ctx, of.FIELD_SAMPLES, None, 0),
    }
    cons_ms = statistics.median(c0.elapsed_time(c1) for c0, c1 in (i["cons"] for i in info))
    evals = (8 ** scene.max_depth + 2 * out["leaves_initial"]) * g.F
    out["construction"] = {"ms": cons_ms, "eq1_evaluations": evals,
                           "eq1_evaluations_per_s": evals / (cons_ms * 1e-3),
                           "share_of_step": cons_ms * a.steps / sum(times)}

    # ---- one more step with per-launch events on the two iteration kernels
    # (kept out of the timed steps above)
    flush.zero_()
    info.clear()
    of.ofu_profile(ctx, max(rule[0], 1))
    pe0 = g.event()
    li_prof = step()
    pe1 = g.event()
    ms, nl, ab = of.ofu_profile_read(ctx)
    of.ofu_profile(ctx, False)
    prof_step_ms = pe0.elapsed_time(pe1)
    timed_iters = int(nl[0])
    assert timed_iters == info[-1]["iters"], "per-launch event pool smaller than the step"
    out["profile"] = {"ms": list(ms), "launches": list(nl), "alg_bytes": list(ab),
                      "leaf_iterations": li_prof, "step_ms": prof_step_ms}
    out["iterate_only"] = {"value": li_prof / ((ms[0] + ms[1]) * 1e-3), "unit": METRIC,
                           "kernels": ["k_dual", "k_primal"],
                           "scope": "one profiled step after the timed ones (rank 0)",
                           "share_of_step": (ms[0] + ms[1]) / prof_step_ms}

    if with_e2e:
        out["e2e"] = e2e(a, g, ctx, of, torch, dist, dev, flush, out)
    of.ofu_destroy(ctx)
    return out


def e2e(a, g, ctx, of, torch, dist, dev, flush, out):
    """The same steps through the C ABI from pinned host buffers: the frames
    go in and every leaf (key, level, u) comes back inside the timed region."""
    scene = g.scene
    rule = stop_rule(a, scene)
    depth_h = torch.from_numpy(scene.depth).pin_memory()
    intr_h = torch.from_numpy(scene.intr.copy()).pin_memory()
    pose_h = torch.from_numpy(scene.pose.reshape(-1, 16).copy()).pin_memory()
    cap = 4 * max(out["leaves_initial"], out["leaves_final"])
    keys_h = torch.empty(cap, dtype=torch.int64).pin_memory()
    lev_h = torch.empty(cap, dtype=torch.uint8).pin_memory()
    u_h = torch.empty(cap, dtype=torch.float32).pin_memory()
    ts, lis, d2h = [], 0, 0
    if dist:
        dist.barrier()
    for _ in range(a.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        of.ofu_integrate_frames(ctx, g.F, g.H, g.W, depth_h.data_ptr(), intr_h.data_ptr(), pose_h.data_ptr())
        done, li, e = run_solve(of, ctx, rule)
        n = of.ofu_export_leaves(ctx, keys_h.data_ptr(), lev_h.data_ptr(), u_h.data_ptr(), cap)
        ts.append(time.perf_counter() - t0)
        lis += li
        d2h = n * (8 + 1 + 4) + 24
    total, lis = aggregate(dist, sum(ts), lis, dev)
    return {"value": lis / total, "unit": METRIC,
            "h2d_bytes_per_step": int(scene.depth.nbytes + scene.intr.nbytes + scene.pose.nbytes),
            "d2h_bytes_per_step": int(d2h)}


def time_to_energy(a, scene, of, torch, dev):
    """Reference energy E* = the plain float32 solver's primal energy at a
    relative gap below 1e-5: split/join every R iterations during the
    workload's refinement iterations (its whole iteration count when it has
    no gap rule), then on that structure, gap checked every 50 iterations
    (cap 20000 iterations).  Then, per form, the device time from the frames
    (construction included) and the iterations until the primal energy
    first drops to E* (1 + 1e-4), checked after every window of the same
    schedule."""
    g = Gpu(scene, of, torch, dev)
    cap, R, refine, check, tol = stop_rule(a, scene)
    refine = refine or cap
    check = check or 50
    limit = 20000
    from paper_1608_07411_gb300 import warm_start
    try:
        net = of.ofu_mlp_create(g.stream.cuda_stream)
        of.ofu_mlp_set_params(net, warm_start.load_params())
    except (OSError, ValueError):
        net = None

    def ctx_for(fp16, warm=False):
        c = g.ctx(fp16)
        g.integrate(c)
        if warm:
            of.ofu_warm_start(c, net)
        return c

    def windows(c, stop):
        """Runs the schedule window by window until stop(it, energies) or the cap."""
        it, e = 0, None
        while it < limit:
            n = R if it < refine else check
            _, _, e = of.ofu_solve(c, n, 0, n, 0.0)
            it += n
            if stop(it, e):
                return it, e, True
            if it < refine:
                of.ofu_restructure(c)
        return it, e, False

    traj = []

    def ref_stop(it, e):
        traj.append([it, e[0], rel_gap(e), of.ofu_num_leaves(c)])
        return it >= refine and rel_gap(e) < 1e-5

    c = ctx_for(False)
    it, e, conv = windows(c, ref_stop)
    of.ofu_destroy(c)
    target = e[0] * (1 + 1e-4)
    step = max(1, len(traj) // 30)
    out = {"reference": f"plain float32: split/join every {R} iterations for {refine}, then that structure "
                        f"until the relative gap < 1e-5 (checked every {check})",
           "reference_iters": it, "reference_energy": e[0], "reference_rel_gap": rel_gap(e),
           "converged": conv, "target": target,
           "gap_trajectory": traj[::step] + ([traj[-1]] if (len(traj) - 1) % step else [])}
    forms = [("plain_f32", False, False), ("f16_samples", True, False)]
    if net is not None:
        forms += [("f32_warm_start", False, True), ("f16_warm_start", True, True)]
    for name, fp16, warm in forms:
        torch.cuda.synchronize()
        ev0 = g.event()
        c = ctx_for(fp16, warm)
        it, e, reached = windows(c, lambda it, e: e[0] <= target)
        ev1 = g.event()
        ev1.synchronize()
        out[name] = {"ms": ev0.elapsed_time(ev1), "iters": it, "reached": reached, "energy": e[0]}
        of.ofu_destroy(c)
    if net is not None:
        of.ofu_mlp_destroy(net)
    return out


def _field_err(x, ref):
    d = np.abs(np.asarray(x, np.float64) - np.asarray(ref, np.float64))
    return {"max_abs": float(d.max()) if d.size else 0.0, "rms": float(np.sqrt((d * d).mean())) if d.size else 0.0}


def precision(a, scene, of, torch, dev, iters=100):
    """The float16-sample form against float32 and against the FP64 oracle on
    one fixed structure (no restructuring, so leaves correspond one to one):
    (1) on the oracle's bounded sample (a node of the scan, built by both
    sides bit for bit), per-field max-abs and RMS errors of u and p after
    `iters` iterations of each form against float64; (2) on the whole scan,
    float16 against float32 and the primal kernel's GB/s of each form."""
    from oracle import solver
    out = {"iterations": iters, "fixed_structure": True}
    crop, st = oracle_crop(scene)
    solver.step(st, iters)
    from oracle import tsdf
    st16 = solver.initial_state(crop)
    st16.fs = st16.fs.astype(np.float32).astype(np.float16).astype(np.float64)
    st16.u = tsdf.median(st16.fs, st16.W)   # the float16 form starts from the rounded samples' median
    st16.ubar = st16.u.copy()
    solver.step(st16, iters)
    gc = Gpu(crop, of, torch, dev)
    for name, fp16 in (("f32", False), ("f16", True)):
        c = gc.ctx(fp16)
        gc.integrate(c)
        keys = np.empty(of.ofu_num_leaves(c), np.uint64)
        of.ofu_export_leaves(c, keys, None, None, len(keys))
        assert np.array_equal(keys, st.keys), "crop structure differs from the oracle's"
        of.ofu_iterate(c, iters)
        u = np.empty(len(keys), np.float32)
        p = np.empty(3 * len(keys), np.float32)
        of.ofu_export_field(c, of.FIELD_U, u, len(u))
        of.ofu_export_field(c, of.FIELD_P, p, len(p))
        p = p.reshape(3, -1).T
        out[f"{name}_vs_fp64_oracle"] = {"u": _field_err(u, st.u), "p": _field_err(p, st.p),
                                         "leaves": len(keys)}
        if fp16:
            out["f16_vs_fp64_oracle_on_f16_rounded_samples"] = {"u": _field_err(u, st16.u),
                                                                "p": _field_err(p, st16.p)}
        of.ofu_destroy(c)
    g = Gpu(scene, of, torch, dev)
    fields = {}
    for name, fp16 in (("f32", False), ("f16", True)):
        c = g.ctx(fp16)
        g.integrate(c)
        of.ofu_profile(c, True)
        of.ofu_iterate(c, iters)
        ms, nl, ab = of.ofu_profile_read(c)
        of.ofu_profile(c, False)
        n = of.ofu_num_leaves(c)
        u = np.empty(n, np.float32)
        p = np.empty(3 * n, np.float32)
        of.ofu_export_field(c, of.FIELD_U, u, n)
        of.ofu_export_field(c, of.FIELD_P, p, 3 * n)
        fields[name] = (u, p)
        out[f"{name}_primal_kernel"] = {"GB_s": ab[1] / (ms[1] * 1e-3) / 1e9, "us": 1e3 * ms[1] / nl[1],
                                        "alg_bytes_per_launch": ab[1] / nl[1]}
        out[f"{name}_iteration_us"] = 1e3 * (ms[0] + ms[1]) / nl[0]
        of.ofu_destroy(c)
    out["f16_vs_f32_whole_scan"] = {"u": _field_err(fields["f16"][0], fields["f32"][0]),
                                    "p": _field_err(fields["f16"][1], fields["f32"][1]),
                                    "leaves": len(fields["f32"][0])}
    return out


def descent_line(a, scene, of, torch, dev, flush, iters=100):
    """The paper's own solver (Eq. 4-6, Sec. 4: eps-L1 gradient descent, step
    0.1 halved every 20, 100 iterations) on the same scan: device time of the
    iterations alone after construction, steps as the main measurement."""
    g = Gpu(scene, of, torch, dev)
    c = g.ctx(a.fp16)
    times, li = [], 0
    for k in range(max(a.warmup, 0) + a.steps):
        g.integrate(c)
        n = of.ofu_num_leaves(c)
        flush.zero_()
        e0 = g.event()
        of.ofu_descend(c, iters, 0, 1e-3, 0.1, 20)
        e1 = g.event()
        e1.synchronize()
        if k >= a.warmup:
            times.append(e0.elapsed_time(e1))
            li += n * iters
    P, _, _ = of.ofu_energy(c)
    of.ofu_destroy(c)
    return {"workload": scene.name, "value": li / (sum(times) * 1e-3), "unit": METRIC,
            "iterations": iters, "ms": statistics.median(times), "leaves": n,
            "us_per_iteration": 1e3 * statistics.median(times) / iters,
            "energy_after": P, "schedule": "eps 1e-3, xi 0.1 halved every 20 (no split/join)"}


def mesh_line(of, torch, dev, big_scene=None):
    """Marching cubes (Sec. 3.3) and the synthetic-sphere accuracy (Sec. 4):
    the sphere workload fused adaptively and fully refined (every leaf at
    D_max, no split/join), both meshed; vertex distances to the analytic
    surface r = 0.4, and from each adaptive vertex to the nearest vertex of the
    fully refined mesh (the paper compares its octree result with the dense
    one).  Then the extraction time on a large scan."""
    from scipy.spatial import cKDTree

    from paper_1608_07411_gb300.scenes import make_scene
    sc = make_scene("sphere", 0)
    g = Gpu(sc, of, torch, dev)
    out = {"workload": "sphere: r=0.4, 8 views 160x120, D_max 6, 200 iterations, split/join every 10",
           "voxel_mm": 1e3 * sc.extent / (1 << sc.max_depth)}
    meshes = {}
    for name, kw in (("adaptive", {}), ("fully_refined", dict(spread_tau=-1.0, tau_split=2.0, tau_join=2.0))):
        p = of.params_for(sc)
        for k, v in kw.items():
            setattr(p, k, v)
        c = of.ofu_create_octree(p, g.stream.cuda_stream)
        g.integrate(c)
        of.ofu_solve(c, sc.iters, 0 if kw else sc.restructure_every, 0, 0.0)
        nv, nt = of.ofu_extract_mesh(c)
        V = np.empty((nv, 3), np.float32)
        T = np.empty((nt, 3), np.int32)
        of.ofu_extract_mesh(c, V, nv, T, nt)
        meshes[name] = V.astype(np.float64)
        d = np.abs(np.linalg.norm(V.astype(np.float64), axis=1) - 0.4)
        out[name] = {"leaves": of.ofu_num_leaves(c), "vertices": nv, "triangles": nt,
                     "dist_to_sphere_mm_mean": 1e3 * float(d.mean()), "dist_to_sphere_mm_std": 1e3 * float(d.std()),
                     "dist_to_sphere_mm_max": 1e3 * float(d.max())}
        of.ofu_destroy(c)
    dd, _ = cKDTree(meshes["fully_refined"]).query(meshes["adaptive"])
    out["adaptive_to_fully_refined_mm"] = {"mean": 1e3 * float(dd.mean()), "std": 1e3 * float(dd.std())}
    if big_scene is not None:
        gb = Gpu(big_scene, of, torch, dev)
        c = gb.ctx(False)
        gb.integrate(c)
        of.ofu_extract_mesh(c)   # scratch allocated outside the timing
        e0 = gb.event()
        nv, nt = of.ofu_extract_mesh(c)
        e1 = gb.event()
        e1.synchronize()
        out["extraction"] = {"workload": big_scene.name, "finest_voxels": 8 ** big_scene.max_depth,
                             "vertices": nv, "triangles": nt, "ms_counts_only": e0.elapsed_time(e1)}
        of.ofu_destroy(c)
    return out


def frame_tree_line(scene, of, torch, dev):
    """Per-frame TSDF octrees (data_term = 1, Sec. 3.1 / Fig. 4): build time
    with the construction, Table 1's dense and octree data-term bytes, the
    device bytes this library keeps, and one solve on tree samples."""
    g = Gpu(scene, of, torch, dev)
    p = of.params_for(scene, frame_trees=True)
    c = of.ofu_create_octree(p, g.stream.cuda_stream)
    g.integrate(c)   # warm-up (allocations)
    torch.cuda.synchronize()
    e0 = g.event()
    g.integrate(c)
    e1 = g.event()
    e1.synchronize()
    F = scene.depth.shape[0]
    nodes = np.empty(F, np.int64)
    dense, octb, devb = of.ofu_data_term_memory(c, nodes)
    e2 = g.event()
    done, li, e = of.ofu_solve(c, scene.iters, scene.restructure_every, 0, 0.0)
    e3 = g.event()
    e3.synchronize()
    out = {"workload": scene.name, "frames": F, "integrate_ms_with_trees": e0.elapsed_time(e1),
           "dense_MB": dense / 2 ** 20, "octree_MB": octb / 2 ** 20, "device_MB": devb / 2 ** 20,
           "octree_over_dense": octb / dense, "nodes_per_frame_median": int(np.median(nodes)),
           "solve_iterations": done, "solve_ms": e2.elapsed_time(e3), "leaf_iterations_per_s": li / (e2.elapsed_time(e3) * 1e-3),
           "energy": e[0]}
    of.ofu_destroy(c)
    return out


def quantisation_study(scene, of, torch, dev, checkpoints=(10, 20, 50, 100, 200, 500), sweep_iters=200):
    """Eq. 7 and Sec. 4.2 (Fig. 10 / 11) on the GPU: the quantisation error
    between the adaptive solve (split/join every R iterations) and a fully
    refined run of the same scan (every leaf at D_max: construction threshold
    below 0, no split or join), at the given iteration counts; then a sweep of
    the split and join thresholds with the leaf count, primal energy and the
    error against the fully refined run after `sweep_iters` iterations."""
    g = Gpu(scene, of, torch, dev)
    R = scene.restructure_every
    D = scene.max_depth
    nf = 8 ** D

    def ctx(**kw):
        p = of.params_for(scene)
        for k, v in kw.items():
            setattr(p, k, v)
        c = of.ofu_create_octree(p, g.stream.cuda_stream)
        g.integrate(c)
        return c

    fine = torch.empty(nf, dtype=torch.float32, device=dev)
    ev0 = g.event()
    dense = ctx(spread_tau=-1.0, tau_split=2.0, tau_join=2.0)
    nd = of.ofu_num_leaves(dense)
    assert nd == nf
    adap = ctx()
    rows, done = [], 0
    for t in checkpoints:
        while done < t:
            of.ofu_iterate(dense, R)
            of.ofu_iterate(adap, R)
            done += R
            if done < t:
                of.ofu_restructure(adap)
        of.ofu_export_field(dense, of.FIELD_U, fine.data_ptr(), nf)
        err = of.ofu_quantisation_error(adap, fine.data_ptr(), nf)
        n = of.ofu_num_leaves(adap)
        Pa, _, Ga = of.ofu_energy(adap)
        Pd, _, Gd = of.ofu_energy(dense)
        rows.append({"iteration": t, "leaves": n, "eq7_error": err, "eq7_error_per_leaf": err / n,
                     "energy_adaptive": Pa, "energy_dense": Pd, "rel_gap_adaptive": Ga / max(abs(Pa), 1),
                     "rel_gap_dense": Gd / max(abs(Pd), 1)})
        if done < checkpoints[-1]:
            of.ofu_restructure(adap)
        if t == sweep_iters:
            fine_sweep = fine.clone()
            Pd_sweep = Pd
    of.ofu_destroy(adap)
    of.ofu_destroy(dense)
    sweep = []
    for ts in (0.5, 0.8, 0.9, 0.95):
        for tj in (0.95, 0.99, 1.01):
            if tj < ts:
                continue
            c = ctx(tau_split=ts, tau_join=tj)
            of.ofu_solve(c, sweep_iters, R, 0, 0.0)
            P, _, G = of.ofu_energy(c)
            err = of.ofu_quantisation_error(c, fine_sweep.data_ptr(), nf)
            n = of.ofu_num_leaves(c)
            sweep.append({"tau_split": ts, "tau_join": tj, "joins": tj <= 1.0, "leaves": n,
                          "energy": P, "energy_vs_dense": P / Pd_sweep - 1.0, "eq7_error": err,
                          "eq7_error_per_leaf": err / n})
            of.ofu_destroy(c)
    ev1 = g.event()
    ev1.synchronize()
    return {"workload": scene.name, "dense_leaves": nd, "adaptive_vs_dense": rows,
            "sweep_iterations": sweep_iters, "sweep": sweep, "ms": ev0.elapsed_time(ev1)}


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


# Least bytes of one primal-step leaf update: u, ubar, level, six face
# entries, p, tau and the sample offset (57 B), the rank hint read and written
# (4 B) and one 32-byte sector holding the two samples that bracket the prox.
PRIMAL_MIN_BYTES_PER_LEAF = 93


def roofline(res, workload):
    ms, nl, ab = res["profile"]["ms"], res["profile"]["launches"], res["profile"]["alg_bytes"]
    names = ("k_dual", "k_primal")
    dom = 0 if ms[0] > ms[1] else 1
    achieved = ab[dom] / (ms[dom] * 1e-3) / 1e9 if ms[dom] > 0 else 0.0
    peak, kind = peak_hbm()
    per = ab[dom] / max(nl[dom], 1)
    traffic = measured_traffic(names[dom], workload, per)
    o = 1 - dom
    out = {"kernel": names[dom], "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
           "frac": achieved / peak, "peak_kind": kind, "traffic": traffic, "alg_bytes_per_launch": per,
           "launches": int(nl[dom]), "avg_launch_us": 1e3 * ms[dom] / max(nl[dom], 1),
           "other": {"kernel": names[o], "achieved": ab[o] / (ms[o] * 1e-3) / 1e9 if ms[o] > 0 else 0.0,
                     "frac": (ab[o] / (ms[o] * 1e-3) / 1e9) / peak if ms[o] > 0 else 0.0,
                     "avg_launch_us": 1e3 * ms[o] / max(nl[o], 1)}}
    # The primal step's search starts at each leaf's rank of the previous
    # iteration, so a settled leaf reads one sector of samples, not all of
    # them: its rate against the least bytes it moves, beside the count above.
    li = res["profile"].get("leaf_iterations", 0)
    if ms[1] > 0 and li:
        ach = PRIMAL_MIN_BYTES_PER_LEAF * li / (ms[1] * 1e-3) / 1e9
        out["k_primal_min_bytes"] = {"bytes_per_leaf": PRIMAL_MIN_BYTES_PER_LEAF, "achieved": ach,
                                     "frac": ach / peak}
    return out


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
    dev = torch.device("cuda", torch.cuda.current_device())
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        uuid = ""
    clocks = Clocks(uuid)
    res = measure(a, scene, of, torch, dev, flush, dist, a.fp16, with_e2e=True)
    clk = clocks.stop()

    second = None
    sec_scene = None
    if a.second not in ("none", a.workload):
        sec_scene = make_scene(a.second, a.seed + rank)
        r2 = measure(a, sec_scene, of, torch, dev, flush, dist, a.fp16, with_e2e=False)
        second = {"workload": f"{sec_scene.name}: {WORKLOAD_TEXT[sec_scene.name]}", "value": r2["value"],
                  "unit": METRIC, "ms_per_step": r2["ms_per_step"], "iterations": r2["iterations"],
                  "leaves_initial": r2["leaves_initial"], "leaves_final": r2["leaves_final"],
                  "samples_initial": r2["samples_initial"], "iterate_only": r2["iterate_only"],
                  "roofline": roofline(r2, sec_scene.name), "construction": r2["construction"]}

    fp16_step = None
    if not a.fp16 and not a.no_precision and rank == 0:
        # the same protocol with float16 samples (config 4's bandwidth comparison on this scan)
        r16 = measure(a, scene, of, torch, dev, flush, None, True, with_e2e=False)
        rf16 = roofline(r16, scene.name)
        fp16_step = {"samples": "float16", "value": r16["value"], "unit": METRIC,
                     "ms_per_step": r16["ms_per_step"], "iterations": r16["iterations"],
                     "rel_gap": r16["rel_gap"], "gap_reached": r16["gap_reached"],
                     "final_energy": r16["final_energy"],
                     "primal_kernel": {"achieved_GB_s": rf16["achieved"] if rf16["kernel"] == "k_primal"
                                       else rf16["other"]["achieved"],
                                       "avg_launch_us": rf16["avg_launch_us"] if rf16["kernel"] == "k_primal"
                                       else rf16["other"]["avg_launch_us"]},
                     "iterate_only": r16["iterate_only"]["value"]}
    tte = None if a.no_tte or rank != 0 else time_to_energy(a, scene, of, torch, dev)
    desc = [descent_line(a, sc, of, torch, dev, flush) for sc in (scene, sec_scene) if sc is not None] \
        if rank == 0 and not a.no_descent else None
    prec = None
    if not a.no_precision and rank == 0:
        pscene = sec_scene if sec_scene is not None and sec_scene.name == "torus_box" else \
            make_scene("torus_box", a.seed)
        prec = precision(a, pscene, of, torch, dev)

    study = None
    if not a.no_study and rank == 0:
        sscene = sec_scene if sec_scene is not None and sec_scene.name == "torus_box" else \
            make_scene("torus_box", a.seed)
        study = quantisation_study(sscene, of, torch, dev)

    mesh = frames_ = None
    if rank == 0 and not a.no_study:
        mesh = mesh_line(of, torch, dev, scene)
        fscene = sec_scene if sec_scene is not None and sec_scene.name == "torus_box" else \
            make_scene("torus_box", a.seed)
        frames_ = frame_tree_line(fscene, of, torch, dev)

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        r = cpu_rate(scene, a.cpu_seconds)
        pt, sub = CROP[scene.name]
        val, cores = (r["all_cores"], r["cores"]) if r["all_cores"] else (r["one_core"], 1)
        cpu = {"value": val, "unit": METRIC, "cores": cores, "kind": "oracle",
               "one_core": r["one_core"], "host_cores": r["cores"], "cpu_model": cpu_model(),
               "sample": f"float64 NumPy/SciPy oracle on the {r['leaves']} leaves of the level-{sub} node "
                         f"around {pt} (its own construction, {r['setup_s']:.1f} s, untimed): "
                         f"{r['seconds']:.0f} s of iterations in one process, then the same in "
                         f"{r['cores']} independent processes at once (value = their sum)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": res["value"], "unit": METRIC, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": res["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f16-samples/f32" if a.fp16 else "f32",
            "data": "synthetic", "config": config_of(a, scene, extra={
                "leaves_initial": res["leaves_initial"], "leaves_final": res["leaves_final"],
                "samples_initial": res["samples_initial"], "samples_final": res["samples_final"]}),
            "solve": {"iterations": res["iterations"], "rel_gap": res["rel_gap"], "gap_tol": res["gap_tol"],
                      "gap_reached": res["gap_reached"], "final_energy": res["final_energy"],
                      "leaf_iterations_per_step": res["leaf_iterations_per_step"]},
            "e2e": res["e2e"], "gpu_launches": int(res["gpu_launches"]),
            "roofline": roofline(res, scene.name), "clocks": clk, "cpu_baseline": cpu,
            "iterate_only": res["iterate_only"], "construction": res["construction"],
            "time_to_energy": tte, "precision": prec, "fp16_step": fp16_step, "second_workload": second,
            "quantisation_study": study, "descent": desc, "mesh": mesh, "frame_trees": frames_,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
