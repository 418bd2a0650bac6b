"""Seeded synthetic range data: the inputs both the CUDA path and the oracle consume.

This module only renders depth maps of analytic shapes and states the solver
parameters of each workload.  It holds none of the fusion arithmetic (no TSDF,
no operators, no solver): a depth map is what a range sensor would deliver,
D_i: Omega_2 -> R+ together with its projection pi_i (Sec. 3.1).

Conventions shared by every consumer:
  * depth:  float32 [F, H, W], z-depth in metres along the camera's optical
            axis; +inf where the ray misses every shape; 0 or NaN never
            appears in rendered maps (callers may add them to test validity).
  * intr:   float64 [F, 4] = (fx, fy, cx, cy); pixel (px, py) has its centre at
            (px + 0.5, py + 0.5).
  * pose:   float64 [F, 4, 4] camera-to-world, row-major, OpenCV axes
            (x right, y down, z forward).  Column 3 is the centre C_i.

Workloads (sizes follow the paper's scans; the paper's own datasets are not
available, so these scenes stand in for them):
  * "sphere"      sphere r=0.4 in [-0.5,0.5]^3, 8 views 160x120 on a ring at
                  distance 1.5 (fx=fy=140), N(0, 1 mm) depth noise, D_max=6.
  * "torus_box"   torus (R=0.3, r=0.08) united with an axis-aligned 0.3^3 box,
                  32 views 640x480 from a seeded Fibonacci sphere at distance
                  1.2 (fx=fy=600), N(0, 2 mm) noise plus 1 % outlier pixels
                  uniform in [0.5, 2.0] m, D_max=8.
  * "at_scale"    5 seeded spheres/tori/boxes in [-1,1]^3, 100 views 640x480
                  at distance 3.0, noise N(0, (0.0015 z^2) m), D_max=9; solved
                  to a relative primal-dual gap below 1e-5: split/join every
                  10 iterations during the first 500, then on that structure
                  with the gap checked every 50 iterations (cap 20000).
Every scene takes keyword overrides (frames, width, height, max_depth, ...)
so tests can build the same kind of scene at a size a CPU finishes quickly.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = ["Scene", "make_scene", "WORKLOADS"]


@dataclasses.dataclass
class Scene:
    name: str
    seed: int
    depth: np.ndarray          # float32 [F, H, W]
    intr: np.ndarray           # float64 [F, 4]
    pose: np.ndarray           # float64 [F, 4, 4]
    origin: np.ndarray         # float64 [3], min corner of the cubic domain
    extent: float              # edge length of the domain (m)
    max_depth: int             # D_max
    delta: float               # truncation band (m)
    eta: float                 # observation threshold (m)
    lam: float                 # TV weight lambda
    gamma: float               # normaliser offset gamma
    tau_split: float
    tau_join: float
    spread_tau: float          # construction threshold tau of Eq. 2
    iters: int                 # iteration count of the workload
    restructure_every: int
    gap_tol: float             # relative primal-dual gap stop (0 = fixed count)
    refine_iters: int = 0      # with gap_tol: split/join only during these first iterations
    gap_check_every: int = 0   # with gap_tol: iterations between gap checks once refined

    @property
    def frames(self) -> int:
        return int(self.depth.shape[0])

    @property
    def voxel(self) -> float:
        return self.extent / (1 << self.max_depth)


# ----------------------------------------------------------------------------
# cameras


def _look_at(centre: np.ndarray, target: np.ndarray) -> np.ndarray:
    fwd = target - centre
    fwd = fwd / np.linalg.norm(fwd)
    up = np.array([0.0, 1.0, 0.0])
    if abs(float(fwd @ up)) > 0.99:
        up = np.array([0.0, 0.0, 1.0])
    x = np.cross(fwd, up)
    x = x / np.linalg.norm(x)
    y = np.cross(fwd, x)
    pose = np.eye(4)
    pose[:3, 0] = x
    pose[:3, 1] = y
    pose[:3, 2] = fwd
    pose[:3, 3] = centre
    return pose


def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def _fibonacci_dirs(n: int, rot: np.ndarray) -> np.ndarray:
    k = np.arange(n) + 0.5
    phi = np.arccos(1.0 - 2.0 * k / n)
    theta = math.pi * (1.0 + math.sqrt(5.0)) * k
    d = np.stack([np.cos(theta) * np.sin(phi), np.sin(theta) * np.sin(phi), np.cos(phi)], 1)
    return d @ rot.T


# ----------------------------------------------------------------------------
# analytic shapes: each returns the ray parameter s of the first hit
# (rays are o + s*d, d with unit camera-z component, so s is z-depth) or +inf


class _Sphere:
    def __init__(self, centre, radius):
        self.c = np.asarray(centre, float)
        self.r = float(radius)

    def hit(self, o, d):
        oc = o - self.c
        a = np.einsum("ij,ij->i", d, d)
        b = 2.0 * np.einsum("ij,ij->i", d, oc)
        c = np.einsum("ij,ij->i", oc, oc) - self.r * self.r
        disc = b * b - 4 * a * c
        s = np.full(len(d), np.inf)
        ok = disc >= 0
        sq = np.sqrt(np.where(ok, disc, 0.0))
        s0 = (-b - sq) / (2 * a)
        s1 = (-b + sq) / (2 * a)
        s = np.where(ok & (s0 > 1e-9), s0, np.where(ok & (s1 > 1e-9), s1, np.inf))
        return s


class _Box:
    def __init__(self, centre, half, rot=None):
        self.c = np.asarray(centre, float)
        self.h = np.asarray(half, float)
        self.rot = np.eye(3) if rot is None else rot   # local -> world

    def hit(self, o, d):
        lo = (o - self.c) @ self.rot
        ld = d @ self.rot
        with np.errstate(divide="ignore", invalid="ignore"):
            inv = 1.0 / ld
            t1 = (-self.h - lo) * inv
            t2 = (self.h - lo) * inv
        tmin = np.nanmax(np.minimum(t1, t2), axis=1)
        tmax = np.nanmin(np.maximum(t1, t2), axis=1)
        s = np.where((tmax >= tmin) & (tmax > 1e-9), np.where(tmin > 1e-9, tmin, tmax), np.inf)
        return s


class _Torus:
    """Torus around the local y axis; hits by sphere tracing its exact SDF."""

    def __init__(self, centre, R, r, rot=None):
        self.c = np.asarray(centre, float)
        self.R = float(R)
        self.r = float(r)
        self.rot = np.eye(3) if rot is None else rot

    def _sdf(self, p):
        q = np.sqrt(p[:, 0] ** 2 + p[:, 2] ** 2) - self.R
        return np.sqrt(q * q + p[:, 1] ** 2) - self.r

    def hit(self, o, d):
        n = len(d)
        s_out = np.full(n, np.inf)
        lo = (o - self.c) @ self.rot
        ld = d @ self.rot
        bound = _Sphere(np.zeros(3), self.R + self.r + 1e-6)
        a = np.einsum("ij,ij->i", ld, ld)
        b = 2.0 * np.einsum("ij,ij->i", ld, lo)
        c = np.einsum("ij,ij->i", lo, lo) - bound.r ** 2
        disc = b * b - 4 * a * c
        cand = np.nonzero(disc >= 0)[0]
        if cand.size == 0:
            return s_out
        sq = np.sqrt(disc[cand])
        s0 = np.maximum((-b[cand] - sq) / (2 * a[cand]), 0.0)
        s1 = (-b[cand] + sq) / (2 * a[cand])
        keep = s1 > 0
        idx, s, s1 = cand[keep], s0[keep], s1[keep]
        dn = np.sqrt(a[idx])
        for _ in range(400):
            if idx.size == 0:
                break
            p = lo[idx] + s[:, None] * ld[idx]
            dist = self._sdf(p)
            hit = dist < 1e-7
            gone = s > s1
            if np.any(hit):
                s_out[idx[hit]] = s[hit]
            live = ~(hit | gone)
            idx, s, s1, dn, dist = idx[live], s[live], s1[live], dn[live], dist[live]
            s = s + dist / dn
        return s_out


def _render(shapes, pose, intr, width, height) -> np.ndarray:
    fx, fy, cx, cy = intr
    px, py = np.meshgrid(np.arange(width, dtype=float), np.arange(height, dtype=float))
    dcam = np.stack([(px.ravel() + 0.5 - cx) / fx, (py.ravel() + 0.5 - cy) / fy,
                     np.ones(width * height)], 1)
    dw = dcam @ pose[:3, :3].T
    o = np.broadcast_to(pose[:3, 3], dw.shape)
    s = np.full(width * height, np.inf)
    for sh in shapes:
        s = np.minimum(s, sh.hit(o, dw))
    return s.reshape(height, width)


# ----------------------------------------------------------------------------
# workloads


WORKLOADS = ("sphere", "torus_box", "at_scale")


def _frame_rng(seed: int, i: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, i])))


def make_scene(name: str, seed: int = 0, **over) -> Scene:
    """Render the named workload with a seed; keyword overrides shrink it."""
    if name == "sphere":
        cfg = dict(frames=8, width=160, height=120, focal=140.0, dist=1.5,
                   max_depth=6, extent=1.0, iters=200, gap_tol=0.0, refine_iters=0,
                   gap_check_every=0)
    elif name == "torus_box":
        cfg = dict(frames=32, width=640, height=480, focal=600.0, dist=1.2,
                   max_depth=8, extent=1.0, iters=500, gap_tol=0.0, refine_iters=0,
                   gap_check_every=0)
    elif name == "at_scale":
        cfg = dict(frames=100, width=640, height=480, focal=600.0, dist=3.0,
                   max_depth=9, extent=2.0, iters=20000, gap_tol=1e-5, refine_iters=500,
                   gap_check_every=50)
    else:
        raise ValueError(f"unknown workload {name!r}; choose from {WORKLOADS}")
    cfg.update(lam=0.5, gamma=1e-3, tau_split=0.95, tau_join=0.99, spread_tau=0.1,
               restructure_every=10, delta_voxels=4.0, eta_deltas=2.0)
    unknown = set(over) - set(cfg)
    if unknown:
        raise ValueError(f"unknown overrides {sorted(unknown)}")
    cfg.update(over)
    F, Wd, Hd = int(cfg["frames"]), int(cfg["width"]), int(cfg["height"])
    f = float(cfg["focal"]) * Wd / {"sphere": 160, "torus_box": 640, "at_scale": 640}[name]
    extent = float(cfg["extent"])
    origin = np.full(3, -0.5 * extent)
    srng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 1 << 20])))

    if name == "sphere":
        shapes = [_Sphere([0.0, 0.0, 0.0], 0.4)]
        ang = 2 * math.pi * np.arange(F) / F
        centres = float(cfg["dist"]) * np.stack([np.cos(ang), np.zeros(F), np.sin(ang)], 1)
    elif name == "torus_box":
        bc = srng.uniform(-0.2, 0.2, size=3)
        shapes = [_Torus([0.0, 0.0, 0.0], 0.3, 0.08), _Box(bc, [0.15, 0.15, 0.15])]
        centres = float(cfg["dist"]) * _fibonacci_dirs(F, _random_rotation(srng))
    else:
        shapes = []
        for _ in range(5):
            kind = srng.integers(0, 3)
            c = srng.uniform(-0.7, 0.7, size=3)
            rot = _random_rotation(srng)
            if kind == 0:
                shapes.append(_Sphere(c, srng.uniform(0.1, 0.35)))
            elif kind == 1:
                shapes.append(_Torus(c, srng.uniform(0.15, 0.35), srng.uniform(0.03, 0.08), rot))
            else:
                shapes.append(_Box(c, 0.5 * srng.uniform(0.1, 0.4, size=3), rot))
        centres = float(cfg["dist"]) * _fibonacci_dirs(F, _random_rotation(srng))

    depth = np.empty((F, Hd, Wd), np.float32)
    intr = np.empty((F, 4))
    pose = np.empty((F, 4, 4))
    for i in range(F):
        intr[i] = (f, f, Wd / 2.0, Hd / 2.0)
        pose[i] = _look_at(centres[i], np.zeros(3))
        z = _render(shapes, pose[i], intr[i], Wd, Hd)
        rng = _frame_rng(seed, i)
        hitm = np.isfinite(z)
        zf = np.where(hitm, z, 0.0)     # noise is drawn for every pixel, applied to hits
        if name == "sphere":
            z = np.where(hitm, z + rng.normal(0.0, 0.001, z.shape), z)
        elif name == "torus_box":
            z = np.where(hitm, z + rng.normal(0.0, 0.002, z.shape), z)
            out = rng.random(z.shape) < 0.01
            z = np.where(out, rng.uniform(0.5, 2.0, z.shape), z)
        else:
            z = np.where(hitm, zf + rng.normal(0.0, 1.0, z.shape) * 0.0015 * zf * zf, z)
        depth[i] = z.astype(np.float32)

    vox = extent / (1 << int(cfg["max_depth"]))
    delta = float(cfg["delta_voxels"]) * vox
    return Scene(name=name, seed=seed, depth=depth, intr=intr, pose=pose, origin=origin,
                 extent=extent, max_depth=int(cfg["max_depth"]), delta=delta,
                 eta=float(cfg["eta_deltas"]) * delta, lam=float(cfg["lam"]),
                 gamma=float(cfg["gamma"]), tau_split=float(cfg["tau_split"]),
                 tau_join=float(cfg["tau_join"]), spread_tau=float(cfg["spread_tau"]),
                 iters=int(cfg["iters"]), restructure_every=int(cfg["restructure_every"]),
                 gap_tol=float(cfg["gap_tol"]), refine_iters=int(cfg["refine_iters"]),
                 gap_check_every=int(cfg["gap_check_every"]))
