"""Eq. 1 TSDF samples and binary weights (test infrastructure, see ``oracle``).

Sec. 3.1 defines, for frame i with range map D_i, projection pi_i and centre C_i,
    phi_i(x) = D_i(pi_i(x)) - ||x - C_i||,
    f_i(x)   = sgn(phi_i) if |phi_i| > delta else phi_i / delta,
and a binary weight w_i(x) that marks x as observed unless phi_i(x) < -eta.

Readings taken where the paper is silent:
  * frames hold z-depth; the range along the pixel's ray is D times the length
    of K^-1 (px + 0.5, py + 0.5, 1); the pixel is the one x projects into
    (nearest pixel, floor of the projected coordinates);
  * a point is unobserved (w = 0) when it lies behind the camera, projects
    outside the image, or hits a pixel whose depth is 0, negative or NaN;
  * a depth of +inf is a ray that saw no surface: phi = +inf, f = +1, w = 1.

Precision: the paper keeps its TSDF values as floats (Sec. 4.1).  Eq. 1 is
therefore evaluated in float32 -- camera parameters, point coordinates and
every intermediate are rounded to float32 -- in the exact operation order
written below, each operation rounded once (no fused multiply-add).  The pixel
a point falls into is an integer decision taken in that precision, so any
implementation that follows the same order reaches the same pixel and the
same float32 sample bit for bit.
"""
from __future__ import annotations

import numpy as np

from . import morton


def centres(keys, levels, origin, extent: float, dmax: int) -> np.ndarray:
    """World coordinates of node centres in float32:
    origin + (corner + h/2) * (extent / 2^D_max), one rounding per operation."""
    x, y, z = morton.decode(keys, dmax)
    h = morton.edge(levels, dmax)
    s = np.float32(np.float32(extent) / np.float32(1 << dmax))
    out = np.empty((len(x), 3), np.float32)
    for k, c in enumerate((x, y, z)):
        mid = (c.astype(np.float32) + np.float32(0.5) * h.astype(np.float32)).astype(np.float32)
        out[:, k] = np.float32(origin[k]) + mid * s
    return out


def samples(points: np.ndarray, depth: np.ndarray, intr: np.ndarray, pose: np.ndarray,
            delta: float, eta: float) -> np.ndarray:
    """f_i at each point for each frame (Eq. 1); NaN where w_i = 0.

    `points` are float32 world coordinates.  Returns float64 [N, F] holding
    float32 values (exactly representable)."""
    f32 = np.float32
    pts = np.asarray(points, np.float32)
    n = pts.shape[0]
    F, H, W = depth.shape
    out = np.full((n, F), np.nan)
    d32, e32 = f32(delta), f32(eta)
    for i in range(F):
        R = pose[i, :3, :3].astype(np.float32)
        C = pose[i, :3, 3].astype(np.float32)
        fx, fy, cx, cy = (f32(v) for v in intr[i])
        dx = pts[:, 0] - C[0]
        dy = pts[:, 1] - C[1]
        dz = pts[:, 2] - C[2]
        # camera coordinates R^T (x - C), summed left to right
        xc = (R[0, 0] * dx + R[1, 0] * dy) + R[2, 0] * dz
        yc = (R[0, 1] * dx + R[1, 1] * dy) + R[2, 1] * dz
        zc = (R[0, 2] * dx + R[1, 2] * dy) + R[2, 2] * dz
        front = zc > f32(0.0)
        with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
            u = fx * (xc / zc) + cx
            v = fy * (yc / zc) + cy
        inside = front & (u >= f32(0.0)) & (u < f32(W)) & (v >= f32(0.0)) & (v < f32(H))
        px = np.where(inside, np.floor(np.where(inside, u, f32(0.0))), f32(0.0)).astype(np.int64)
        py = np.where(inside, np.floor(np.where(inside, v, f32(0.0))), f32(0.0)).astype(np.int64)
        d = depth[i][py, px].astype(np.float32)
        with np.errstate(invalid="ignore"):
            valid = inside & (d > f32(0.0))
        a = ((px.astype(np.float32) + f32(0.5)) - cx) / fx
        b = ((py.astype(np.float32) + f32(0.5)) - cy) / fy
        with np.errstate(invalid="ignore", over="ignore"):
            rng = d * np.sqrt((a * a + b * b) + f32(1.0))
            dist = np.sqrt((dx * dx + dy * dy) + dz * dz)
            phi = rng - dist
            w = valid & (phi >= -e32)
            f = np.minimum(np.maximum(phi / d32, f32(-1.0)), f32(1.0))
        assert f.dtype == np.float32 and phi.dtype == np.float32
        out[w, i] = f[w].astype(np.float64)
    return out


def sorted_samples(f: np.ndarray):
    """Observed samples of each point sorted ascending (NaN padding last), and W."""
    fs = np.sort(f, axis=1)
    W = np.sum(~np.isnan(fs), axis=1).astype(np.int64)
    return fs, W


def median(fs: np.ndarray, W: np.ndarray) -> np.ndarray:
    """Median of each row's W observed samples; mean of the two middle values
    for even W, (a + b) * 0.5 in float64; -1 (unseen space is taken as solid,
    Sec. 3.1) when W = 0."""
    n = fs.shape[0]
    out = np.full(n, -1.0)
    has = W > 0
    r = np.nonzero(has)[0]
    w = W[r]
    lo = fs[r, (w - 1) // 2]
    hi = fs[r, w // 2]
    out[r] = np.where(w % 2 == 1, lo, (lo + hi) * 0.5)
    return out
