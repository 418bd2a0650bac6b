"""Independent dense-grid TV-L1 solver (test infrastructure, see ``oracle``).

The fully refined octree is a dense voxel grid, the setting of the dense
method the paper compares against (Sec. 4).  This module solves the same
normalised energy on an [n, n, n] array with array slicing only: forward
differences with a zero difference on the far boundary, their negative
adjoint (backward differences) as divergence, and the same diagonal step sizes
written out for a grid.  The data-term prox is found by trying every candidate
minimiser (each sample and each piece's stationary point) instead of the median
formula.  It shares nothing with ``operators``/``solver`` beyond NumPy.
"""
from __future__ import annotations

import numpy as np


def grad(u):
    g = np.zeros(u.shape + (3,))
    g[:-1, :, :, 0] = u[1:] - u[:-1]
    g[:, :-1, :, 1] = u[:, 1:] - u[:, :-1]
    g[:, :, :-1, 2] = u[:, :, 1:] - u[:, :, :-1]
    return g


def div(p):
    d = np.zeros(p.shape[:3])
    for ax in range(3):
        q = np.moveaxis(p[..., ax], ax, 0)
        r = np.zeros_like(q)
        r[:-1] += q[:-1]
        r[1:] -= q[:-1]
        d += np.moveaxis(r, 0, ax)
    return d


def steps(n):
    i = np.arange(n)
    fwd = (i < n - 1).astype(float)      # has a +d neighbour
    bwd = (i >= 1).astype(float)         # has a -d neighbour
    cnt = np.zeros((n, n, n))
    anyrow = np.zeros((n, n, n), bool)
    for ax in range(3):
        shape = [1, 1, 1]
        shape[ax] = n
        cnt = cnt + (fwd + bwd).reshape(shape)
        anyrow |= np.broadcast_to(fwd.reshape(shape) > 0, (n, n, n))
    tau = np.where(cnt > 0, 1.0 / np.maximum(cnt, 1), 1.0)
    sigma = np.where(anyrow, 0.5, 0.0)
    return tau, sigma


def prox(v, t, c, fs, W):
    """Brute force: evaluate the objective at every candidate, keep the best."""
    F = fs.shape[-1]
    out = np.empty(v.shape)
    flat_v, flat_t, flat_c = v.ravel(), t.ravel(), c.ravel()
    flat_f, flat_W = fs.reshape(-1, F), W.ravel()
    for i in range(flat_v.size):
        f = flat_f[i, :flat_W[i]]
        w = flat_W[i]
        cand = list(f) + [flat_v[i] + flat_t[i] * flat_c[i] * (w - 2 * k) for k in range(w + 1)]
        cand = np.clip(np.array(cand), -1.0, 1.0)
        obj = (cand - flat_v[i]) ** 2 / (2 * flat_t[i]) + flat_c[i] * np.abs(
            cand[:, None] - f[None, :]).sum(axis=1)
        out.flat[i] = cand[np.argmin(obj)]
    return out


def solve(fs, W, u0, lam, gamma, iters):
    """fs: [n, n, n, F] sorted samples (NaN padded), W: [n, n, n]."""
    n = u0.shape[0]
    tau, sigma = steps(n)
    c = 1.0 / (W + gamma)
    u = u0.copy()
    ubar = u.copy()
    p = np.zeros(u.shape + (3,))
    for _ in range(iters):
        q = p + sigma[..., None] * grad(ubar)
        nrm = np.sqrt((q * q).sum(-1))
        p = q / np.maximum(1.0, nrm / lam)[..., None]
        un = prox(u + tau * div(p), tau, c, fs, W)
        ubar = 2 * un - u
        u = un
    return u, p
