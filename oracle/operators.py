"""Level-aware gradient, divergence and diagonal step sizes (test infrastructure).

The paper takes forward differences for the gradient of u* and backward
differences for the divergence, fetched from the neighbouring nodes of each
node (Sec. 3.2, "Optimization on the Octree"; Fig. 5), without a formula for
neighbours of another size.  Reading used here (equal to the textbook
forward/backward differences when all leaves have one size):

  g_d(l) = sum over m touching the +d face of l of
           alpha_lm * (u_m - u_l) / Delta_lm,
  alpha_lm = min(1, (h_m / h_l)^2)   (share of l's face that m covers),
  Delta_lm = (h_l + h_m) / 2         (centre distance along d),

an empty list (domain boundary) giving g_d(l) = 0.  The integral of Eq. 3-5
weights every leaf by its volume h^3, so the divergence is the negative
adjoint of the gradient under the h^3-weighted inner products:
div = -W_u^-1 K^T W_p.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import morton


def volumes(levels, dmax) -> np.ndarray:
    return morton.edge(levels, dmax).astype(np.float64) ** 3


def gradient_matrix(levels, dmax, nbrs) -> sp.csr_matrix:
    """K as a sparse [3N, N] matrix, row d*N + l holding g_d(l).
    `nbrs` is the output of ``octree.neighbours``; only the +x, +y, +z lists
    (the first three) enter."""
    N = len(levels)
    h = morton.edge(levels, dmax).astype(np.float64)
    rows, cols, vals = [], [], []
    for d in range(3):
        off, idx = nbrs[d]
        own = np.repeat(np.arange(N), np.diff(off))
        hl, hm = h[own], h[idx]
        coef = np.minimum(1.0, (hm / hl) ** 2) / ((hl + hm) / 2.0)
        rows += [d * N + own, d * N + own]
        cols += [idx, own]
        vals += [coef, -coef]
    K = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(3 * N, N))
    K.sum_duplicates()
    return K


def divergence(K, p: np.ndarray, vol: np.ndarray) -> np.ndarray:
    """div p = -(K* p), K* the adjoint under volume-weighted inner products.
    p: [N, 3] (column d is the d component)."""
    wp = (p * vol[:, None]).T.reshape(-1)          # row order d*N + l
    return -(K.T @ wp) / vol


def gradient(K, u: np.ndarray) -> np.ndarray:
    """g = K u as [N, 3]."""
    N = len(u)
    return (K @ u).reshape(3, N).T


def step_sizes(K, vol: np.ndarray):
    """Diagonal preconditioning (Pock & Chambolle 2011, alpha = 1) of the
    primal-dual iteration.  With the volume weights absorbed into the
    variables the operator is K~ = W_p^1/2 K W_u^-1/2; then
      sigma_(n,d) = 1 / sum_j |K~_(n,d),j|,   tau_j = 1 / sum_(n,d) |K~_(n,d),j|.
    One sigma per leaf (the smallest of its non-empty rows) keeps the
    projection onto |p_n| <= lambda exact; a leaf with three empty rows gets
    sigma = 0.  A column with no entry (a leaf with no neighbour at all) gets
    tau = 1, any positive value being equivalent there.
    Returns (tau [N], sigma [N])."""
    N = K.shape[1]
    sq = np.sqrt(vol)
    Kt = sp.diags(np.tile(sq, 3)) @ abs(K) @ sp.diags(1.0 / sq)
    row = np.asarray(Kt.sum(axis=1)).ravel().reshape(3, N)
    col = np.asarray(Kt.sum(axis=0)).ravel()
    with np.errstate(divide="ignore"):
        srow = np.where(row > 0, 1.0 / np.where(row > 0, row, 1.0), np.inf)
    sigma = srow.min(axis=0)
    sigma[~np.isfinite(sigma)] = 0.0
    tau = np.where(col > 0, 1.0 / np.where(col > 0, col, 1.0), 1.0)
    return tau, sigma
