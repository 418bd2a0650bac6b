"""Quantisation error between a dense field and its octree counterpart
(Eq. 7; test infrastructure, see ``oracle``).

    err(u, u*) = sum over leaves n of u* | u*(n) - (1 / |n|) integral over n of u |

with u given on the finest voxels of the same domain (a fully refined run)
and u* on the leaves.  On the finest grid the integral mean over a leaf is
the plain mean of the h^3 voxels it covers; in Morton order those voxels are
the contiguous range [key, key + h^3).
"""
from __future__ import annotations

import numpy as np

from . import morton


def block_means(keys, levels, dmax, u_fine) -> np.ndarray:
    """Mean of the finest-voxel field (Morton order, 8^dmax values) over each leaf."""
    h3 = morton.edge(levels, dmax).astype(np.int64) ** 3
    c = np.concatenate([[0.0], np.cumsum(np.asarray(u_fine, np.float64))])
    k = np.asarray(keys, np.int64)
    return (c[k + h3] - c[k]) / h3


def error(keys, levels, dmax, u_leaves, u_fine) -> float:
    """Eq. 7 for one iterate pair."""
    return float(np.abs(np.asarray(u_leaves, np.float64) - block_means(keys, levels, dmax, u_fine)).sum())
