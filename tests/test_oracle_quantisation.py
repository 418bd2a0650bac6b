"""Pins of the Eq. 7 quantisation error (no GPU)."""
import numpy as np

from oracle import morton, quantisation
from tests._helpers import random_octree


def _dense(dmax, seed):
    return np.random.default_rng(seed).uniform(-1, 1, 8 ** dmax)


def test_brute_force_over_voxel_coordinates():
    """The leaf mean taken box by box over x, y, z instead of a Morton range."""
    dmax = 3
    k, lv = random_octree(dmax, 2)
    u = _dense(dmax, 1)
    us = np.random.default_rng(3).uniform(-1, 1, len(k))
    n = 1 << dmax
    grid = np.zeros((n, n, n))
    vx, vy, vz = morton.decode(np.arange(8 ** dmax, dtype=np.uint64), dmax)
    grid[vx, vy, vz] = u
    x, y, z = morton.decode(k, dmax)
    h = morton.edge(lv, dmax)
    ref = sum(abs(us[i] - grid[x[i]:x[i] + h[i], y[i]:y[i] + h[i], z[i]:z[i] + h[i]].mean())
              for i in range(len(k)))
    assert abs(quantisation.error(k, lv, dmax, us, u) - ref) <= 1e-12 * ref


def test_zero_for_the_block_means_and_special_cases():
    dmax = 3
    k, lv = random_octree(dmax, 5)
    u = _dense(dmax, 6)
    m = quantisation.block_means(k, lv, dmax, u)
    assert quantisation.error(k, lv, dmax, m, u) <= 1e-12
    # fully refined: the plain sum of absolute differences
    kf = np.arange(8 ** dmax, dtype=np.uint64)
    lf = np.full(len(kf), dmax, np.uint8)
    us = _dense(dmax, 7)
    assert abs(quantisation.error(kf, lf, dmax, us, u) - np.abs(us - u).sum()) <= 1e-10
    # a single root leaf: |u* - mean u|
    r = quantisation.error(np.zeros(1, np.uint64), np.zeros(1, np.uint8), dmax, [0.25], u)
    assert abs(r - abs(0.25 - u.mean())) <= 1e-14
