"""Pins of the oracle's gradient, divergence and step sizes (no GPU)."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import dense, morton, octree, operators
from tests._helpers import random_octree


def _ops(k, lv, dmax):
    nb = octree.neighbours(k, lv, dmax)
    K = operators.gradient_matrix(lv, dmax, nb)
    return nb, K, operators.volumes(lv, dmax)


@pytest.mark.parametrize("seed", range(4))
def test_linear_field_exact(seed):
    """u = a x_d at leaf centres: each +d difference divides a centre offset
    of exactly Delta along d, and the face shares alpha sum to one."""
    dmax = 4
    k, lv = random_octree(dmax, seed)
    nb, K, vol = _ops(k, lv, dmax)
    x, y, z = morton.decode(k, dmax)
    h = morton.edge(lv, dmax)
    cen = np.stack([x, y, z], 1) + 0.5 * h[:, None]
    for d in range(3):
        g = operators.gradient(K, 0.37 * cen[:, d])
        has = np.diff(nb[d][0]) > 0
        np.testing.assert_allclose(g[has, d], 0.37, rtol=1e-13)
        np.testing.assert_array_equal(g[~has, d], 0.0)


def test_hand_case_coarse_next_to_fine():
    """Coarse leaf (h = 2) whose +x face touches four finest leaves (h = 1):
    alpha = 1/4, Delta = 3/2, so each coefficient is 1/6; and a finest leaf
    whose +x face touches the coarse leaf has alpha = 1, Delta = 3/2."""
    dmax = 2
    keys, levels = [], []
    for i in range(8):
        c = np.array([i & 1, (i >> 1) & 1, (i >> 2) & 1]) * 2
        if i == 1:   # the octant at x = 2..4 is split
            for j in range(8):
                keys.append(morton.encode(*(c + [j & 1, (j >> 1) & 1, (j >> 2) & 1]), dmax))
                levels.append(2)
        else:
            keys.append(morton.encode(*c, dmax)); levels.append(1)
    o = np.argsort(keys)
    k, lv = np.array(keys, np.uint64)[o], np.array(levels, np.uint8)[o]
    nb, K, vol = _ops(k, lv, dmax)
    N = len(k)
    coarse = int(np.searchsorted(k, morton.encode(0, 0, 0, dmax)))
    row = K.getrow(0 * N + coarse).toarray().ravel()
    fine = [int(np.searchsorted(k, morton.encode(2, y, z, dmax))) for y in (0, 1) for z in (0, 1)]
    np.testing.assert_allclose(row[fine], 1 / 6)
    np.testing.assert_allclose(row[coarse], -4 / 6)
    assert np.count_nonzero(row) == 5
    # a finest leaf at x = 3 on the +x side looks at the boundary
    f3 = int(np.searchsorted(k, morton.encode(3, 0, 0, dmax)))
    assert K.getrow(f3).nnz == 0
    # finest leaf at (2,0,0) looking -x sees the coarse leaf; its +y neighbour
    # is the finest leaf (2,1,0)
    f2 = fine[0]
    r = K.getrow(1 * N + f2).toarray().ravel()
    j = int(np.searchsorted(k, morton.encode(2, 1, 0, dmax)))
    assert r[j] == 1.0 and r[f2] == -1.0
    # divergence: div p at the coarse leaf from p_x of the four fine leaves
    p = np.zeros((N, 3))
    p[fine, 0] = 1.0
    dv = operators.divergence(K, p, vol)
    # the coarse leaf holds p = 0 and has no -face neighbour, so div = 0;
    # each fine leaf's own +x row (neighbour at x = 3, coefficient 1) gives 1,
    # and its -x neighbour (the coarse leaf) holds p = 0
    assert dv[coarse] == 0.0
    np.testing.assert_allclose(dv[fine], 1.0)


@pytest.mark.parametrize("seed", range(3))
def test_adjointness(seed):
    dmax = 4
    k, lv = random_octree(dmax, seed)
    nb, K, vol = _ops(k, lv, dmax)
    rng = np.random.default_rng(seed)
    u = rng.normal(size=len(k))
    p = rng.normal(size=(len(k), 3))
    lhs = (vol[:, None] * operators.gradient(K, u) * p).sum()
    rhs = -(vol * u * operators.divergence(K, p, vol)).sum()
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def _grid_order(k, dmax):
    x, y, z = morton.decode(k, dmax)
    n = 1 << dmax
    return (x * n + y) * n + z


def test_fully_refined_is_textbook_grid():
    dmax = 3
    n = 1 << dmax
    k = np.arange(n ** 3, dtype=np.uint64)
    lv = np.full(n ** 3, dmax, np.uint8)
    nb, K, vol = _ops(k, lv, dmax)
    gi = _grid_order(k, dmax)
    rng = np.random.default_rng(0)
    ug = rng.normal(size=(n, n, n))
    u = ug.ravel()[gi]
    np.testing.assert_allclose(operators.gradient(K, u), dense.grad(ug).reshape(-1, 3)[gi], atol=1e-15)
    pg = rng.normal(size=(n, n, n, 3))
    np.testing.assert_allclose(operators.divergence(K, pg.reshape(-1, 3)[gi], vol),
                               dense.div(pg).ravel()[gi], atol=1e-13)
    tau, sigma = operators.step_sizes(K, vol)
    td, sd = dense.steps(n)
    np.testing.assert_allclose(tau, td.ravel()[gi])
    np.testing.assert_allclose(sigma, sd.ravel()[gi])
    interior = np.all((np.stack(morton.decode(k, dmax)) > 0) & (np.stack(morton.decode(k, dmax)) < n - 1), 0)
    assert np.allclose(tau[interior], 1 / 6) and np.allclose(sigma[interior], 1 / 2)


@pytest.mark.parametrize("seed", range(4))
def test_step_sizes_satisfy_convergence_bound(seed):
    """Pock & Chambolle: with these steps ||S^1/2 K~ T^1/2||_2 <= 1, where the
    scaled operator absorbs the volume weights and S repeats sigma_n per row."""
    dmax = 3 if seed < 2 else 4
    k, lv = random_octree(dmax, seed)
    nb, K, vol = _ops(k, lv, dmax)
    tau, sigma = operators.step_sizes(K, vol)
    sq = np.sqrt(vol)
    Kt = (sp.diags(np.tile(sq, 3)) @ K @ sp.diags(1 / sq)).toarray()
    M = np.sqrt(np.tile(sigma, 3))[:, None] * Kt * np.sqrt(tau)[None, :]
    assert np.linalg.norm(M, 2) <= 1.0 + 1e-12
    assert np.all(tau > 0) and np.all(sigma >= 0)
