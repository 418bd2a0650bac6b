"""Pins of the oracle's energy, prox and primal-dual solver (no GPU)."""
import dataclasses

import numpy as np
import pytest

from oracle import dense, morton, octree, operators, solver, tsdf
from paper_1608_07411_gb300.scenes import Scene, make_scene
from tests._helpers import random_octree

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _random_samples(N, F, seed):
    rng = np.random.default_rng(seed)
    W = rng.integers(0, F + 1, N)
    f = rng.uniform(-1.2, 1.2, (N, F)).clip(-1, 1)
    f[np.arange(F)[None, :] >= W[:, None]] = np.nan
    return np.sort(f, axis=1), W


def test_prox_matches_brute_force():
    rng = np.random.default_rng(0)
    N, F = 400, 7
    fs, W = _random_samples(N, F, 1)
    v = rng.uniform(-1.5, 1.5, N)
    t = rng.uniform(0.01, 2.0, N)
    c = 1.0 / (W + 1e-3)
    got = solver.prox_data(v, t, c, fs, W)
    ref = dense.prox(v, t, c, fs, W)
    np.testing.assert_allclose(got, ref, atol=1e-14)
    # and against a fine scan of the objective
    grid = np.linspace(-1, 1, 20001)
    for i in range(0, N, 37):
        f = fs[i, :W[i]]
        obj = (grid - v[i]) ** 2 / (2 * t[i]) + c[i] * np.abs(grid[:, None] - f[None]).sum(1)
        assert abs(grid[np.argmin(obj)] - got[i]) <= 2e-4
    # W = 0: plain clamp
    z = W == 0
    np.testing.assert_array_equal(got[z], np.clip(v[z], -1, 1))


def test_zero_tv_weight_converges_to_median():
    """lambda = 0: p stays zero and the prox iteration is a proximal-point
    method for the data term alone, whose minimisers are the median interval."""
    dmax = 3
    k, lv = random_octree(dmax, 3)
    fs, W = _random_samples(len(k), 6, 4)
    st = solver.State(dmax=dmax, keys=k, levels=lv, fs=fs, W=W, u=np.zeros(len(k)),
                      ubar=np.zeros(len(k)), p=np.zeros((len(k), 3)), lam=0.0, gamma=1e-3)
    st.rebuild_operators()
    solver.step(st, 300)
    has = W > 0
    lo = fs[has, (W[has] - 1) // 2]
    hi = fs[has, W[has] // 2]
    assert np.all(st.u[has] >= lo - 1e-9) and np.all(st.u[has] <= hi + 1e-9)
    assert np.all(st.p == 0)


def _tiny_scene(**over):
    base = dict(frames=4, width=40, height=30, max_depth=3)
    base.update(over)
    return make_scene("sphere", 5, **base)


def test_fully_refined_octree_equals_dense_solver():
    s = _tiny_scene(spread_tau=-1.0)
    st = solver.initial_state(s)
    n = 1 << s.max_depth
    assert len(st.keys) == n ** 3
    x, y, z = morton.decode(st.keys, s.max_depth)
    F = st.fs.shape[1]
    fg = np.full((n, n, n, F), np.nan)
    fg[x, y, z] = st.fs
    Wg = np.zeros((n, n, n), np.int64)
    Wg[x, y, z] = st.W
    ug = np.zeros((n, n, n))
    ug[x, y, z] = st.u
    ud, pd = dense.solve(fg, Wg, ug, s.lam, s.gamma, 25)
    solver.step(st, 25)
    np.testing.assert_allclose(st.u, ud[x, y, z], atol=1e-12)
    np.testing.assert_allclose(st.p, pd[x, y, z], atol=1e-12)


def test_energy_brute_force_loops():
    """Energy evaluated with explicit loops: face contacts found box by box,
    the sum over samples written out."""
    dmax = 3
    k, lv = random_octree(dmax, 8)
    N = len(k)
    fs, W = _random_samples(N, 5, 9)
    rng = np.random.default_rng(2)
    u = rng.uniform(-1, 1, N)
    st = solver.State(dmax=dmax, keys=k, levels=lv, fs=fs, W=W, u=u, ubar=u, p=np.zeros((N, 3)),
                      lam=0.7, gamma=1e-3)
    st.rebuild_operators()
    x, y, z = morton.decode(k, dmax)
    h = morton.edge(lv, dmax)
    lo = np.stack([x, y, z], 1)
    E = 0.0
    for l in range(N):
        data = sum(abs(u[l] - fs[l, i]) for i in range(W[l])) / (W[l] + 1e-3)
        g = [0.0, 0.0, 0.0]
        for d in range(3):
            for m in range(N):
                if lo[m, d] != lo[l, d] + h[l]:
                    continue
                if all(min(lo[l, a] + h[l], lo[m, a] + h[m]) > max(lo[l, a], lo[m, a])
                       for a in range(3) if a != d):
                    alpha = min(1.0, (h[m] / h[l]) ** 2)
                    g[d] += alpha * (u[m] - u[l]) / ((h[l] + h[m]) / 2)
        E += h[l] ** 3 * (data + 0.7 * np.sqrt(sum(v * v for v in g)))
    assert abs(E - solver.primal_energy(st)) <= 1e-10 * abs(E)


@pytest.mark.parametrize("seed", range(3))
def test_weak_duality(seed):
    dmax = 3
    k, lv = random_octree(dmax, seed)
    N = len(k)
    fs, W = _random_samples(N, 5, seed)
    rng = np.random.default_rng(seed)
    st = solver.State(dmax=dmax, keys=k, levels=lv, fs=fs, W=W, u=rng.uniform(-1, 1, N),
                      ubar=np.zeros(N), p=np.zeros((N, 3)), lam=0.5, gamma=1e-3)
    st.rebuild_operators()
    for _ in range(20):
        u = rng.uniform(-1, 1, N)
        p = rng.normal(size=(N, 3))
        p *= (0.5 * rng.random(N) / np.linalg.norm(p, axis=1))[:, None]
        assert solver.primal_energy(st, u) >= solver.dual_value(st, p) - 1e-12


def test_gap_shrinks_on_fixed_structure():
    s = make_scene("sphere", 2, max_depth=5, width=80, height=60)
    st = solver.initial_state(s)
    gaps = []
    done = 0
    for target in (10, 20, 40, 80, 160):
        solver.step(st, target - done)
        done = target
        P, D, G = solver.energies(st)
        assert G >= -1e-9 * abs(P)
        gaps.append(G)
    assert all(b <= a for a, b in zip(gaps, gaps[1:])), gaps
    assert gaps[-1] < 0.05 * gaps[0] and gaps[-1] < 1e-3 * P


def test_single_noiseless_frame_small_tv_returns_data():
    """One noiseless view, lambda = 0.05: since lambda times the largest
    divergence coefficient stays below c = 1/(1+gamma), the observed TSDF
    itself is the minimiser on leaves seen once."""
    n, f_ = 64, 60.0
    pose = np.eye(4)
    pose[:3, 3] = (0.0, 0.0, -1.5)
    # a tilted plane z = 0.1 x + 0.05 y, rendered as z-depth along pixel rays
    px, py = np.meshgrid(np.arange(n) + 0.5, np.arange(n) + 0.5)
    a, b = (px - n / 2) / f_, (py - n / 2) / f_
    s_hit = 1.5 / (1.0 - 0.1 * a - 0.05 * b)
    depth = s_hit.astype(np.float32)[None]
    dmax = 4
    vox = 1.0 / (1 << dmax)
    sc = Scene(name="plane", seed=0, depth=depth, intr=np.array([[f_, f_, n / 2, n / 2]]),
               pose=pose[None], origin=np.full(3, -0.5), extent=1.0, max_depth=dmax,
               delta=4 * vox, eta=8 * vox, lam=0.05, gamma=1e-3, tau_split=0.95,
               tau_join=0.99, spread_tau=0.1, iters=0, restructure_every=0, gap_tol=0.0)
    st = solver.initial_state(sc)
    f1 = st.fs[:, 0]
    st.u = np.zeros(len(st.u))          # start away from the data
    st.ubar = st.u.copy()
    solver.step(st, 400)
    seen = st.W == 1
    assert seen.sum() > 100
    assert np.max(np.abs(st.u[seen] - f1[seen])) < 1e-4


@pytest.mark.slow
def test_sphere_zero_level_set():
    """The tiny sphere workload converges to a zero level set within one
    finest voxel of r = 0.4."""
    s = make_scene("sphere", 1)
    st = solver.solve(s)
    x, y, z = morton.decode(st.keys, s.max_depth)
    fine = st.levels == s.max_depth
    cen = tsdf.centres(st.keys, st.levels, s.origin, s.extent, s.max_depth)
    r = np.linalg.norm(cen, axis=1)
    # sign changes across +x faces between finest leaves
    off, idx = st.nbrs[0]
    own = np.repeat(np.arange(len(st.keys)), np.diff(off))
    cross = fine[own] & fine[idx] & (np.sign(st.u[own]) != np.sign(st.u[idx]))
    rc = 0.5 * (r[own[cross]] + r[idx[cross]])
    assert cross.sum() > 100
    assert np.max(np.abs(rc - 0.4)) < 1.0 * s.voxel + 0.5 * s.voxel
