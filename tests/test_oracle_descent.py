"""Pins of the oracle's eps-L1 gradient-descent solver (the paper's own
scheme, Eq. 4-6 and Sec. 4); no GPU."""
import numpy as np
import pytest

from oracle import dense, descent, morton, solver, tsdf
from paper_1608_07411_gb300.scenes import make_scene
from tests._helpers import random_octree

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _random_samples(N, F, seed, odd=False):
    rng = np.random.default_rng(seed)
    W = rng.integers(0, F + 1, N)
    if odd:
        W = 2 * rng.integers(0, (F + 1) // 2, N) + 1
    f = rng.uniform(-1.2, 1.2, (N, F)).clip(-1, 1)
    f[np.arange(F)[None, :] >= W[:, None]] = np.nan
    return np.sort(f, axis=1), W


def _state(dmax, seed, lam=0.6, F=5, odd=False, u=None):
    k, lv = random_octree(dmax, seed)
    N = len(k)
    fs, W = _random_samples(N, F, seed + 100, odd)
    if u is None:
        u = np.random.default_rng(seed + 200).uniform(-1, 1, N)
    st = solver.State(dmax=dmax, keys=k, levels=lv, fs=fs, W=W, u=u, ubar=u.copy(),
                      p=np.zeros((N, 3)), lam=lam, gamma=1e-3)
    st.rebuild_operators()
    return st


def test_step_schedule_of_the_paper():
    """Sec. 4: initial step 0.1, halved every 20 iterations, 100 iterations."""
    xs = [descent.step_size(t) for t in range(descent.ITERS)]
    assert descent.ITERS == 100
    for t, x in enumerate(xs):
        assert x == 0.1 / 2 ** (t // 20)
    assert xs[0] == 0.1 and xs[19] == 0.1 and xs[20] == 0.05 and xs[99] == 0.1 / 16


def test_energy_brute_force_loops():
    """E_eps written out: face contacts found box by box, samples summed one
    by one, Gamma applied to each residual and to the gradient norm."""
    dmax, eps, lam = 3, 0.03, 0.7
    st = _state(dmax, 8, lam=lam)
    N = len(st.keys)
    u, fs, W = st.u, st.fs, st.W
    x, y, z = morton.decode(st.keys, dmax)
    h = morton.edge(st.levels, dmax)
    lo = np.stack([x, y, z], 1)
    E = 0.0
    for l in range(N):
        data = sum(np.sqrt((u[l] - fs[l, i]) ** 2 + eps ** 2) for i in range(W[l])) / (W[l] + 1e-3)
        g = [0.0, 0.0, 0.0]
        for d in range(3):
            for m in range(N):
                if lo[m, d] != lo[l, d] + h[l]:
                    continue
                if all(min(lo[l, a] + h[l], lo[m, a] + h[m]) > max(lo[l, a], lo[m, a])
                       for a in range(3) if a != d):
                    g[d] += min(1.0, (h[m] / h[l]) ** 2) * (u[m] - u[l]) / ((h[l] + h[m]) / 2)
        E += h[l] ** 3 * (data + lam * np.sqrt(sum(v * v for v in g) + eps ** 2))
    assert abs(E - descent.energy(st, eps)) <= 1e-10 * abs(E)


@pytest.mark.parametrize("seed", range(3))
def test_gradient_is_the_derivative_of_the_energy(seed):
    """G(u)_l = dE_eps/du_l / h_l^3, checked by central differences."""
    eps = 0.05
    st = _state(3, seed)
    G = descent.gradient(st, eps)
    h = 1e-6
    for l in np.random.default_rng(seed).choice(len(st.u), min(25, len(st.u)), replace=False):
        up, um = st.u.copy(), st.u.copy()
        up[l] += h
        um[l] -= h
        fd = (descent.energy(st, eps, up) - descent.energy(st, eps, um)) / (2 * h) / st.vol[l]
        assert abs(fd - G[l]) <= 1e-6 * max(1.0, abs(G[l]))


def test_energy_within_eps_of_the_exact_energy():
    """0 <= Gamma(x) - |x| <= eps, so 0 <= E_eps - E <= eps sum_l h^3 (c W + lambda)."""
    for eps in (1e-1, 1e-2, 1e-4):
        st = _state(3, 4)
        gap = descent.energy(st, eps) - solver.primal_energy(st)
        bound = eps * float((st.vol * (st.c * st.W + st.lam)).sum())
        assert -1e-9 <= gap <= bound * (1 + 1e-12)


def test_fully_refined_octree_equals_dense_descent():
    """On a fully refined octree the descent is the textbook grid scheme:
    forward differences (zero across the far boundary), their negative
    adjoint as divergence, written with ``dense`` array slicing only."""
    s = make_scene("sphere", 5, frames=4, width=40, height=30, max_depth=3, spread_tau=-1.0)
    st = solver.initial_state(s)
    n = 1 << s.max_depth
    assert len(st.keys) == n ** 3
    x, y, z = morton.decode(st.keys, s.max_depth)
    F = st.fs.shape[1]
    fg = np.full((n, n, n, F), np.nan)
    fg[x, y, z] = st.fs
    Wg = np.zeros((n, n, n))
    Wg[x, y, z] = st.W
    ug = np.zeros((n, n, n))
    ug[x, y, z] = st.u
    eps, c = 1e-3, 1.0 / (Wg + s.gamma)
    for t in range(30):
        r = ug[..., None] - fg
        data = c * np.nansum(r / np.sqrt(r * r + eps * eps), axis=-1)
        g = dense.grad(ug)
        q = g / np.sqrt((g * g).sum(-1) + eps * eps)[..., None]
        ug = ug - descent.step_size(t) * (data - s.lam * dense.div(q))
    descent.descend(st, 30, 0, eps)
    np.testing.assert_allclose(st.u, ug[x, y, z], atol=1e-12)


def test_small_steps_decrease_the_energy():
    """Descent lemma on a uniform grid (unit volumes, |grad|^2 <= 12): with
    a step below 1 / L, L = max(c W) / eps + 12 lambda / eps, every step
    lowers E_eps."""
    s = make_scene("sphere", 6, frames=4, width=40, height=30, max_depth=3, spread_tau=-1.0)
    st = solver.initial_state(s)
    eps = 0.05
    L = float((st.c * st.W).max()) / eps + 12 * st.lam / eps
    E = [descent.energy(st, eps)]
    for t in range(40):
        descent.descend(st, 1, t, eps, xi0=0.9 / L, halve_every=10 ** 9)
        E.append(descent.energy(st, eps))
    assert np.all(np.diff(E) < 0)


def test_zero_tv_weight_descends_to_the_median():
    """lambda = 0 and an odd number of samples per leaf: every leaf minimises
    sum_i Gamma(u - f_i) alone, whose minimiser tends to the median sample as
    eps -> 0; a long halving schedule reaches it."""
    st = _state(3, 11, lam=0.0, F=7, odd=True, u=None)
    # total travel sum(xi) = 20 covers any start in [-1, 1] even where the net
    # pull is c = 1 / W; the last steps are ~1e-7
    descent.descend(st, 2000, 0, eps=1e-7, halve_every=100)
    med = st.fs[np.arange(len(st.W)), (st.W - 1) // 2]
    np.testing.assert_allclose(st.u, med, atol=1e-4)


def test_sphere_zero_level_set():
    """The paper's schedule (100 iterations, split/join every 10) on the
    8-view sphere: sign changes between neighbouring finest leaves lie within
    two finest voxels of r = 0.4."""
    s = make_scene("sphere", 1)
    st = descent.solve(s, eps=1e-3)
    fine = st.levels == s.max_depth
    cen = tsdf.centres(st.keys, st.levels, s.origin, s.extent, s.max_depth)
    r = np.linalg.norm(cen, axis=1)
    off, idx = st.nbrs[0]
    own = np.repeat(np.arange(len(st.keys)), np.diff(off))
    cross = fine[own] & fine[idx] & (np.sign(st.u[own]) != np.sign(st.u[idx]))
    rc = 0.5 * (r[own[cross]] + r[idx[cross]])
    assert cross.sum() > 100
    assert np.max(np.abs(rc - 0.4)) < 2.0 * s.voxel
