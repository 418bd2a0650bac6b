"""Normalised TV-L1 energy on octree leaves and its primal-dual solver
(test infrastructure, see ``oracle``).

Energy (Eq. 5 with the exact L1 terms of Eq. 3, i.e. epsilon = 0 in Eq. 4),
each leaf weighted by its volume h^3:
    E(u) = sum_l h_l^3 [ c_l sum_i w_li |u_l - f_li| + lambda |g(l)| ],
    c_l  = 1 / (sum_i w_li + gamma),
with u restricted to the TSDF range [-1, 1].

The paper minimises the epsilon-smoothed energy by gradient descent (Eq. 6)
and names primal-dual methods as future work (Sec. 5).  This oracle solves the
exact energy with the first-order primal-dual algorithm of Chambolle & Pock
(theta = 1) with diagonal step sizes:
    p  <- proj_{|p_n| <= lambda}(p + sigma K ubar)
    u' <- prox_{tau G}(u + tau div p)
    ubar <- 2 u' - u,  u <- u'
where G is the data term plus the box constraint.  The prox of G at v is
the median of the 2W+1 numbers {f_1..f_W} and {v + tau c (W - 2k)}_{k=0..W}
(Li & Osher 2009), clamped to [-1, 1].
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import morton, octree, operators, tsdf


@dataclasses.dataclass
class State:
    dmax: int
    keys: np.ndarray         # uint64 [N]
    levels: np.ndarray       # uint8  [N]
    fs: np.ndarray           # float64 [N, F] sorted samples, NaN padded
    W: np.ndarray            # int64 [N]
    u: np.ndarray            # float64 [N]
    ubar: np.ndarray         # float64 [N]
    p: np.ndarray            # float64 [N, 3]
    lam: float
    gamma: float
    nbrs: list = None
    K: object = None
    vol: np.ndarray = None
    tau: np.ndarray = None
    sigma: np.ndarray = None

    @property
    def c(self) -> np.ndarray:
        return 1.0 / (self.W + self.gamma)

    def rebuild_operators(self):
        self.nbrs = octree.neighbours(self.keys, self.levels, self.dmax)
        self.K = operators.gradient_matrix(self.levels, self.dmax, self.nbrs)
        self.vol = operators.volumes(self.levels, self.dmax)
        self.tau, self.sigma = operators.step_sizes(self.K, self.vol)


def prox_data(v, tau, c, fs, W) -> np.ndarray:
    """argmin_t (t - v)^2 / (2 tau) + c sum_i |t - f_i| over t in [-1, 1]:
    the median of the 2W+1 values, padded so that unused slots do not move
    it (-inf for missing samples, +inf for k > W), then clamped."""
    n, F = fs.shape
    a = np.where(np.isnan(fs), -np.inf, fs)
    k = np.arange(F + 1)
    b = v[:, None] + (tau * c)[:, None] * (W[:, None] - 2 * k[None, :])
    b = np.where(k[None, :] <= W[:, None], b, np.inf)
    allv = np.sort(np.concatenate([a, b], axis=1), axis=1)
    return np.clip(allv[:, F], -1.0, 1.0)


def step(st: State, n: int = 1) -> None:
    """n primal-dual iterations on a fixed structure."""
    for _ in range(n):
        g = operators.gradient(st.K, st.ubar)
        q = st.p + st.sigma[:, None] * g
        nrm = np.sqrt((q * q).sum(axis=1))
        q = q / np.maximum(1.0, nrm / st.lam)[:, None] if st.lam > 0 else np.zeros_like(q)
        st.p = q
        v = st.u + st.tau * operators.divergence(st.K, st.p, st.vol)
        un = prox_data(v, st.tau, st.c, st.fs, st.W)
        st.ubar = 2.0 * un - st.u
        st.u = un


def data_sum(t: np.ndarray, fs: np.ndarray) -> np.ndarray:
    """sum_i |t - f_i| over observed samples, row by row."""
    return np.nansum(np.abs(t[:, None] - fs), axis=1)


def primal_energy(st: State, u=None) -> float:
    u = st.u if u is None else u
    g = operators.gradient(st.K, u)
    per = st.c * data_sum(u, st.fs) + st.lam * np.sqrt((g * g).sum(axis=1))
    return float((st.vol * per).sum())


def dual_value(st: State, p=None) -> float:
    """D(p) = sum_l h^3 min_{t in [-1,1]} [c sum_i |t - f_i| - t div p(l)];
    the minimum of a convex piecewise-linear function is attained at one of
    its breakpoints or at an end of the interval, all of which are tried."""
    p = st.p if p is None else p
    dv = operators.divergence(st.K, p, st.vol)
    N, F = st.fs.shape
    best = np.full(N, np.inf)
    cands = np.concatenate([np.clip(st.fs, -1.0, 1.0), np.full((N, 1), -1.0),
                            np.full((N, 1), 1.0)], axis=1)
    for j in range(cands.shape[1]):
        t = cands[:, j]
        ok = ~np.isnan(t)
        val = st.c * data_sum(np.where(ok, t, 0.0), st.fs) - np.where(ok, t, 0.0) * dv
        best = np.where(ok, np.minimum(best, val), best)
    return float((st.vol * best).sum())


def energies(st: State):
    P = primal_energy(st)
    D = dual_value(st)
    return P, D, P - D


# ----------------------------------------------------------------------------
# whole pipeline on a scene


def leaf_samples(keys, levels, scene, dmax):
    pts = tsdf.centres(keys, levels, scene.origin, scene.extent, dmax)
    f = tsdf.samples(pts, scene.depth, scene.intr, scene.pose, scene.delta, scene.eta)
    return tsdf.sorted_samples(f)


def initial_state(scene, keys=None, levels=None) -> State:
    """Construction (Sec. 3.1) on the median field unless a structure is
    given, Eq. 1 samples at leaf centres, u = median, p = 0, ubar = u."""
    dmax = scene.max_depth
    if keys is None:
        u0 = octree.dense_u0(scene.origin, scene.extent, dmax, scene.depth, scene.intr,
                             scene.pose, scene.delta, scene.eta)
        keys, levels = octree.construct(u0, dmax, scene.spread_tau)
    fs, W = leaf_samples(keys, levels, scene, dmax)
    u = tsdf.median(fs, W)
    st = State(dmax=dmax, keys=keys, levels=levels, fs=fs, W=W, u=u, ubar=u.copy(),
               p=np.zeros((len(keys), 3)), lam=scene.lam, gamma=scene.gamma)
    st.rebuild_operators()
    return st


def restructure(st: State, scene):
    """Split/join pass (``octree.restructure``) followed by Eq. 1 samples for
    every new leaf, new operators and ubar = u.  Returns (n_split, n_join)."""
    keys, levels, u, p, src, ns, nj = octree.restructure(
        st.keys, st.levels, st.u, st.p, st.dmax, scene.tau_split, scene.tau_join)
    F = st.fs.shape[1]
    fs = np.full((len(keys), F), np.nan)
    W = np.zeros(len(keys), np.int64)
    kept = src >= 0
    fs[kept] = st.fs[src[kept]]
    W[kept] = st.W[src[kept]]
    new = np.nonzero(~kept)[0]
    if new.size:
        fn, wn = leaf_samples(keys[new], levels[new], scene, st.dmax)
        fs[new] = fn
        W[new] = wn
    st.keys, st.levels, st.fs, st.W = keys, levels, fs, W
    st.u, st.p, st.ubar = u, p, u.copy()
    st.rebuild_operators()
    return ns, nj


def solve(scene, iters=None, restructure_every=None, st: State = None):
    """Full pipeline: iterate, restructuring after every `restructure_every`
    iterations except after the last one."""
    iters = scene.iters if iters is None else iters
    R = scene.restructure_every if restructure_every is None else restructure_every
    st = initial_state(scene) if st is None else st
    done = 0
    while done < iters:
        n = min(R, iters - done) if R > 0 else iters - done
        step(st, n)
        done += n
        if R > 0 and done < iters:
            restructure(st, scene)
    return st
