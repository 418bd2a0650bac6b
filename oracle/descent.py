"""The paper's own solver (test infrastructure, see ``oracle``): gradient
descent on the epsilon-smoothed normalised energy (Eq. 4-6).

Energy, on the same octree leaves and operators as the primal-dual path:
    E_eps(u) = sum_l h_l^3 [ c_l sum_i Gamma(u_l - f_li) + lambda Gamma(|g(l)|) ],
    Gamma(x) = sqrt(x^2 + eps^2)          (the eps-L1 approximation, Eq. 4),
    c_l = 1 / (W_l + gamma)               (point-wise normalisation, Eq. 5),
    g = K u                               (level-aware forward differences).

Its derivative with respect to u_l, divided by the leaf volume h_l^3 (the
gradient in the volume-weighted inner product the integral defines), is
Eq. 6 with the opposite sign:
    G(u)_l = c_l sum_i (u_l - f_li) / Gamma(u_l - f_li)
             - lambda div( g / Gamma(|g|) )(l),
where div is the negative adjoint of K under the volume-weighted inner
products (``operators.divergence``).  One iteration is u <- u - xi_t G(u)
with xi_t = 0.1 * 0.5^floor(t / 20) (Sec. 4: 100 iterations, initial step
0.1 halved every 20).  The paper states no value for epsilon (default 1e-3
here) and no bound on u (none is applied).  It restructures while it sweeps
the tree in every iteration; here, as on the primal-dual path, the split/join
pass runs every `restructure_every` iterations on the current u.
"""
from __future__ import annotations

import numpy as np

from . import operators, solver

XI0 = 0.1
HALVE_EVERY = 20
ITERS = 100
EPS = 1e-3


def step_size(t: int, xi0: float = XI0, halve_every: int = HALVE_EVERY) -> float:
    """xi_t of iteration t (0-based): xi0 halved every `halve_every` iterations."""
    return xi0 * 0.5 ** (t // halve_every)


def gamma_eps(x, eps):
    return np.sqrt(x * x + eps * eps)


def energy(st: solver.State, eps: float = EPS, u=None) -> float:
    """E_eps(u) of a solver.State (its u unless `u` is given)."""
    u = st.u if u is None else u
    g = operators.gradient(st.K, u)
    data = np.nansum(gamma_eps(u[:, None] - st.fs, eps), axis=1)
    per = st.c * data + st.lam * gamma_eps(np.sqrt((g * g).sum(axis=1)), eps)
    return float((st.vol * per).sum())


def gradient(st: solver.State, eps: float = EPS, u=None) -> np.ndarray:
    """G(u): dE_eps/du_l / h_l^3 for every leaf."""
    u = st.u if u is None else u
    r = u[:, None] - st.fs
    data = st.c * np.nansum(r / gamma_eps(r, eps), axis=1)
    g = operators.gradient(st.K, u)
    q = g / gamma_eps(np.sqrt((g * g).sum(axis=1)), eps)[:, None]
    return data - st.lam * operators.divergence(st.K, q, st.vol)


def descend(st: solver.State, n: int, t0: int = 0, eps: float = EPS, xi0: float = XI0,
            halve_every: int = HALVE_EVERY) -> int:
    """n iterations on a fixed structure, the first being global iteration t0;
    returns the next iteration index.  u and ubar are updated together (ubar
    only keeps the restructuring code of the primal-dual state usable)."""
    for t in range(t0, t0 + n):
        st.u = st.u - step_size(t, xi0, halve_every) * gradient(st, eps)
    st.ubar = st.u.copy()
    return t0 + n


def solve(scene, iters: int = ITERS, restructure_every: int = 10, eps: float = EPS,
          st: solver.State = None) -> solver.State:
    """Median initialisation (as on the primal-dual path), then `iters`
    descent iterations, restructuring after every `restructure_every` of
    them except after the last one."""
    st = solver.initial_state(scene) if st is None else st
    t = 0
    while t < iters:
        n = min(restructure_every, iters - t) if restructure_every > 0 else iters - t
        t = descend(st, n, t, eps)
        if restructure_every > 0 and t < iters:
            solver.restructure(st, scene)
    return st
