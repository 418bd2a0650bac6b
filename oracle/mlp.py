"""Per-leaf warm-start network in float64 (test infrastructure, see ``oracle``).

Not in the paper: a small network predicts each leaf's initial u from its
own Eq. 1 samples and its neighbourhood, replacing the median initialisation
where the leaf is observed.  Definitions, restated here so both
implementations follow one text:

Features (39 per leaf, leaf l with W sorted samples f_1 <= ... <= f_W):
  x_j     = f_(r_j), r_j = ceil((2j - 1) W / 64), j = 1..32 (nearest-rank
            quantiles at levels (j - 1/2)/32; 0 when W = 0)
  x_33    = level / D_max
  x_34+f  = for face f in (+x, +y, +z, -x, -y, -z): the mean of the face
            neighbours' u weighted by the share of the face each covers
            (alpha = min(1, (h_m / h_l)^2)); the leaf's own u on the boundary.

Network (parameters packed in this order, float32 on the device):
  W1 [64 x 39], b1 [64], W2 [64 x 64], b2 [64], w3 [64], b3 [1]   (6785 values)
  h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), y = tanh(w3 . h2 + b3)
  (relu'(a) = 1 for a > 0, else 0)

Loss over a batch with targets t and weights w (leaf volumes):
  L = sum_i w_i (y_i - t_i)^2 / sum_i w_i

Adam (Kingma & Ba 2015) with beta1 = 0.9, beta2 = 0.999, eps = 1e-8 and
bias correction at step k (1-based).
"""
from __future__ import annotations

import numpy as np

from . import morton

D_IN, HID = 39, 64
SIZES = (("W1", (HID, D_IN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)),
         ("w3", (HID,)), ("b3", (1,)))
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(theta):
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = np.asarray(theta[o:o + n], np.float64).reshape(shape)
        o += n
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], np.float64).ravel() for name, _ in SIZES])


def init(seed):
    """He-style initialisation (input scaling sqrt(2 / fan_in)), zero biases."""
    rng = np.random.Generator(np.random.PCG64(seed))
    p = {"W1": rng.normal(0, np.sqrt(2.0 / D_IN), (HID, D_IN)), "b1": np.zeros(HID),
         "W2": rng.normal(0, np.sqrt(2.0 / HID), (HID, HID)), "b2": np.zeros(HID),
         "w3": rng.normal(0, np.sqrt(1.0 / HID), HID), "b3": np.zeros(1)}
    return pack(p)


def forward(theta, X):
    p = unpack(theta)
    a1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(a2, 0.0)
    y = np.tanh(h2 @ p["w3"] + p["b3"][0])
    return y, (X, a1, h1, a2, h2, y)


def loss(theta, X, t, w):
    y, _ = forward(theta, X)
    return float(np.sum(w * (y - t) ** 2) / np.sum(w))


def grad(theta, X, t, w):
    """Analytic gradient of :func:`loss` (backpropagation)."""
    p = unpack(theta)
    y, (X, a1, h1, a2, h2, y) = forward(theta, X)
    d3 = 2.0 * w * (y - t) / np.sum(w) * (1.0 - y * y)          # dL/da3
    g = {"w3": h2.T @ d3, "b3": np.array([d3.sum()])}
    d2 = np.outer(d3, p["w3"]) * (a2 > 0)                        # dL/da2
    g["W2"] = d2.T @ h1
    g["b2"] = d2.sum(axis=0)
    d1 = (d2 @ p["W2"]) * (a1 > 0)                               # dL/da1
    g["W1"] = d1.T @ X
    g["b1"] = d1.sum(axis=0)
    return pack(g)


def adam(theta, m, v, g, k, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** k)
    vh = v / (1 - b2 ** k)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def features(st, u=None):
    """[N, 39] features of the leaves of a solver.State (u defaults to st.u)."""
    u = st.u if u is None else u
    N = len(st.keys)
    X = np.zeros((N, D_IN))
    W = st.W
    j = np.arange(1, 33)
    has = W > 0
    r = ((2 * j[None, :] - 1) * W[has, None] + 63) // 64           # 1-based ranks
    X[has, :32] = np.take_along_axis(st.fs[has], r - 1, axis=1)
    X[:, 32] = st.levels.astype(np.float64) / st.dmax
    h = morton.edge(st.levels, st.dmax).astype(np.float64)
    for f in range(6):
        off, idx = st.nbrs[f]
        cnt = np.diff(off)
        own = np.repeat(np.arange(N), cnt)
        alpha = np.minimum(1.0, (h[idx] / h[own]) ** 2)
        num = np.bincount(own, alpha * u[idx], minlength=N)
        den = np.bincount(own, alpha, minlength=N)
        X[:, 33 + f] = np.where(cnt > 0, num / np.where(den > 0, den, 1.0), u)
    return X


WARM_EDGE = 0.05


def warm_start(st, theta):
    """u0 = network output where W > 0 (median elsewhere or if not finite)."""
    X = features(st)
    y, _ = forward(theta, X)
    return np.where((st.W > 0) & np.isfinite(y), y, st.u)


def dual_start(st, u, g0=WARM_EDGE):
    """p0 = lambda g / |g| where |g| >= g0 (g = grad u), else 0: the optimal
    dual of the TV term wherever the field has an edge."""
    from . import operators
    g = operators.gradient(st.K, u)
    n = np.sqrt((g * g).sum(axis=1))
    sc = np.where((n >= g0) & (n > 0), st.lam / np.where(n > 0, n, 1.0), 0.0)
    return g * sc[:, None], n
