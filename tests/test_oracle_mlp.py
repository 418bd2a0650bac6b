"""Pins of the oracle's warm-start network (no GPU)."""
import numpy as np
import pytest

from oracle import mlp, solver
from paper_1608_07411_gb300.scenes import make_scene


def _batch(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1, 1, (n, mlp.D_IN))
    t = np.clip(rng.normal(0, 0.6, n), -0.99, 0.99)
    w = rng.choice([1.0, 8.0, 64.0], n)
    return X, t, w


def test_parameter_count_and_pack():
    assert mlp.N_PARAMS == 64 * 39 + 64 + 64 * 64 + 64 + 64 + 1 == 6785
    th = mlp.init(3)
    assert np.array_equal(mlp.pack(mlp.unpack(th)), th)


def test_gradient_matches_central_differences():
    X, t, w = _batch(40, 1)
    th = mlp.init(2)
    th[6000:6100] += 0.05          # non-zero biases take part too
    g = mlp.grad(th, X, t, w)
    rng = np.random.default_rng(0)
    idx = np.concatenate([rng.choice(mlp.N_PARAMS, 200, replace=False), [mlp.N_PARAMS - 1]])
    eps = 1e-6
    for i in idx:
        e = np.zeros_like(th)
        e[i] = eps
        fd = (mlp.loss(th + e, X, t, w) - mlp.loss(th - e, X, t, w)) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (i, fd, g[i])


def test_forward_closed_form_single_unit():
    """Only one path open: y = tanh(w3_0 * relu(W2_00 * relu(W1_0 . x + b1_0) + b2_0) + b3)."""
    p = {k: np.zeros(s) for k, s in mlp.SIZES}
    p["W1"][0, :3] = [0.5, -1.0, 2.0]
    p["b1"][0] = 0.1
    p["W2"][0, 0] = 1.5
    p["b2"][0] = -0.2
    p["w3"][0] = 0.7
    p["b3"][0] = 0.05
    x = np.zeros((2, mlp.D_IN))
    x[0, :3] = [1.0, 0.5, 0.25]      # a1 = 0.5 - 0.5 + 0.5 + 0.1 = 0.6
    x[1, :3] = [-1.0, 1.0, 0.0]      # a1 = -1.4 -> relu 0
    y, _ = mlp.forward(mlp.pack(p), x)
    np.testing.assert_allclose(y, [np.tanh(0.7 * (1.5 * 0.6 - 0.2) + 0.05), np.tanh(0.05)], rtol=1e-15)


def test_adam_first_step_is_sign_times_lr():
    """With bias correction, the first Adam step moves every parameter by
    lr * g / (|g| + eps), i.e. about lr in the gradient's direction."""
    th = np.zeros(5)
    g = np.array([0.3, -2.0, 1e-3, 0.0, 5.0])
    th1, m, v = mlp.adam(th, np.zeros(5), np.zeros(5), g, 1, 1e-2)
    np.testing.assert_allclose(th1, -1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_training_reduces_loss():
    X, _, w = _batch(400, 5)
    t = np.tanh(0.8 * X[:, 0] - 0.5 * X[:, 33])
    th = mlp.init(1)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    l0 = mlp.loss(th, X, t, w)
    for k in range(1, 301):
        th, m, v = mlp.adam(th, m, v, mlp.grad(th, X, t, w), k, 3e-3)
    assert mlp.loss(th, X, t, w) < 0.1 * l0


def test_features_definition():
    s = make_scene("sphere", 2, frames=6, width=64, height=48, max_depth=4)
    st = solver.initial_state(s)
    X = mlp.features(st)
    i = int(np.argmax(st.W))
    Wi = st.W[i]
    fs = st.fs[i, :Wi]
    # nearest-rank quantiles written out for one leaf
    for j in (1, 7, 16, 32):
        r = int(np.ceil((j - 0.5) * Wi / 32))
        assert X[i, j - 1] == fs[r - 1]
    assert X[i, 32] == st.levels[i] / s.max_depth
    # W = 0 leaves have zero quantile features
    z = st.W == 0
    assert np.all(X[z, :32] == 0)
    # boundary faces carry the leaf's own value; single neighbours their value
    off, idx = st.nbrs[0]
    cnt = np.diff(off)
    b = np.nonzero(cnt == 0)[0]
    np.testing.assert_array_equal(X[b, 33], st.u[b])
    one = np.nonzero(cnt == 1)[0]
    np.testing.assert_array_equal(X[one, 33], st.u[idx[off[one]]])


def test_warm_start_fallbacks():
    """The network's output where W > 0 and finite; the median otherwise."""
    s = make_scene("sphere", 2, frames=6, width=64, height=48, max_depth=4)
    st = solver.initial_state(s)
    st.W[::7] = 0                     # some leaves seen by no frame
    st.fs[::7] = np.nan
    th = mlp.init(5)
    y, _ = mlp.forward(th, mlp.features(st))
    u = mlp.warm_start(st, th)
    seen = st.W > 0
    assert seen.any() and (~seen).any()
    np.testing.assert_array_equal(u[seen], y[seen])
    np.testing.assert_array_equal(u[~seen], st.u[~seen])
    bad = th.copy()
    bad[:] = np.nan
    np.testing.assert_array_equal(mlp.warm_start(st, bad), st.u)


def test_dual_start_closed_form_on_a_ramp():
    """u = a x on a fully refined grid: grad u = (a, 0, 0) inside and 0 on the
    far x boundary, so p = lambda (sign a, 0, 0) where |a| >= g0, 0 where the
    ramp is flatter than g0 or on the boundary layer."""
    s = make_scene("sphere", 2, frames=2, width=16, height=12, max_depth=3, spread_tau=-1.0)
    st = solver.initial_state(s)
    from oracle import morton
    x, _, _ = morton.decode(st.keys, s.max_depth)
    n = 1 << s.max_depth
    for a, g0 in ((0.2, 0.05), (-0.2, 0.05), (0.01, 0.05)):
        p, g = mlp.dual_start(st, a * x.astype(np.float64), g0)
        inner = x < n - 1
        np.testing.assert_allclose(g[inner], abs(a), rtol=1e-14)
        np.testing.assert_array_equal(g[~inner], 0.0)
        want = st.lam * np.sign(a) if abs(a) >= g0 else 0.0
        np.testing.assert_allclose(p[inner, 0], want, rtol=1e-14)
        np.testing.assert_array_equal(p[:, 1:], 0.0)
        np.testing.assert_array_equal(p[~inner], 0.0)
