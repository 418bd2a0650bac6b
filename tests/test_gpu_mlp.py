"""Warm-start network: CUDA kernels vs the FP64 oracle, and what training gains."""
import os

import numpy as np
import pytest

from oracle import mlp, solver
from paper_1608_07411_gb300 import octfuse as of
from paper_1608_07411_gb300.scenes import make_scene

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def lib():
    import __graft_entry__
    __graft_entry__.build()
    return of.load()


def dev(a, dtype=None):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


@pytest.fixture
def net():
    h = of.ofu_mlp_create(torch.cuda.current_stream().cuda_stream)
    yield h
    of.ofu_mlp_destroy(h)


def _batch(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1, 1, (n, mlp.D_IN))
    t = np.clip(rng.normal(0, 0.6, n), -0.99, 0.99)
    w = rng.choice([1.0, 8.0, 64.0], n)
    return X, t, w


def test_forward_matches_oracle(net):
    th = mlp.init(4)
    th[mlp.N_PARAMS - 200:] += 0.03
    X, _, _ = _batch(1000, 1)
    of.ofu_mlp_set_params(net, th.astype(np.float32))
    Xd = dev(X, np.float32)
    y = torch.empty(1000, device="cuda")
    of.ofu_mlp_forward(net, Xd.data_ptr(), 1000, y.data_ptr())
    torch.cuda.synchronize()
    ref, _ = mlp.forward(th.astype(np.float32).astype(np.float64), X.astype(np.float32).astype(np.float64))
    np.testing.assert_allclose(y.cpu().numpy(), ref, atol=2e-5)


@pytest.mark.parametrize("B", [1, 127, 128, 1000, 5000])
def test_gradient_matches_oracle(net, B):
    th = mlp.init(7).astype(np.float32)
    X, t, w = _batch(B, B)
    of.ofu_mlp_set_params(net, th)
    g = np.empty(mlp.N_PARAMS, np.float32)
    # keep the device tensors alive for the call (their memory is reused once freed)
    Xd, td, wd = dev(X, np.float32), dev(t, np.float32), dev(w, np.float32)
    loss = of.ofu_mlp_gradient(net, Xd.data_ptr(), td.data_ptr(), wd.data_ptr(), None, B, g)
    X64 = X.astype(np.float32).astype(np.float64)
    t64 = t.astype(np.float32).astype(np.float64)
    gr = mlp.grad(th.astype(np.float64), X64, t64, w)
    lr = mlp.loss(th.astype(np.float64), X64, t64, w)
    assert abs(loss - lr) <= 1e-5 * max(lr, 1e-3)
    scale = np.abs(gr).max()
    np.testing.assert_allclose(g, gr, atol=2e-4 * scale)


def test_gradient_with_row_selection_and_adam(net):
    th = mlp.init(9)
    X, t, w = _batch(3000, 3)
    rows = np.random.default_rng(0).integers(0, 3000, 700).astype(np.int32)
    of.ofu_mlp_set_params(net, th.astype(np.float32))
    Xd, td, wd, rd = dev(X, np.float32), dev(t, np.float32), dev(w, np.float32), dev(rows)
    X64 = X.astype(np.float32).astype(np.float64)[rows]
    t64 = t.astype(np.float32).astype(np.float64)[rows]
    ref = th.astype(np.float32).astype(np.float64)
    m = np.zeros_like(ref)
    v = np.zeros_like(ref)
    for k in range(1, 4):
        of.ofu_mlp_train_step(net, Xd.data_ptr(), td.data_ptr(), wd.data_ptr(), rd.data_ptr(), 700, 1e-3)
        ref, m, v = mlp.adam(ref, m, v, mlp.grad(ref, X64, t64, w[rows]), k, 1e-3)
    got = np.empty(mlp.N_PARAMS, np.float32)
    of.ofu_mlp_get_params(net, got)
    np.testing.assert_allclose(got, ref, atol=5e-6)


def _state(scene):
    o = of.Octree(of.params_for(scene))
    o.integrate_frames(scene.depth, scene.intr, scene.pose)
    return o, solver.initial_state(scene)


def test_features_and_warm_start_match_oracle(net):
    scene = make_scene("torus_box", 21, frames=12, width=160, height=120, max_depth=6)
    o, st = _state(scene)
    n = o.n
    X = torch.empty((n, 39), device="cuda")
    of.ofu_features(o.ctx, X.data_ptr(), n)
    torch.cuda.synchronize()
    Xo = mlp.features(st)
    Xg = X.cpu().numpy()
    np.testing.assert_array_equal(Xg[:, :32], Xo[:, :32].astype(np.float32))
    np.testing.assert_array_equal(Xg[:, 32], Xo[:, 32].astype(np.float32))
    np.testing.assert_allclose(Xg[:, 33:], Xo[:, 33:], atol=1e-6)
    th = mlp.init(11).astype(np.float32)
    of.ofu_mlp_set_params(net, th)
    of.ofu_warm_start(o.ctx, net)
    u = o.field(of.FIELD_U)
    ub = o.field(of.FIELD_UBAR)
    ref = mlp.warm_start(st, th.astype(np.float64))
    np.testing.assert_allclose(u, ref, atol=2e-5)
    np.testing.assert_array_equal(u, ub)
    np.testing.assert_array_equal(u[st.W == 0], st.u[st.W == 0].astype(np.float32))
    # dual start from the warm-started field (the threshold decision may flip
    # only where |grad u| is within float32 rounding of it)
    p = o.field(of.FIELD_P)
    pref, gn = mlp.dual_start(st, u.astype(np.float64))
    firm = np.abs(gn - mlp.WARM_EDGE) > 1e-4
    assert firm.mean() > 0.99
    np.testing.assert_allclose(p[firm], pref[firm], atol=1e-5)


def _energies(scene, params, iters, restructure_every=10):
    """Primal energy at the start and after each window of the solve."""
    o = of.Octree(of.params_for(scene))
    o.integrate_frames(scene.depth, scene.intr, scene.pose)
    net = None
    if params is not None:
        net = of.ofu_mlp_create(torch.cuda.current_stream().cuda_stream)
        of.ofu_mlp_set_params(net, params)
        of.ofu_warm_start(o.ctx, net)
    out = [o.energy()[0]]
    it = 0
    while it < iters:
        _, _, (P, _, _) = o.solve(restructure_every, 0, restructure_every, 0.0)
        out.append(P)
        it += restructure_every
        if it < iters:
            o.restructure()
    if net:
        of.ofu_mlp_destroy(net)
    o.close()
    return np.array(out)


def test_trained_warm_start_gains():
    """On a scan outside the training seeds (torus_box seed 0; training uses
    seeds 100..), the trained network starts the solve at a lower energy than
    the median initialisation and is still lower after the first window,
    while an untrained network starts far higher.  The gain in iterations
    and time to the plain solver's converged energy is measured by bench.py
    (time_to_energy) and by warm_start.evaluate on held-out scans."""
    from paper_1608_07411_gb300 import warm_start
    params = warm_start.load_params()
    scene = make_scene("torus_box", 0)
    plain = _energies(scene, None, 30)
    warm = _energies(scene, params, 30)
    raw = _energies(scene, warm_start.init_params(0), 30)
    print("energy per window: plain", plain, "warm", warm, "untrained", raw)
    assert warm[0] < plain[0] < raw[0]
    assert warm[1] < plain[1]
    # after the first split/join passes both runs reach the same energies to
    # within 1e-4 (the iterations and time to the converged energy are the
    # gain, measured on held-out scans by the evaluation protocol)
    assert np.all(warm[2:] <= plain[2:] * (1 + 1e-4))


def test_training_protocol_small():
    """The config-5 protocol end to end at a small size: targets converged to a
    relative gap of 1e-5 on the constructed structure, a few hundred Adam
    steps, then the held-out evaluation of every form against the plain
    solver's converged energy (split/join during the refinement iterations,
    then the structure kept)."""
    from paper_1608_07411_gb300 import warm_start
    scans = [make_scene("torus_box", warm_start.TRAIN_SEED0 + k, frames=8, width=128, height=96,
                        max_depth=6) for k in range(3)]
    params, losses = warm_start.train(3, 4000, 300, 8192, 2e-3, 0, gap_tol=1e-5, rows_per_scan=6000,
                                      scan_iter=iter(scans), log=lambda *_: None)
    assert params.shape == (of.ofu_mlp_num_params(),) and np.all(np.isfinite(params))
    assert losses[-1][1] < 0.5 * losses[0][1]
    held = make_scene("at_scale", 1000, frames=12, width=128, height=96, max_depth=6)
    rows = warm_start.evaluate(params, [held], torch, log=lambda *_: None)
    r = rows[0]
    assert r["converged"] and r["seed"] == 1000
    for form in ("plain_f32", "f16_samples", "f32_warm_start", "f16_warm_start"):
        assert r[form]["iters"] > 0 and r[form]["ms"] > 0
    assert r["plain_f32"]["reached"]
