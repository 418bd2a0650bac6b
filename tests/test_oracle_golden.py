"""Golden fixtures (no GPU): the paper's printed constants as the oracle and
the workloads use them, and regression values of the oracle itself
(tests/golden/oracle_tiny.json, written by tests/golden/make_golden.py)."""
import importlib.util
import json
import os

import numpy as np
import pytest

from oracle import descent, octree
from paper_1608_07411_gb300.scenes import make_scene
from tests._helpers import blocky_field, random_octree

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return json.load(fh)


def test_paper_constants():
    paper = _load("paper_values.json")
    sched = paper["descent_schedule"]
    assert (descent.XI0, descent.HALVE_EVERY, descent.ITERS) == (
        sched["xi0"], sched["halve_every"], sched["iterations"])
    for name in ("sphere", "torus_box", "at_scale"):
        assert make_scene(name, 0, frames=2, width=8, height=6).spread_tau == \
            paper["spread_threshold"]["tau"]


def test_join_threshold_above_one_disables_joins():
    """|u| <= 1 for every TSDF value, so no leaf passes |u| > tau_j > 1."""
    tau = _load("paper_values.json")["join_disabled_above_one"]["tau_join"] + 1e-9
    k, lv = random_octree(4, 3, p_split=0.7, min_level=2)
    u = blocky_field(k, lv, 4, 0)
    u = np.where(np.abs(u) > 0.9, np.sign(u), u)          # saturated regions at exactly +-1
    _, _, _, _, _, n_split, n_join = octree.restructure(k, lv, u, np.zeros((len(k), 3)), 4,
                                                        0.95, tau)
    assert n_join == 0
    _, _, _, _, _, _, n_join_on = octree.restructure(k, lv, u, np.zeros((len(k), 3)), 4,
                                                     0.95, 0.99)
    assert n_join_on > 0


def test_oracle_regression_values():
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(GOLDEN, "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    want = _load("oracle_tiny.json")
    got = mod.values()
    for key in ("leaves", "structure_sha", "samples", "leaves_after_restructure"):
        assert got[key] == want[key], key
    for key in ("median_init_sum", "descent_energy_after_30"):
        assert got[key] == pytest.approx(want[key], rel=1e-9), key
    np.testing.assert_allclose(got["primal_dual_after_20"], want["primal_dual_after_20"], rtol=1e-9)
