"""Writes tests/golden/oracle_tiny.json: regression values of the oracle on a
tiny seeded scene.  Calls only ``oracle`` and the seeded input generator.

    python tests/golden/make_golden.py
"""
import hashlib
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import descent, solver  # noqa: E402
from paper_1608_07411_gb300.scenes import make_scene  # noqa: E402

SCENE = dict(name="sphere", seed=5, frames=4, width=40, height=30, max_depth=4)


def values():
    kw = {k: v for k, v in SCENE.items() if k not in ("name", "seed")}
    s = make_scene(SCENE["name"], SCENE["seed"], **kw)
    st = solver.initial_state(s)
    out = {"scene": SCENE, "leaves": int(len(st.keys)),
           "structure_sha": hashlib.sha256(st.keys.tobytes() + st.levels.tobytes()).hexdigest()[:16],
           "samples": int(st.W.sum()), "median_init_sum": float(st.u.sum())}
    solver.step(st, 20)
    out["primal_dual_after_20"] = list(solver.energies(st))
    solver.restructure(st, s)
    out["leaves_after_restructure"] = int(len(st.keys))
    d = solver.initial_state(s)
    descent.descend(d, 30, 0)
    out["descent_energy_after_30"] = descent.energy(d)
    return out


if __name__ == "__main__":
    v = values()
    v["_about"] = ("Oracle regression values, written by tests/golden/make_golden.py from oracle/ "
                   "(not from the CUDA path); a change to the oracle's arithmetic changes them.")
    with open(os.path.join(HERE, "oracle_tiny.json"), "w") as fh:
        json.dump(v, fh, indent=1)
    print(json.dumps(v, indent=1))
