"""Write the stored expected values under tests/golden/ from the oracle alone.

The paper prints no worked example, so every fixture here is the FP64
oracle's output on a small seeded scene, written by this script (it imports
only the oracle and the seeded scene generators).  Run from the repo root:

    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle                                    # noqa: E402
from paper_2008_11578_gb300 import scenes         # noqa: E402

STEPS = 3


def golden_scene():
    """48 pedestrians and 4 vehicles in 10 x 10 m (dense: overlaps and
    least-penetration fallbacks on the first step)."""
    s = scenes.open_square(52, 10.0, seed=5)
    s.type[:4] = 1
    s.radius[:4] = np.float32(1.5)
    s.max_speed[:4] = np.float32(5.0)
    return s


def rollout():
    """Oracle steps from the FP32 state, each result rounded to FP32 before
    the next step (the state the CUDA path carries)."""
    s = golden_scene()
    out = []
    for t in range(STEPS):
        r = oracle.step(s)
        out.append((s.pos.copy(), s.vel.copy(), r))
        s.pos = r.pos.astype(np.float32)
        s.vel = r.vel.astype(np.float32)
    return out


def write(path):
    k = golden_scene().params.max_neighbors
    with open(path, "w") as f:
        f.write("# ORCA step (Sec. 3; responsibility table Sec. 3.1) of golden_scene(), "
                "FP64 oracle, %d steps\n" % STEPS)
        f.write("# written by tests/golden/make_golden.py from oracle/ only\n")
        f.write("# t agent cnt flags vel_x vel_y pos_x pos_y nbr[0..%d]\n" % (k - 1))
        for t, (_, _, r) in enumerate(rollout()):
            for i in range(len(r.cnt)):
                f.write("%d %d %d %d %.17g %.17g %.17g %.17g %s\n" % (
                    t, i, r.cnt[i], r.flags[i], r.vel[i, 0], r.vel[i, 1], r.pos[i, 0], r.pos[i, 1],
                    " ".join(str(int(x)) for x in r.nbr[i][:k])))


def read(path):
    rows = [line.split() for line in open(path) if not line.startswith("#")]
    return rows


if __name__ == "__main__":
    oracle.build()
    write(os.path.join(HERE, "oracle_dense_square_52.txt"))
