"""The stored oracle fixture under tests/golden/ (written by
tests/golden/make_golden.py from the oracle alone).

CPU: the oracle still reproduces it exactly (a change of the oracle's
arithmetic shows up here).  GPU: the CUDA step, from the fixture's FP32
states, meets it like it meets the live oracle.
"""
import os
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_golden  # noqa: E402

FIXTURE = os.path.join(HERE, "golden", "oracle_dense_square_52.txt")


def _load():
    rows = make_golden.read(FIXTURE)
    k = make_golden.golden_scene().params.max_neighbors
    t = np.array([int(r[0]) for r in rows])
    steps = []
    for s in range(make_golden.STEPS):
        R = [r for r, tt in zip(rows, t) if tt == s]
        steps.append(dict(
            cnt=np.array([int(r[2]) for r in R]), flags=np.array([int(r[3]) for r in R]),
            vel=np.array([[float(r[4]), float(r[5])] for r in R]),
            pos=np.array([[float(r[6]), float(r[7])] for r in R]),
            nbr=np.array([[int(x) for x in r[8:8 + k]] for r in R])))
    return steps


def test_oracle_reproduces_the_fixture():
    import oracle
    oracle.build()
    steps = _load()
    for (_, _, r), g in zip(make_golden.rollout(), steps):
        assert np.array_equal(r.cnt, g["cnt"]) and np.array_equal(r.nbr[:, :g["nbr"].shape[1]], g["nbr"])
        assert np.array_equal(r.flags, g["flags"])
        assert np.array_equal(r.vel, g["vel"]) and np.array_equal(r.pos, g["pos"])
    # the fixture exercises both LP paths and the vehicle entries
    assert (steps[0]["flags"] & 1).any() and not (steps[0]["flags"] & 1).all()


@pytest.mark.gpu
def test_cuda_step_meets_the_fixture():
    from tests.parity_util import P_TOL, V_TOL, gpu_step, half_ulp
    steps = _load()
    s = make_golden.golden_scene()
    for t, g in enumerate(steps):
        if t:
            s.pos = steps[t - 1]["pos"].astype(np.float32)
            s.vel = steps[t - 1]["vel"].astype(np.float32)
        out = gpu_step(s)
        assert out["status"] == 0
        assert np.array_equal(out["cnt"], g["cnt"]), t
        assert np.array_equal(out["nbr"][:, :g["nbr"].shape[1]], g["nbr"]), t
        assert np.abs(out["vel"].astype(np.float64) - g["vel"]).max() <= V_TOL, t
        assert (np.abs(out["pos"].astype(np.float64) - g["pos"]) <= P_TOL + half_ulp(g["pos"])).all(), t
