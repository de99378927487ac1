"""Failure detection on the GPU without a fault: a bounded wait that runs out.

With ORCA_DEBUG_BARRIER_TIMEOUT the first block of the binning kernel never
arrives at the grid barrier, so every other block's bounded wait gives up.
The step must end by itself well inside a few seconds, report
ORCA_ERR_TIMEOUT through the status call, leave the caller's arrays as they
were, and leave the device usable for the next scene.
"""
import time

import numpy as np
import pytest

from paper_2008_11578_gb300 import api, scenes
from tests.parity_util import compare, gpu_step

pytestmark = pytest.mark.gpu

ORCA_ERR_TIMEOUT = 3


@pytest.mark.parametrize("n,side", [(20000, 200.0), (10, 5.0)])
def test_barrier_timeout_is_reported_and_the_device_stays_usable(n, side):
    import torch
    sc = scenes.open_square(n, side, seed=11)
    ds = api.DeviceScene(sc, "cuda", flags=api.BARRIER_TIMEOUT_TEST)
    p0, v0 = ds.pos.clone(), ds.vel.clone()
    t0 = time.perf_counter()
    ds.step(1)
    torch.cuda.synchronize()
    elapsed = time.perf_counter() - t0
    assert ds.sync_status() == ORCA_ERR_TIMEOUT
    assert elapsed < 10.0
    # the solve kernel saw the error and left the caller's state alone
    assert torch.equal(ds.pos, p0) and torch.equal(ds.vel, v0)
    ds.close()
    # a fresh scene on the same device steps normally and matches the oracle
    g = gpu_step(sc)
    assert g["status"] == 0
    compare(sc, g, sel=np.arange(0, n, max(1, n // 400)))


def test_status_call_clears_the_timeout():
    import torch
    sc = scenes.open_square(5000, 100.0, seed=12)
    ds = api.DeviceScene(sc, "cuda", flags=api.BARRIER_TIMEOUT_TEST)
    ds.step(2)
    torch.cuda.synchronize()
    assert ds.sync_status() == ORCA_ERR_TIMEOUT
    # the error word, barrier words and counts were reset: nothing pending
    assert ds.sync_status() == 0
    ds.close()
