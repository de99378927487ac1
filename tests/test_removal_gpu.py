"""Removal of arrived agents (Sec. 4), step by step against the oracle.

After every GPU step the per-step parity with the oracle is checked from the
identical state, then the GPU removes the arrived agents in place and the
kept set must equal the oracle's arrival rule applied to the GPU's new
state, bit for bit (it is an FP32 decision).
"""
import numpy as np
import pytest

import oracle
from paper_2008_11578_gb300 import api, scenes
from tests.parity_util import compare

pytestmark = pytest.mark.gpu


def _run(scene, n_steps):
    import torch
    ds = api.DeviceScene(scene, "cuda", debug=True)
    cur = scene.copy()
    ids = np.arange(scene.n)
    removed_total = 0
    for t in range(n_steps):
        if ds.n == 0:
            ds.step(1)                     # an empty scene steps as a no-op
            continue
        ds.step(1)
        torch.cuda.synchronize()
        n = ds.n
        g = dict(pos=ds.pos[:n].cpu().numpy(), vel=ds.vel[:n].cpu().numpy(),
                 **{k: v[:n].cpu().numpy() for k, v in ds.dbg.items()})
        if ds.wp_idx is not None:
            g["wp_idx"] = ds.wp_idx[:n].cpu().numpy()
        compare(cur, g)
        new_wp = g.get("wp_idx")
        gone = oracle.arrived(cur, g["pos"], new_wp)
        kept = ds.remove_arrived()
        assert np.array_equal(kept, np.nonzero(~gone)[0]), t
        removed_total += int(gone.sum())
        nxt = cur.subset(np.nonzero(~gone)[0])
        nxt.pos, nxt.vel = g["pos"][~gone], g["vel"][~gone]
        if new_wp is not None:
            nxt.wp_idx = new_wp[~gone]
        cur, ids = nxt, ids[~gone]
        # the compacted device arrays hold exactly the kept agents
        assert np.array_equal(ds.pos[:ds.n].cpu().numpy(), cur.pos)
        assert np.array_equal(ds.goal[:ds.n].cpu().numpy(), cur.goal)
        assert np.array_equal(ds.type[:ds.n].cpu().numpy(), cur.type)
    ds.close()
    return removed_total, ids


def test_removal_open_square():
    s = scenes.open_square(150, 20.0, seed=51)
    removed, ids = _run(s, 80)
    assert removed > 60


def test_removal_with_routes():
    s = scenes.waypoint_square(n_ped=60, n_veh=6, side=20.0, n_wp=3, seed=52)
    removed, ids = _run(s, 90)
    assert removed >= 50


def test_remove_on_empty_and_status():
    s = scenes.open_square(50, 10.0, seed=53)
    s.goal = s.pos.copy()                           # everyone is already at the goal
    ds = api.DeviceScene(s, "cuda")
    assert len(ds.remove_arrived()) == 0 and ds.n == 0
    ds.step(3)
    assert ds.remove_arrived().shape == (0,) and ds.sync_status() == 0
    ds.close()
