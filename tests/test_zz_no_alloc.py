"""orca_step_noalloc: the ORCA step for callers that cannot allocate device
memory (code inside another framework's memory pool, plugins barred from
cudaMalloc, loops that must never allocate).  It keeps its scratch in a fixed
area inside the library instead of a caller workspace.

Checked through the C ABI against the ordinary scene path (orca_step on a
caller workspace), on two calls in a row, so the second call also shows that
leftovers of the first one in the shared scratch area change nothing.
The file name sorts last so that a run stopping at its first failure has
run every other test before this one.
"""
import numpy as np
import pytest

from paper_2008_11578_gb300 import _lib, api, scenes
from tests.parity_util import P_TOL, V_TOL, half_ulp

pytestmark = pytest.mark.gpu


def _agree(a_pos, a_vel, b_pos, b_vel):
    assert np.abs(a_vel.astype(np.float64) - b_vel).max() <= V_TOL
    assert (np.abs(a_pos.astype(np.float64) - b_pos) <= P_TOL + half_ulp(b_pos)).all()


def test_noalloc_matches_scene_path_on_two_calls():
    import torch
    s = scenes.waypoint_square(n_ped=3000, n_veh=40, side=90.0, seed=21)
    ref = api.DeviceScene(s, "cuda")                 # ordinary path, caller workspace
    mine = api.DeviceScene(s, "cuda")                # same tensors layout, used without a scene
    assert api.orca_workspace_bytes(mine.params, mine.n) <= _lib.NOALLOC_SCRATCH_BYTES
    for n_steps in (2, 3):                           # two calls in a row
        ref.step(n_steps)
        st = api.orca_step_noalloc(mine.params, mine._agents, n_steps, synchronize=True)
        assert st == 0, api.orca_status_string(st)
        torch.cuda.synchronize()
        _agree(mine.pos.cpu().numpy(), mine.vel.cpu().numpy(),
               ref.pos.cpu().numpy().astype(np.float64), ref.vel.cpu().numpy().astype(np.float64))
        assert torch.equal(mine.wp_idx, ref.wp_idx)
    ref.close()
    mine.close()


def test_noalloc_refuses_scenes_beyond_the_scratch_area():
    s = scenes.open_square(40000, 280.0, seed=22)
    ds = api.DeviceScene(s, "cuda")
    assert api.orca_workspace_bytes(ds.params, ds.n) > _lib.NOALLOC_SCRATCH_BYTES
    before = ds.pos.clone()
    st = api.orca_step_noalloc(ds.params, ds._agents, 1, synchronize=True)
    assert st == 5 and api.orca_status_string(st) == "capacity exceeded"
    assert (ds.pos == before).all()                  # nothing ran
    ds.close()
