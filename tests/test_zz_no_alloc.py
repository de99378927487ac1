"""orca_step_noalloc: the ORCA step for callers that cannot allocate device
memory (code inside another framework's memory pool, plugins barred from
cudaMalloc, loops that must never allocate).  It keeps its scratch in a fixed
area inside the library instead of a caller workspace.

Checked through the C ABI against the ordinary scene path (orca_step on a
caller workspace) bit for bit, on two calls in a row with a call on a scene
of another size between them, so the second call also shows that leftovers
in the shared scratch area change nothing; the first call is also checked
against the FP64 oracle.
The file name sorts last so that a run stopping at its first failure has
run every other test before this one.
"""
import numpy as np
import pytest

import oracle
from paper_2008_11578_gb300 import _lib, api, scenes
from tests.parity_util import P_TOL, V_TOL, half_ulp

pytestmark = pytest.mark.gpu


def _noalloc(ds, n_steps):
    st = api.orca_step_noalloc(ds.params, ds._agents, n_steps, synchronize=True)
    assert st == 0, api.orca_status_string(st)


def _same(a, b):
    import torch
    assert torch.equal(a.pos, b.pos) and torch.equal(a.vel, b.vel)
    if a.wp_idx is not None:
        assert torch.equal(a.wp_idx, b.wp_idx)


def test_noalloc_matches_scene_path_on_two_calls():
    """Two calls in a row on one scene, with a call on a scene of another
    size and grid between them (its leftovers are in the shared scratch
    area when the second call starts).  Every call equals the ordinary
    scene path bit for bit (both run the same kernels, and the step does not
    depend on the order agents are binned in); the first one also meets
    the FP64 oracle."""
    import torch
    s = scenes.waypoint_square(n_ped=3000, n_veh=40, side=90.0, seed=21)
    o = scenes.open_square(1200, 45.0, seed=23)
    ref = api.DeviceScene(s, "cuda")                 # ordinary path, caller workspace
    mine = api.DeviceScene(s, "cuda")                # same tensors, used without the scene
    other_ref = api.DeviceScene(o, "cuda")
    other = api.DeviceScene(o, "cuda")
    for ds in (mine, other):
        assert api.orca_workspace_bytes(ds.params, ds.n) <= _lib.NOALLOC_SCRATCH_BYTES
    assert (mine.n, mine.params.grid_nx) != (other.n, other.params.grid_nx)

    ref.step(1)
    _noalloc(mine, 1)
    torch.cuda.synchronize()
    _same(mine, ref)
    r = oracle.step(s)
    vel = mine.vel.cpu().numpy().astype(np.float64)
    pos = mine.pos.cpu().numpy().astype(np.float64)
    assert np.abs(vel - r.vel).max() <= V_TOL
    assert (np.abs(pos - r.pos) <= P_TOL + half_ulp(r.pos)).all()
    assert np.array_equal(mine.wp_idx.cpu().numpy(), r.wp_idx)

    other_ref.step(2)
    _noalloc(other, 2)                               # another scene in between
    torch.cuda.synchronize()
    _same(other, other_ref)

    ref.step(3)
    _noalloc(mine, 3)                                # second call on the first scene
    torch.cuda.synchronize()
    _same(mine, ref)
    for ds in (ref, mine, other_ref, other):
        ds.close()


def test_noalloc_refuses_scenes_beyond_the_scratch_area():
    s = scenes.open_square(40000, 280.0, seed=22)
    ds = api.DeviceScene(s, "cuda")
    assert api.orca_workspace_bytes(ds.params, ds.n) > _lib.NOALLOC_SCRATCH_BYTES
    before = ds.pos.clone()
    st = api.orca_step_noalloc(ds.params, ds._agents, 1, synchronize=True)
    assert st == 5 and api.orca_status_string(st) == "capacity exceeded"
    assert (ds.pos == before).all()                  # nothing ran
    ds.close()
