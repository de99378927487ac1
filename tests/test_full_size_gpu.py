"""Parity at the full sizes of the workloads, in the launch shapes the
benchmark times, on outputs the oracle computes agent by agent.

The benchmark advances the 1M-agent and 65k-agent scenes by one-step calls
(every call bins its first step in the order the previous call recorded),
and the 512-scene batch with the autotuner's cell factor and block size.
Every test below does the same, then checks sampled agents of every step
against the FP64 oracle from the identical FP32 state, and the cells of all
agents bit for bit.
"""
import numpy as np
import pytest

import oracle
from paper_2008_11578_gb300 import api, scenes
from tests.parity_util import cells_oracle, compare
from tests.parity_util import gpu_step as gpu_step_from

pytestmark = pytest.mark.gpu


def _calls(scene, cell_size, block_size, n_calls, n_sample, seed, cell_height=None):
    import torch
    ds = api.DeviceScene(scene, "cuda", cell_size=cell_size, block_size=block_size, debug=True,
                         cell_height=cell_height)
    cur = scene.copy()
    rng = np.random.default_rng(seed)
    fallbacks = 0
    for t in range(n_calls):
        ds.step(1)
        torch.cuda.synchronize()
        assert ds.sync_status() == 0
        g = dict(pos=ds.pos.cpu().numpy(), vel=ds.vel.cpu().numpy(),
                 **{k: v.cpu().numpy() for k, v in ds.dbg.items()})
        if ds.wp_idx is not None:
            g["wp_idx"] = ds.wp_idx.cpu().numpy()
        assert np.array_equal(g["cell"], cells_oracle(cur, cell_size, cell_height)), t
        # every sample includes fallback agents (the least-penetration path)
        inf = np.nonzero(g["flags"] & 1)[0]
        sel = rng.choice(scene.n, n_sample, replace=False)
        if len(inf):
            sel = np.concatenate([sel, rng.choice(inf, min(len(inf), n_sample // 4), replace=False)])
        st = compare(cur, g, sel=np.unique(sel))
        fallbacks += st["infeasible_oracle"]
        cur.pos, cur.vel = g["pos"], g["vel"]
        if "wp_idx" in g:
            cur.wp_idx = g["wp_idx"]
    ds.close()
    return fallbacks


def test_clusters_1m_bench_shape_two_calls():
    """990,000 pedestrians + 10,000 vehicles in 64 clusters over 2 x 2 km;
    cell 1.5 m and solve block 64 (the autotuner's choice for this workload)."""
    assert _calls(scenes.clusters(), 1.5, 64, 2, 3000, 1) > 1000


def test_shared_space_65k_bench_shape_three_calls():
    """64,000 pedestrians in two counter-flowing streams + 1,000 vehicles in
    east-west lanes, 500 x 500 m."""
    s = scenes.shared_space()
    assert s.n == 65000
    _calls(s, float(s.params.cell_size), 0, 3, 3000, 2)


def test_batch_512_scenes_bench_shape():
    """The 512-scene batch (1.79M agents) with the cell factor and block size
    the autotuner picks for it (0.5 x each scene's cell, block 64): one step,
    then the batch's graph of two more, checked on sampled scenes."""
    import torch
    sl = scenes.batched()
    assert len(sl) == 512
    b = api.DeviceBatch(sl, "cuda", cell_sizes=[0.5 * float(sc.params.cell_size) for sc in sl],
                        block_size=64, debug=True)
    rng = np.random.default_rng(5)
    sizes = np.array([sc.n for sc in sl])
    pick = np.unique(np.concatenate([rng.choice(len(sl), 24, replace=False),
                                     [int(np.argmax(sizes)), int(np.argmin(sizes))]]))
    cur = [sc.copy() for sc in sl]
    for t in range(2):
        b.step(1)
        torch.cuda.synchronize()
        assert b.sync_status() == 0
        pos, vel = b.pos.cpu().numpy(), b.vel.cpu().numpy()
        dbg = {k: v.cpu().numpy() for k, v in b.dbg.items()}
        for s in pick:
            r = b.scene_slice(int(s))
            g = dict(pos=pos[r], vel=vel[r], cell=dbg["cell"][r], cnt=dbg["cnt"][r],
                     flags=dbg["flags"][r],
                     nbr=np.where(dbg["nbr"][r] >= 0, dbg["nbr"][r] - r.start, -1))
            sel = np.sort(rng.choice(cur[s].n, min(cur[s].n, 200), replace=False))
            compare(cur[s], g, sel=sel)
        for s, sc in enumerate(cur):
            r = b.scene_slice(s)
            sc.pos, sc.vel = pos[r], vel[r]
    b.close()


def test_clusters_1m_long_run_stays_consistent():
    """A soak run at full size: 100 one-step calls (each binning its first
    step in the order the previous call recorded) and one 100-step call, in
    the benchmark's launch shape.  The status stays clean, the state stays
    finite and collision-free in aggregate, and the last step still meets the
    oracle on sampled agents."""
    import torch
    s = scenes.clusters()
    ds = api.DeviceScene(s, "cuda", cell_size=1.5, block_size=64, debug=True)
    for _ in range(100):
        ds.step(1)
    ds.step(100)
    torch.cuda.synchronize()
    assert ds.sync_status() == 0
    pos, vel = ds.pos.cpu().numpy(), ds.vel.cpu().numpy()
    assert np.isfinite(pos).all() and np.isfinite(vel).all()
    assert (np.hypot(vel[:, 0], vel[:, 1]) <= s.max_speed * (1 + 1e-5) + 1e-5).all()
    cur = s.copy()
    cur.pos, cur.vel = pos.copy(), vel.copy()
    ds.step(1)
    torch.cuda.synchronize()
    assert ds.sync_status() == 0
    g = dict(pos=ds.pos.cpu().numpy(), vel=ds.vel.cpu().numpy(),
             **{k: v.cpu().numpy() for k, v in ds.dbg.items()})
    rng = np.random.default_rng(9)
    compare(cur, g, sel=np.sort(rng.choice(s.n, 3000, replace=False)))
    ds.close()


def _jammed_state(scene, n_calls, **shape):
    import torch
    ds = api.DeviceScene(scene, "cuda", **shape)
    for _ in range(n_calls):
        ds.step(1)
    torch.cuda.synchronize()
    assert ds.sync_status() == 0
    cur = scene.copy()
    cur.pos, cur.vel = ds.pos.cpu().numpy(), ds.vel.cpu().numpy()
    ds.close()
    return cur


def test_cluster_density_after_24_steps_every_agent():
    """Jams form after a few steps: many agents are pressed together with
    nearly equal velocities, and their LPs sit on the edge of feasibility
    (t* close to 0, several half-planes through nearly one point).  From the
    state after 24 steps, one step is compared with the oracle for EVERY
    agent of the 62,500-agent cluster scene."""
    s = scenes.clusters(n=62500, side=500.0, n_clusters_axis=2)
    cur = _jammed_state(s, 24, cell_size=3.0, cell_height=1.5, block_size=64)
    g = gpu_step_from(cur, cell_size=3.0, cell_height=1.5, block_size=64)
    st = compare(cur, g)
    assert st["infeasible_oracle"] > 10000


def test_clusters_1m_near_feasible_agents_after_24_calls():
    """The 1M workload after 24 one-step calls (the state the benchmark
    times): every agent whose step reports a least penetration t* in
    (0, 0.2) m/s, the near-feasible band, and 2,000 random agents against
    the oracle."""
    s = scenes.clusters()
    cur = _jammed_state(s, 24, cell_size=3.0, cell_height=1.5, block_size=64)
    g = gpu_step_from(cur, cell_size=3.0, cell_height=1.5, block_size=64)
    near = np.nonzero((g["tstar"] > 0.0) & (g["tstar"] < 0.2))[0]
    rng = np.random.default_rng(24)
    sel = np.unique(np.concatenate([near, rng.choice(s.n, 2000, replace=False)]))
    assert len(near) > 100
    compare(cur, g, sel=sel)
