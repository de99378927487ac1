"""Batched scenes and CUDA graphs (needs a GPU).

A batch advances many independent scenes by one launch per phase of the
step.  Every scene of a batch must compute exactly what the single-scene
path computes for it alone (bit for bit), a replayed CUDA graph exactly what
the eager calls compute, and the autotuner's launch shapes exactly what the
default shape computes.  Sampled agents are also checked against the FP64
oracle scene by scene.
"""
import numpy as np
import pytest

from paper_2008_11578_gb300 import api, autotune, scenes
from tests.parity_util import compare, gpu_step

pytestmark = pytest.mark.gpu


def _mixed_batch():
    """Uneven scenes: empty, one agent, uniform squares of several sizes and
    densities, a shared-space crossing, a waypoint scene and a k = 32 scene."""
    out = scenes.batched(n_scenes=12, lo=100, hi=3000, seed=31)
    out.insert(3, scenes.open_square(0, 10.0))
    out.insert(5, scenes.open_square(1, 10.0, seed=5))
    out.append(scenes.shared_space(n_ped=2000, n_veh=40, side=90.0, seed=6))
    out.append(scenes.waypoint_square(n_ped=800, n_veh=16, side=45.0, seed=7))
    k32 = scenes.open_square(900, 35.0, seed=8)
    k32.params.max_neighbors = 32
    out.append(k32)
    return out


def _batch_run(scene_list, n_steps, **kw):
    import torch
    b = api.DeviceBatch(scene_list, "cuda", debug=True, **kw)
    b.step(n_steps)
    torch.cuda.synchronize()
    assert b.sync_status() == 0
    out = dict(pos=b.pos.cpu().numpy(), vel=b.vel.cpu().numpy(),
               wp_idx=None if b.wp_idx is None else b.wp_idx.cpu().numpy(),
               **{k: v.cpu().numpy() for k, v in b.dbg.items()})
    offsets = b.offsets.copy()
    b.close()
    return out, offsets


def test_batch_equals_each_scene_alone():
    sl = _mixed_batch()
    got, off = _batch_run(sl, 3)
    for s, sc in enumerate(sl):
        sl_ = slice(off[s], off[s + 1])
        ref = gpu_step(sc, n_steps=3)
        assert np.array_equal(got["pos"][sl_], ref["pos"]), s
        assert np.array_equal(got["vel"][sl_], ref["vel"]), s
        k = sc.params.max_neighbors
        nb = got["nbr"][sl_][:, :k]
        nb = np.where(nb >= 0, nb - off[s], -1)
        assert np.array_equal(nb, ref["nbr"]), s
        assert (got["nbr"][sl_][:, k:] == -1).all()
        assert np.array_equal(got["cell"][sl_], ref["cell"]), s
        if sc.route is not None:
            assert np.array_equal(got["wp_idx"][sl_], ref["wp_idx"])


def test_batch_against_oracle_per_scene():
    """One step of every scene of a 40-scene batch against the oracle."""
    import torch
    sl = scenes.batched(n_scenes=40, lo=100, hi=5000, seed=32)
    b = api.DeviceBatch(sl, "cuda", debug=True)
    b.step(1)
    torch.cuda.synchronize()
    pos, vel = b.pos.cpu().numpy(), b.vel.cpu().numpy()
    dbg = {k: v.cpu().numpy() for k, v in b.dbg.items()}
    rng = np.random.default_rng(3)
    for s, sc in enumerate(sl):
        r = b.scene_slice(s)
        g = dict(pos=pos[r], vel=vel[r], cell=dbg["cell"][r], cnt=dbg["cnt"][r],
                 flags=dbg["flags"][r],
                 nbr=np.where(dbg["nbr"][r] >= 0, dbg["nbr"][r] - r.start, -1))
        sel = np.sort(rng.choice(sc.n, min(sc.n, 300), replace=False))
        compare(sc, g, sel=sel)
    b.close()


def test_graph_replay_equals_eager_and_launch_count():
    import torch
    sl = scenes.batched(n_scenes=30, lo=100, hi=4000, seed=33)
    eager = api.DeviceBatch(sl, "cuda")
    eager.step(5)
    graph = api.DeviceBatch(sl, "cuda")
    graph.capture(5)
    assert np.array_equal(graph.pos.cpu().numpy(), np.concatenate([s.pos for s in sl]))
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(eager.pos, graph.pos) and torch.equal(eager.vel, graph.vel)
    # a second replay continues from the new state, like a second eager call
    eager.step(5)
    graph.replay(torch.cuda.Stream())
    torch.cuda.synchronize()
    assert torch.equal(eager.pos, graph.pos) and torch.equal(eager.vel, graph.vel)
    assert eager.launch_count(50) == 2 * 50      # binning + solve per step, any scene count
    assert graph.sync_status() == 0
    eager.close()
    graph.close()


def test_scene_graph_equals_eager():
    import torch
    s = scenes.waypoint_square(n_ped=1000, n_veh=20, side=50.0, seed=34)
    a = api.DeviceScene(s, "cuda")
    b = api.DeviceScene(s, "cuda")
    d = torch.as_tensor(np.random.default_rng(0).normal(0, 0.2, (4, s.n, 2)).astype(np.float32),
                        device="cuda")
    a.step(4, d)
    b.capture(4, d)
    b.replay()
    torch.cuda.synchronize()
    assert torch.equal(a.pos, b.pos) and torch.equal(a.vel, b.vel)
    assert torch.equal(a.wp_idx, b.wp_idx)
    a.close()
    b.close()


def test_autotuned_shapes_change_nothing():
    import torch
    sl = scenes.batched(n_scenes=16, lo=100, hi=3000, seed=35)
    res = autotune.tune_batch(sl, alphas=(0.5, 1.0, 2.0), aspects=(1.0, 4.0), blocks=(64, 128),
                              steps=2)
    assert len(res.table) == 12 and res.ms_per_step > 0
    ref = api.DeviceBatch(sl, "cuda")
    ref.step(4)
    for a, asp, bs, _ in res.table:
        b = api.DeviceBatch(sl, "cuda", cell_sizes=[asp * a * s.params.cell_size for s in sl],
                            cell_heights=[a * s.params.cell_size for s in sl], block_size=bs)
        b.step(4)
        torch.cuda.synchronize()
        assert torch.equal(ref.pos, b.pos) and torch.equal(ref.vel, b.vel), (a, asp, bs)
        b.close()
    ref.close()


def test_single_scene_batch_equals_scene():
    import torch
    s = scenes.open_square(2000, 60.0, seed=36)
    b = api.DeviceBatch([s], "cuda")
    b.step(3)
    g = gpu_step(s, n_steps=3)
    torch.cuda.synchronize()
    assert np.array_equal(b.pos.cpu().numpy(), g["pos"])
    b.close()


def test_batch_nonfinite_reports_status():
    import torch
    sl = scenes.batched(n_scenes=5, lo=100, hi=500, seed=37)
    sl[2].pos[3, 1] = np.inf
    b = api.DeviceBatch(sl, "cuda")
    b.step(1)
    torch.cuda.synchronize()
    assert b.sync_status() == 4
    b.close()
