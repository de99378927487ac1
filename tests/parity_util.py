"""Helpers shared by the GPU parity tests: run one step on both sides and
compare element by element.

Tolerances (from the accuracy target of the method's per-step update):
  * cells, neighbour sets and their order: bit-exact;
  * new velocity: |dv| <= 1e-4 m/s per component;
  * new position: |dp| <= 1e-5 m per component on top of the FP32
    representation error of the stored position (half an ulp of |p|),
    since the CUDA path stores FP32 positions and the oracle's are FP64.
"""
from __future__ import annotations

import numpy as np

import oracle

V_TOL = 1e-4
P_TOL = 1e-5


def half_ulp(x):
    x = np.abs(np.asarray(x, dtype=np.float32))
    return 0.5 * (np.nextafter(x, np.float32(np.inf)) - x).astype(np.float64)


def gpu_step(scene, n_steps=1, cell_size=None, block_size=0, vpref_delta=None, debug=True,
             flags=0, cell_height=None):
    """Run the CUDA path on a copy of ``scene``; returns numpy outputs."""
    import torch
    from paper_2008_11578_gb300 import api
    ds = api.DeviceScene(scene, "cuda", cell_size=cell_size, block_size=block_size, debug=debug,
                         flags=flags, cell_height=cell_height)
    vpd = None
    if vpref_delta is not None:
        vpd = torch.as_tensor(np.ascontiguousarray(vpref_delta, dtype=np.float32), device="cuda")
    ds.step(n_steps, vpd)
    torch.cuda.synchronize()
    st = ds.sync_status()
    out = dict(pos=ds.pos.cpu().numpy(), vel=ds.vel.cpu().numpy(), status=st)
    if ds.wp_idx is not None:
        out["wp_idx"] = ds.wp_idx.cpu().numpy()
    if debug:
        for k, v in ds.dbg.items():
            out[k] = v.cpu().numpy()
    ds.close()
    return out


def cells_oracle(scene, cell_size=None, cell_height=None):
    """The oracle's cell of every agent for a w x h grid over the scene box."""
    p = scene.params
    w, h = p.cell_dims(cell_size, cell_height)
    nx, ny = p.grid_dims(cell_size, cell_height)
    inv = (np.float32(1.0) / np.float32(w), np.float32(1.0) / np.float32(h))
    return oracle.cells(scene.pos, p.origin, inv, nx, ny)


def compare(scene, g, sel=None, r=None, vpref_delta=None):
    """Compare a GPU step ``g`` (from ``scene``'s state) with the oracle.

    Returns a dict of statistics; raises AssertionError on any discrete
    mismatch or tolerance violation.
    """
    if r is None:
        r = oracle.step(scene, sel=sel, vpref_delta=vpref_delta)
    idx = np.arange(scene.n) if sel is None else np.asarray(sel)
    k = scene.params.max_neighbors
    # discrete parts: bit-exact
    cnt_g = g["cnt"][idx]
    assert np.array_equal(cnt_g, r.cnt), f"neighbour counts differ at {np.nonzero(cnt_g != r.cnt)[0][:10]}"
    nb_g = g["nbr"][idx][:, :k]
    assert np.array_equal(nb_g, r.nbr), f"neighbour lists differ at {np.nonzero((nb_g != r.nbr).any(1))[0][:10]}"
    if "wp_idx" in g:
        assert np.array_equal(g["wp_idx"][idx], r.wp_idx)
    dv = np.abs(g["vel"][idx].astype(np.float64) - r.vel)
    dp = np.abs(g["pos"][idx].astype(np.float64) - r.pos)
    ptol = P_TOL + half_ulp(r.pos)
    bad_v = (dv > V_TOL).any(1)
    bad_p = (dp > ptol).any(1)
    stats = dict(n=len(idx), max_dv=float(dv.max(initial=0)), max_dp=float(dp.max(initial=0)),
                 p9999_dv=float(np.quantile(dv.max(1), 0.9999)) if len(idx) else 0.0,
                 n_bad_v=int(bad_v.sum()), n_bad_p=int(bad_p.sum()),
                 infeasible_oracle=int((r.flags & 1).sum()),
                 infeasible_gpu=int((g["flags"][idx] & 1).sum()),
                 ill_conditioned=int((r.cond > 1e3).sum()))
    if bad_v.any() or bad_p.any():
        w = np.nonzero(bad_v | bad_p)[0][:8]
        detail = [(int(idx[i]), dv[i].max(), float(r.cond[i]), int(r.flags[i]),
                   int(g["flags"][idx[i]]), float(r.tstar[i])) for i in w]
        raise AssertionError(f"tolerance exceeded: {stats}; (agent, dv, cond, flags_o, flags_g, t*) {detail}")
    return stats
