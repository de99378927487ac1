"""The FP64 autograd reference of the adjoint, pinned to the oracle (CPU).

tests/adjoint_reference.py restates one ORCA step in float64 torch with the
step's discrete choices (neighbours, active set, constructions, waypoint)
taken from the FP64 oracle, and differentiates it with autograd.  Two pins
tie it to the oracle:
  * its forward rollout reproduces the oracle's trajectory (so the closed
    forms of the LP cases and the half-plane constructions are the oracle's
    results, case by case);
  * its gradient of the adjoint benchmark's loss matches central finite
    differences of the oracle's loss, component by component, for the
    preferred-velocity offsets and the waypoints.  Components where the two
    one-sided differences disagree by more than 10 % sit on a kink (an
    active-set or neighbour switch inside +-h) and are reported, not
    compared.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2008_11578_gb300 import scenes
from tests import adjoint_reference as ref


def _scene(side=9.0):
    # dense enough for overlaps, infeasible LPs and every LP case
    return scenes.waypoint_square(n_ped=40, n_veh=6, side=side, n_wp=4, seed=41)


def oracle_rollout(scene, n_steps, delta=None, W=None, record=False):
    sc = scene.copy()
    if W is not None:
        sc.waypoints = np.asarray(W, np.float64)
    pos = sc.pos.astype(np.float64)
    vel = sc.vel.astype(np.float64)
    wpi = None if sc.wp_idx is None else sc.wp_idx.copy()
    vt, recs = [], []
    for t in range(n_steps):
        r = oracle.step(sc, pos=pos, vel=vel, wp_idx=wpi,
                        vpref_delta=None if delta is None else delta[t], want_lines=record)
        if record:
            vp = ref.preferred_velocity_np(sc, pos, r.wp_idx,
                                           None if delta is None else delta[t])
            nl, idx, kind, circ = ref.oracle_frozen(sc, r, r.vel, vp)
            cap, ov = ref.construction_bits(sc, pos, vel, r.nbr, idx, nl)
            recs.append(ref.Frozen(r.nbr, kind, circ, nl, idx, cap, ov, r.wp_idx, r.vel))
        pos, vel = r.pos, r.vel
        wpi = None if wpi is None else r.wp_idx.copy()
        vt.append(vel)
    return pos, np.stack(vt), recs


def reference_grad(scene, n_steps, delta, W, recs):
    d = torch.tensor(delta, dtype=torch.float64, requires_grad=True)
    w = torch.tensor(W, dtype=torch.float64, requires_grad=True)
    p = torch.as_tensor(scene.pos, dtype=torch.float64)
    v = torch.as_tensor(scene.vel, dtype=torch.float64)
    vt = []
    for t in range(n_steps):
        p, v = ref.step(scene, p, v, d[t], w, recs[t])
        vt.append(v)
    L = ref.loss(scene, p, torch.stack(vt))
    L.backward()
    return float(L.detach()), p.detach().numpy(), d.grad.numpy(), w.grad.numpy()


T_STEPS = 6


def test_reference_forward_reproduces_oracle_and_covers_cases():
    s = _scene()
    rng = np.random.default_rng(0)
    delta = rng.normal(0, 0.2, (T_STEPS, s.n, 2))
    W = s.waypoints.astype(np.float64)
    pT, vt, recs = oracle_rollout(s, T_STEPS, delta, W, record=True)
    L, p_ref, _, _ = reference_grad(s, T_STEPS, delta, W, recs)
    assert np.abs(p_ref - pT).max() <= 1e-9
    assert abs(L - ref.loss_np(s, pT, vt)) <= 1e-9 * max(1.0, abs(L))
    cases = set()
    for fz in recs:
        cases |= {(int(k), int(c), int(n)) for k, c, n in zip(fz.kind, fz.circ, fz.nl)}
    # projections onto 0/1/2 lines and least-penetration vertices both occur
    assert {(0, 0, 1), (0, 0, 2)} <= cases
    assert any(k == 1 for k, _, _ in cases), cases


def _components(rng, g, n_nonzero, n_any):
    """Indices of g: some where it is non-zero (where the oracle's loss
    should move), some drawn uniformly (mostly exact zeros: LP results that
    do not depend on the preferred velocity)."""
    nz = np.argwhere(np.abs(g) > 1e-9)
    pick = [tuple(x) for x in nz[rng.permutation(len(nz))[:n_nonzero]]]
    pick += [tuple(int(rng.integers(0, m)) for m in g.shape) for _ in range(n_any)]
    return pick


@pytest.mark.parametrize("side,seed", [(9.0, 0), (16.0, 1)])
def test_reference_gradient_matches_oracle_finite_differences(side, seed):
    s = _scene(side)
    rng = np.random.default_rng(seed)
    delta = rng.normal(0, 0.2, (T_STEPS, s.n, 2))
    W = s.waypoints.astype(np.float64)
    _, _, recs = oracle_rollout(s, T_STEPS, delta, W, record=True)
    _, _, gd, gw = reference_grad(s, T_STEPS, delta, W, recs)
    L0 = ref.loss_np(s, *oracle_rollout(s, T_STEPS, delta, W)[:2])
    h = 1e-5
    comps = [("d", ix) for ix in _components(rng, gd, 20, 8)]
    comps += [("w", ix) for ix in _components(rng, gw, 6, 4)]
    fd, gr, kinks = [], [], 0
    for kind, ix in comps:
        vals = []
        for sgn in (1.0, -1.0):
            d2, W2 = delta.copy(), W.copy()
            (d2 if kind == "d" else W2)[ix] += sgn * h
            vals.append(ref.loss_np(s, *oracle_rollout(s, T_STEPS, d2, W2)[:2]))
        fwd, bwd = (vals[0] - L0) / h, (L0 - vals[1]) / h
        if abs(fwd - bwd) > 0.1 * max(abs(fwd), abs(bwd), 1e-6):
            kinks += 1
            continue
        fd.append((vals[0] - vals[1]) / (2 * h))
        gr.append((gd if kind == "d" else gw)[ix])
    fd, gr = np.array(fd), np.array(gr)
    assert kinks <= 3, kinks
    assert len(fd) >= 30
    assert (np.abs(fd) > 1e-4).sum() >= 15       # most compared components move the loss
    err = np.abs(fd - gr)
    assert (err <= 1e-4 * np.abs(fd) + 2e-6).all(), np.c_[fd, gr][err > 1e-4 * np.abs(fd) + 2e-6]
    assert np.linalg.norm(fd - gr) <= 1e-5 * np.linalg.norm(fd)
