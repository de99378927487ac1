"""The CUDA adjoint of ORCA rollouts (needs a GPU).

* Against the FP64 autograd reference (tests/adjoint_reference.py, itself
  pinned to finite differences of the oracle) along the GPU's own
  trajectory: the GPU steps one at a time recording its states, neighbour
  lists and LP active sets; the reference takes the vector-Jacobian product
  of every step at those states in float64, chained in reverse.  This
  isolates the hand-written adjoint from FP32/FP64 trajectory differences.
* Checkpoint interval and segment boundaries change nothing beyond the
  atomics' summation order; the rollout's forward equals orca_step.
* torch.autograd.Function end to end, and the launch count.
"""
import numpy as np
import pytest
import torch

from paper_2008_11578_gb300 import api, scenes
from paper_2008_11578_gb300.adjoint import Rollout, workload_loss
from tests import adjoint_reference as ref

pytestmark = pytest.mark.gpu


def _cuda_grads(scene, n_steps, ckpt, delta, want_state0=False):
    roll = Rollout(scene, n_steps, ckpt)
    d = torch.as_tensor(delta, dtype=torch.float32, device="cuda").contiguous()
    roll.forward_raw(d)
    pos_T = roll.ds.pos.clone().double().requires_grad_(True)
    vt = roll.vel_traj.clone().double().requires_grad_(True)
    goal = torch.as_tensor(scene.goal, dtype=torch.float64, device="cuda")
    veh = torch.as_tensor(scene.type == 1, device="cuda")
    L = workload_loss(pos_T, vt, goal, veh)
    gp, gv = torch.autograd.grad(L, [pos_T, vt])
    dvpd, dwp, dp0, dv0 = roll.backward_raw(d, gp.float(), gv.float(), want_state0=want_state0)
    torch.cuda.synchronize()
    out = dict(L=float(L.detach()), pos_T=roll.ds.pos.cpu().numpy(), vel_traj=roll.vel_traj.cpu().numpy(),
               dvpd=dvpd.cpu().numpy().astype(np.float64),
               dwp=None if dwp is None else dwp.cpu().numpy().astype(np.float64),
               dp0=None if dp0 is None else dp0.cpu().numpy().astype(np.float64),
               dv0=None if dv0 is None else dv0.cpu().numpy().astype(np.float64),
               launches=api.orca_adjoint_launch_count(roll.ds.handle, n_steps, ckpt))
    roll.close()
    return out


def _gpu_records(scene, n_steps, delta):
    """Step the scene one step at a time on the GPU, recording per step the
    state at its start, neighbours, active sets, waypoint used and result."""
    ds = api.DeviceScene(scene, "cuda")
    ds.enable_debug(active=True)
    recs = []
    for t in range(n_steps):
        p0, v0 = ds.pos.cpu().numpy().copy(), ds.vel.cpu().numpy().copy()
        d = torch.as_tensor(delta[t:t + 1], dtype=torch.float32, device="cuda").contiguous()
        ds.step(1, d)
        torch.cuda.synchronize()
        wp = None if ds.wp_idx is None else ds.wp_idx.cpu().numpy().copy()
        act = ds.dbg["act"].cpu().numpy().view(np.uint32)
        fz = ref.Frozen.from_act(ds.dbg["nbr"].cpu().numpy(), act, wp, ds.vel.cpu().numpy())
        recs.append((p0, v0, fz))
    pos_T = ds.pos.cpu().numpy()
    ds.close()
    return recs, pos_T


def _reference_vjp(scene, recs, pos_T, vel_traj, delta):
    """Reverse chain of per-step float64 VJPs at the recorded GPU states."""
    T = len(recs)
    W = None if scene.waypoints is None else torch.as_tensor(scene.waypoints, dtype=torch.float64)
    pT = torch.as_tensor(pos_T, dtype=torch.float64).requires_grad_(True)
    vt = torch.as_tensor(vel_traj, dtype=torch.float64).requires_grad_(True)
    L = ref.loss(scene, pT, vt)
    gp, gvt = torch.autograd.grad(L, [pT, vt])
    pbar, vbar = gp, torch.zeros_like(gp)
    dd = np.zeros((T, scene.n, 2))
    dW = None if W is None else torch.zeros_like(W)
    for t in range(T - 1, -1, -1):
        p0, v0, fz = recs[t]
        p = torch.as_tensor(p0, dtype=torch.float64).requires_grad_(True)
        v = torch.as_tensor(v0, dtype=torch.float64).requires_grad_(True)
        d = torch.as_tensor(delta[t], dtype=torch.float64).requires_grad_(True)
        w = None if W is None else W.clone().requires_grad_(True)
        p1, v1 = ref.step(scene, p, v, d, w, fz)
        ins = [p, v, d] + ([w] if w is not None else [])
        g = torch.autograd.grad([p1, v1], ins, [pbar, vbar + gvt[t]], allow_unused=True)
        pbar = g[0] if g[0] is not None else torch.zeros_like(p)
        vbar = g[1] if g[1] is not None else torch.zeros_like(v)
        dd[t] = 0.0 if g[2] is None else g[2].numpy()
        if w is not None and g[3] is not None:
            dW = dW + g[3]
    return dict(dvpd=dd, dwp=None if dW is None else dW.numpy(), dp0=pbar.numpy(),
                dv0=vbar.numpy())


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


# k = 16 and 17 straddle the step's constraint order: with up to 16 lines the
# LP takes them sorted by penetration and the recorded active set is mapped
# back through the packed slot permutation, with more only the two most
# violated are moved to the front
@pytest.mark.parametrize("side,n_steps,ckpt,k", [(40.0, 12, 5, 10), (60.0, 10, 4, 10),
                                                 (60.0, 10, 4, 16), (60.0, 10, 4, 17)])
def test_adjoint_matches_fp64_reference_on_gpu_trajectory(side, n_steps, ckpt, k):
    s = scenes.waypoint_square(n_ped=400, n_veh=16, side=side, seed=43)
    s.params.max_neighbors = k
    rng = np.random.default_rng(5)
    delta = rng.normal(0, 0.2, (n_steps, s.n, 2)).astype(np.float32)
    g = _cuda_grads(s, n_steps, ckpt, delta, want_state0=True)
    recs, pos_T = _gpu_records(s, n_steps, delta)
    assert np.array_equal(pos_T, g["pos_T"])          # the rollout is the plain step
    r = _reference_vjp(s, recs, g["pos_T"], g["vel_traj"], delta)
    assert np.linalg.norm(r["dvpd"]) > 0 and np.linalg.norm(r["dwp"]) > 0
    g["dwp"] = g["dwp"].reshape(r["dwp"].shape)
    for key in ("dvpd", "dwp", "dp0", "dv0"):
        e = _rel(g[key], r[key])
        assert e <= 1e-3, (key, e)
        scale = np.abs(r[key]).max()
        assert np.abs(g[key] - r[key]).max() <= 2e-3 * scale + 1e-6, key


def test_checkpoint_interval_changes_nothing():
    s = scenes.waypoint_square(n_ped=600, n_veh=20, side=35.0, seed=44)
    rng = np.random.default_rng(6)
    delta = rng.normal(0, 0.2, (13, s.n, 2)).astype(np.float32)
    base = _cuda_grads(s, 13, 13, delta)
    for k in (1, 4, 8):
        g = _cuda_grads(s, 13, k, delta)
        assert np.array_equal(g["pos_T"], base["pos_T"])
        assert _rel(g["dvpd"], base["dvpd"]) <= 1e-5, k
        assert _rel(g["dwp"], base["dwp"]) <= 1e-5, k
    assert base["launches"] == 3 * 13   # per step: replayed binning + solve, adjoint kernel


def test_autograd_function_end_to_end():
    s = scenes.waypoint_square(n_ped=300, n_veh=12, side=60.0, seed=45)
    T = 9
    roll = Rollout(s, T, 4)
    delta = torch.zeros((T, s.n, 2), device="cuda", requires_grad=True)
    W = torch.as_tensor(s.waypoints, device="cuda").clone().requires_grad_(True)
    goal = torch.as_tensor(s.goal, device="cuda")
    veh = torch.as_tensor(s.type == 1, device="cuda")
    pos_T, vt = roll(delta, W)
    L = workload_loss(pos_T, vt, goal, veh)
    L.backward()
    assert delta.grad.shape == delta.shape and W.grad.shape == W.shape
    assert torch.isfinite(delta.grad).all() and torch.isfinite(W.grad).all()
    assert delta.grad.abs().sum() > 0 and W.grad.abs().sum() > 0
    # same numbers through the raw calls
    g = _cuda_grads(s, T, 4, np.zeros((T, s.n, 2), np.float32))
    assert _rel(delta.grad.cpu().numpy().astype(np.float64), g["dvpd"]) <= 1e-5
    # a second forward invalidates the first graph's checkpoints
    p2, v2 = roll(delta.detach(), W.detach())
    L1 = workload_loss(*roll(delta, W), goal, veh)
    roll(delta.detach(), W.detach())
    with pytest.raises(RuntimeError):
        L1.backward()
    roll.close()


def test_adjoint_argument_checks():
    s = scenes.open_square(200, 20.0, seed=46)
    roll = Rollout(s, 3, 2)
    d = torch.zeros((3, s.n, 2), device="cuda")
    gp = torch.zeros((s.n, 2), device="cuda")
    with pytest.raises(api.OrcaError):            # no rollout yet
        api.orca_adjoint(roll.ds.handle, 3, 2, d, roll.ws, roll.ws_bytes, gp)
    roll.forward_raw(d)
    with pytest.raises(api.OrcaError):            # different checkpoint interval
        api.orca_adjoint(roll.ds.handle, 3, 3, d, roll.ws, roll.ws_bytes, gp)
    with pytest.raises(api.OrcaError):            # waypoint gradient without routes
        api.orca_adjoint(roll.ds.handle, 3, 2, d, roll.ws, roll.ws_bytes, gp,
                         dl_dwaypoints=torch.zeros((4, 2), device="cuda"))
    out = torch.full((3, s.n, 2), 7.0, device="cuda")
    api.orca_adjoint(roll.ds.handle, 3, 2, d, roll.ws, roll.ws_bytes, gp, dl_dvpref_delta=out)
    torch.cuda.synchronize()
    assert (out == 0).all()                        # zero loss gradient -> zero
    roll.close()


def _oracle_loss(scene, n_steps, delta, W):
    import oracle
    sc = scene.copy()
    sc.waypoints = np.asarray(W, np.float64)
    pos, vel, _, traj = oracle.rollout(sc, n_steps, vpref_delta=delta, fp32_state=False)
    return ref.loss_np(sc, pos, np.stack([v for _, v in traj])), pos, traj


def _vjp_chain(scene, states, pos_T, vel_traj, delta):
    """Chain orca_step_vjp backwards along a given trajectory: states[t] =
    (pos, vel, wp_idx) at the start of step t (rounded to FP32 for the GPU)."""
    T = len(states)
    ds = api.DeviceScene(scene, "cuda")
    nb = api.orca_adjoint_workspace_bytes(ds.handle, 1, 1)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    pT = torch.as_tensor(pos_T, dtype=torch.float64).requires_grad_(True)
    vt = torch.as_tensor(np.asarray(vel_traj), dtype=torch.float64).requires_grad_(True)
    gp, gv = torch.autograd.grad(ref.loss(scene, pT, vt), [pT, vt])
    f32 = lambda a: torch.as_tensor(np.asarray(a), dtype=torch.float32, device="cuda").contiguous()
    pbar, vbar = f32(gp), torch.zeros((scene.n, 2), dtype=torch.float32, device="cuda")
    dvpd = np.zeros((T, scene.n, 2))
    dwp = None if ds.waypoints is None else torch.zeros_like(ds.waypoints)
    for t in range(T - 1, -1, -1):
        p, v, wp = states[t]
        wpt = None if wp is None else torch.as_tensor(wp, dtype=torch.uint8, device="cuda")
        dp = torch.empty_like(pbar)
        dv = torch.empty_like(pbar)
        dd = torch.empty_like(pbar)
        api.orca_step_vjp(ds.handle, ws, nb, f32(p), f32(v), wpt, f32(delta[t]), pbar,
                          vbar + f32(gv[t]), dp, dv, dd, dwp)
        pbar, vbar = dp, dv
        dvpd[t] = dd.cpu().numpy()
    torch.cuda.synchronize()
    out = dict(dvpd=dvpd, dwp=None if dwp is None else dwp.cpu().numpy().astype(np.float64),
               dp0=pbar.cpu().numpy(), dv0=vbar.cpu().numpy())
    ds.close()
    return out


def test_step_vjp_chain_equals_orca_adjoint():
    """orca_step_vjp chained along the GPU's own trajectory is orca_adjoint."""
    s = scenes.waypoint_square(n_ped=500, n_veh=16, side=50.0, seed=47)
    T = 11
    rng = np.random.default_rng(8)
    delta = rng.normal(0, 0.2, (T, s.n, 2)).astype(np.float32)
    g = _cuda_grads(s, T, 4, delta, want_state0=True)
    ds = api.DeviceScene(s, "cuda")
    states = []
    for t in range(T):
        states.append((ds.pos.cpu().numpy().copy(), ds.vel.cpu().numpy().copy(),
                       ds.wp_idx.cpu().numpy().copy()))
        ds.step(1, torch.as_tensor(delta[t:t + 1], device="cuda").contiguous())
    ds.close()
    c = _vjp_chain(s, states, g["pos_T"], g["vel_traj"], delta)
    for key in ("dvpd", "dwp", "dp0", "dv0"):
        assert _rel(c[key].reshape(g[key].shape), g[key]) <= 1e-5, key


def test_adjoint_against_oracle_finite_differences_on_the_workload():
    """The adjoint workload at full size (4,000 pedestrians + 64 vehicles with
    8 waypoints each, 100 x 100 m, 40 steps) against central differences of
    the FP64 oracle's loss.

    FP32 and FP64 trajectories of this crowd separate by roughly a factor 10
    every 1.5 steps (neighbour switches and ill-conditioned LP vertices), so
    the two gradients are compared at ONE trajectory, the oracle's: the CUDA
    step VJP is chained along the oracle's states (rounded to FP32).
    Of 510 sampled gradient components, those whose one-sided differences at
    h = 1e-3 agree to 0.1 % are compared (the loss is smooth across the step
    there); the others straddle a kink (an active-set or neighbour switch
    within h) and are counted, not compared.

    The offsets are a small random draw, not zero: at zero every agent that
    heads straight for its goal has |v_pref| exactly equal to its maximum
    speed, i.e. sits on the kink of the speed circle, where the loss has no
    derivative (one side clips, the other does not)."""
    import oracle
    s = scenes.waypoint_square()
    T = 40
    D = np.random.default_rng(11).normal(0.0, 0.05, (T, s.n, 2)).astype(np.float32).astype(np.float64)
    W = s.waypoints.astype(np.float64)
    L0, pT, traj = _oracle_loss(s, T, D, W)
    states, wp = [], s.wp_idx.copy()
    pos, vel = s.pos.astype(np.float64), s.vel.astype(np.float64)
    for t in range(T):
        states.append((pos, vel, wp))
        r = oracle.step(s, pos=pos, vel=vel, wp_idx=wp, vpref_delta=D[t])
        pos, vel, wp = r.pos, r.vel, r.wp_idx.copy()
    c = _vjp_chain(s, states, pT, np.stack([v for _, v in traj]), D.astype(np.float32))
    gW = c["dwp"].reshape(W.shape)
    rng = np.random.default_rng(7)
    comps = []
    for key, arr, nnz, nany in (("d", c["dvpd"], 420, 20), ("w", gW, 60, 10)):
        # nonzero components, taken along a fixed random order of all indices:
        # the float atomics of the chained VJPs add in a run-dependent order,
        # and a component near the threshold that flips then changes one pick,
        # not the whole sample
        walk = [np.unravel_index(f, arr.shape) for f in rng.permutation(arr.size)]
        comps += [(key, tuple(int(q) for q in ix)) for ix in
                  [ix for ix in walk if abs(arr[ix]) > 1e-7][:nnz]]
        comps += [(key, tuple(int(rng.integers(0, m)) for m in arr.shape)) for _ in range(nany)]

    def one_sided(key, ix, h):
        vals = []
        for sg in (1.0, -1.0):
            D2, W2 = D.copy(), W.copy()
            (D2 if key == "d" else W2)[ix] += sg * h
            vals.append(_oracle_loss(s, T, D2, W2)[0])
        return (vals[0] - L0) / h, (L0 - vals[1]) / h

    def compare_at(h, sample, smooth):
        # a component is compared where its two one-sided differences agree
        # to ``smooth`` (relative): the loss is differentiable across the
        # step there; elsewhere an active-set or neighbour switch lies
        # within h and the component is counted as a kink
        fd, gr, kinks = [], [], 0
        for key, ix in sample:
            fwd, bwd = one_sided(key, ix, h)
            if abs(fwd - bwd) > smooth * max(abs(fwd), abs(bwd), 1e-7):
                kinks += 1
                continue
            fd.append(0.5 * (fwd + bwd))
            gr.append((c["dvpd"] if key == "d" else gW)[ix])
        fd, gr = np.array(fd), np.array(gr)
        moving = np.abs(fd) > 1e-6
        pc = np.abs(fd - gr)[moving] / np.abs(fd)[moving]
        return dict(n=len(fd), kinks=kinks, rel=float(np.linalg.norm(fd - gr) / np.linalg.norm(fd)),
                    median=float(np.median(pc)), p90=float(np.quantile(pc, 0.9)),
                    max=float(pc.max()), within_1e3=float((pc <= 1e-3).mean()))

    # the workload's step h = 1e-3; smooth = one-sided differences within 0.1 %
    r3 = compare_at(1e-3, comps, 1e-3)
    print("central differences of the oracle at h = 1e-3 over %d sampled components:" % len(comps),
          r3, "kink fraction %.2f" % (r3["kinks"] / len(comps)))
    # a smaller step on the first 60 components, with the looser 10 % kink test
    r5 = compare_at(1e-5, comps[:60], 0.1)
    print("at h = 1e-5:", r5)
    # the spec bar: the compared gradient within 1e-3 (relative norm) of
    # central differences at h = 1e-3, on at least 100 components
    assert r3["n"] >= 100 and r3["rel"] <= 1e-3, r3
    # the typical component agrees to 1e-4; a few percent of components sit
    # where FP32 and FP64 take opposite sides of a borderline LP decision
    # (feasibility at t* = 0, a line against the speed circle at a
    # near-corner) somewhere along the 40 steps and differ by percent
    assert r3["median"] <= 1e-4 and r3["within_1e3"] >= 0.85, r3
    assert r5["n"] >= 30 and r5["median"] <= 1e-3, r5
