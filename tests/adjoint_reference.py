"""FP64 PyTorch restatement of one ORCA step with its discrete choices held
fixed, differentiated by torch autograd (test infrastructure).

It recomputes, in float64 torch operations, what one step computes for the
agents it is given: the preferred velocity toward the goal or the current
waypoint, the ORCA half-plane of every active neighbour (cut-off circle, leg
or overlap construction), and the LP result written in closed form for the
recorded active set:
  projection, no line         v = v_pref, or vmax v_pref / |v_pref|
  projection, one line        v = P + (d . (v_pref - P)) d
  projection, two lines       the intersection of the two lines
  projection, line + circle   the intersection nearer the recorded result
  vertex, plane + circle      v = vmax n
  vertex, three planes        n_i . v + t = c_i for the three planes
  vertex, two planes + circle their equal-penetration line on the circle
  valley                      v_pref projected onto the equal-penetration line
with n = (-d_y, d_x) and c = det(d, P).  Autograd through this gives the
derivative of the step at fixed neighbours, active sets and branches: the
quantity the CUDA adjoint computes by hand.  The forward of this module is
checked against the FP64 oracle's trajectory, and its gradient against
central finite differences of the oracle (tests/test_adjoint_reference.py).
"""
from __future__ import annotations

import numpy as np
import torch

PROJ, VERTEX, VALLEY = 0, 1, 2


class Frozen:
    """The discrete choices of one step for every agent (numpy arrays)."""

    def __init__(self, nbr, kind, circ, nl, idx, cap, ov, wp_used, vstar):
        self.nbr, self.kind, self.circ, self.nl = nbr, kind, circ, nl
        self.idx, self.cap, self.ov = idx, cap, ov
        self.wp_used, self.vstar = wp_used, vstar

    @staticmethod
    def from_act(nbr, act, wp_used, vstar):
        """From the packed active-set words the CUDA path records."""
        a = np.asarray(act).astype(np.int64) & 0xFFFFFFFF
        kind = a & 3
        circ = (a >> 2) & 1
        nl = (a >> 3) & 3
        idx = np.stack([(a >> (8 + 8 * m)) & 31 for m in range(3)], 1)
        cap = np.stack([(a >> (13 + 8 * m)) & 1 for m in range(3)], 1)
        ov = np.stack([(a >> (14 + 8 * m)) & 1 for m in range(3)], 1)
        return Frozen(np.asarray(nbr), kind, circ, nl, idx, cap.astype(bool), ov.astype(bool),
                      wp_used, np.asarray(vstar, np.float64))


def _cat(*xs):
    return torch.stack(xs, -1)


def _perp_n(d):
    """n = (-d_y, d_x)."""
    return _cat(-d[..., 1], d[..., 0])


def _c(P, d):
    """c = det(d, P) = d_x P_y - d_y P_x."""
    return d[..., 0] * P[..., 1] - d[..., 1] * P[..., 0]


def pair_lines(pa, va, ra, pb, vb, rb, f, tau, dt, cap, ov):
    """ORCA half-planes (P, d) of pairs A|B (float64 tensors, batched);
    cap/ov (bool numpy) select the construction."""
    M = pa.shape[0]
    P = torch.zeros((M, 2), dtype=torch.float64)
    D = torch.zeros((M, 2), dtype=torch.float64)
    q = pb - pa
    wr = va - vb
    rho = ra + rb
    circ = np.asarray(cap) | np.asarray(ov)
    ic = np.nonzero(circ)[0]
    il = np.nonzero(~circ)[0]
    if len(ic):
        T = torch.as_tensor(np.where(np.asarray(ov)[ic], 1.0 / dt, 1.0 / tau),
                            dtype=torch.float64)[:, None]
        w = wr[ic] - q[ic] * T
        wl = torch.sqrt((w ** 2).sum(-1, keepdim=True))
        h = w / wl
        d = _cat(h[:, 1], -h[:, 0])
        u = (rho[ic, None] * T - wl) * h
        P = P.index_put((torch.as_tensor(ic),), va[ic] + f[ic, None] * u)
        D = D.index_put((torch.as_tensor(ic),), d)
    if len(il):
        qq = (q[il] ** 2).sum(-1)
        l = torch.sqrt((qq - rho[il] ** 2).clamp_min(0.0))
        qx, qy = q[il, 0], q[il, 1]
        side = (qx * wr[il, 1] - qy * wr[il, 0]).detach().numpy() > 0
        r_ = rho[il]
        left = _cat((qx * l - qy * r_) / qq, (qx * r_ + qy * l) / qq)
        right = -_cat((qx * l + qy * r_) / qq, (-qx * r_ + qy * l) / qq)
        sd = torch.as_tensor(side)[:, None]
        d = torch.where(sd, left, right)
        pr = (wr[il] * d).sum(-1, keepdim=True)
        u = pr * d - wr[il]
        P = P.index_put((torch.as_tensor(il),), va[il] + f[il, None] * u)
        D = D.index_put((torch.as_tensor(il),), d)
    return P, D


def _nearest(cands, vstar):
    """Pick per row the candidate (list of (M,2) tensors) nearest vstar."""
    dist = torch.stack([((c.detach() - vstar) ** 2).sum(-1) for c in cands], 0)
    k = torch.argmin(dist, 0)
    out = cands[0]
    for j in range(1, len(cands)):
        out = torch.where((k == j)[:, None], cands[j], out)
    return out


def lp_closed_form(kind, circ, nl, lines, vmax, vp, vstar):
    """LP result for agents that share one (kind, circle, line count) case;
    lines[m] = (P, d) of active line m."""
    R = vmax[:, None]
    if kind == PROJ and nl == 0:
        if not circ:
            return vp
        return R * vp / torch.sqrt((vp ** 2).sum(-1, keepdim=True))
    if kind == PROJ and nl == 1 and not circ:
        P, d = lines[0]
        return P + ((vp - P) * d).sum(-1, keepdim=True) * d
    if kind == PROJ and nl == 2:
        (Pa, da), (Pb, db) = lines
        na, nb = _perp_n(da), _perp_n(db)
        ca, cb = _c(Pa, da), _c(Pb, db)
        det = na[:, 0] * nb[:, 1] - na[:, 1] * nb[:, 0]
        x = (ca * nb[:, 1] - cb * na[:, 1]) / det
        y = (na[:, 0] * cb - nb[:, 0] * ca) / det
        return _cat(x, y)
    if kind == PROJ and nl == 1 and circ:
        P, d = lines[0]
        dp = (d * P).sum(-1, keepdim=True)
        h = torch.sqrt(dp ** 2 - (P ** 2).sum(-1, keepdim=True) + R ** 2)
        return _nearest([P + (-dp + h) * d, P + (-dp - h) * d], vstar)
    if kind == VERTEX and nl == 1 and circ:
        return R * _perp_n(lines[0][1])
    if kind == VERTEX and nl == 3:
        rows, rhs = [], []
        for P, d in lines:
            n = _perp_n(d)
            rows.append(torch.cat([n, torch.ones_like(n[:, :1])], -1))
            rhs.append(_c(P, d))
        A = torch.stack(rows, 1)
        b = torch.stack(rhs, 1)
        z = torch.linalg.solve(A, b)
        return z[:, :2]
    if kind in (VERTEX, VALLEY) and nl == 2:
        (Pa, da), (Pb, db) = lines
        a = _perp_n(db) - _perp_n(da)
        beta = _c(Pb, db) - _c(Pa, da)
        a2 = (a ** 2).sum(-1, keepdim=True)
        if kind == VALLEY:
            return vp + (beta[:, None] - (a * vp).sum(-1, keepdim=True)) / a2 * a
        x0 = a * beta[:, None] / a2
        e = _cat(a[:, 1], -a[:, 0]) / torch.sqrt(a2)
        h = torch.sqrt(R ** 2 - (x0 ** 2).sum(-1, keepdim=True))
        return _nearest([x0 + h * e, x0 - h * e], vstar)
    raise ValueError(f"no closed form for kind={kind} circle={circ} lines={nl}")


def step(scene, p, v, delta, W, fz: Frozen):
    """One step for all agents: returns (p_next, v_next) as float64 tensors.

    p, v, delta: (N, 2) float64 tensors; W: (R, n_wp, 2) float64 tensor or
    None; fz: the step's frozen choices.  Agents whose case has no closed
    form raise ValueError.
    """
    prm = scene.params
    N = p.shape[0]
    tau, dt = float(np.float32(prm.time_horizon)), float(np.float32(prm.dt))
    vmax = torch.as_tensor(scene.max_speed, dtype=torch.float64)
    rad = torch.as_tensor(scene.radius, dtype=torch.float64)
    typ = np.asarray(scene.type, np.int64)
    fT = np.asarray(prm.f, np.float64).reshape(2, 2)
    g = torch.as_tensor(scene.goal, dtype=torch.float64)
    if scene.route is not None and W is not None:
        rt = np.asarray(scene.route)
        routed = np.nonzero(rt >= 0)[0]
        if len(routed):
            gw = W[rt[routed], fz.wp_used[routed].astype(np.int64)]
            g = g.index_put((torch.as_tensor(routed),), gw)
    e = g - p
    e2 = (e ** 2).sum(-1)
    ok = e2.detach() > 0
    # an agent exactly at its goal has v_pref = delta (no direction to differentiate)
    gls = torch.sqrt(torch.where(ok, e2, torch.ones_like(e2)))
    speed_cap = (vmax / gls) < (1.0 / dt)
    sc = torch.where(speed_cap, vmax / gls, torch.full_like(gls, 1.0 / dt))
    vp = torch.where(ok[:, None], e * sc[:, None], torch.zeros_like(e)) + delta

    vstar = torch.as_tensor(fz.vstar, dtype=torch.float64)
    vnew = torch.zeros((N, 2), dtype=torch.float64)
    keys = np.stack([fz.kind, fz.circ, fz.nl], 1)
    for key in np.unique(keys, axis=0):
        kind, circ, nl = (int(x) for x in key)
        sel = np.nonzero((keys == key).all(1))[0]
        ts = torch.as_tensor(sel)
        lines = []
        for m in range(nl):
            j = fz.nbr[sel, fz.idx[sel, m]].astype(np.int64)
            f = torch.as_tensor(fT[typ[sel], typ[j]], dtype=torch.float64)
            lines.append(pair_lines(p[ts], v[ts], rad[ts], p[j], v[j], rad[j], f, tau, dt,
                                    fz.cap[sel, m], fz.ov[sel, m]))
        vs = lp_closed_form(kind, bool(circ), nl, lines, vmax[ts], vp[ts], vstar[ts])
        vnew = vnew.index_put((ts,), vs)
    return p + dt * vnew, vnew


def _boundary_rows(L, idx, v, with_t):
    """Rows dF/dz of the chosen boundaries at v (z = v or (v, t))."""
    rows = []
    for i in idx:
        d = L[i, 2:]
        rows.append([d[1], -d[0]] + ([-1.0] if with_t else []))
    return rows


def _pick(L, S, circ_ok, v, need, with_t):
    """Best-conditioned set of `need` boundaries (lines in S, optionally the
    circle) that determines v: max |det| of the normalised rows."""
    import itertools
    opts = [("l", i) for i in S] + ([("c", -1)] if circ_ok else [])
    best, best_det = None, -1.0
    for comb in itertools.combinations(opts, need):
        rows = []
        for kind, i in comb:
            if kind == "l":
                r = _boundary_rows(L, [i], v, with_t)[0]
            else:
                r = [v[0], v[1]] + ([0.0] if with_t else [])
            r = np.asarray(r, np.float64)
            rows.append(r / np.linalg.norm(r))
        dt_ = abs(np.linalg.det(np.stack(rows)))
        if dt_ > best_det:
            best, best_det = comb, dt_
    if best is None or best_det < 1e-6:
        return None
    lines = [i for kind, i in best if kind == "l"]
    return lines, any(kind == "c" for kind, _ in best)


def oracle_frozen(scene, res, vstar, vpref):
    """Frozen choices of one oracle step (oracle.StepResult with lines).

    The oracle reports every boundary active at its result (mask, circle
    flag).  When more are active than the result needs (e.g. the half-planes
    of f = 0 pairs, which all pass through the agent's own velocity and meet
    at one apex), the best-conditioned determining subset is used; at such
    points the derivative does not depend on the choice."""
    n = scene.n
    mask = res.mask.astype(np.int64)
    infeas = (res.flags & 1) != 0
    on_circ = ((res.flags >> 3) & 1) != 0
    nl = np.zeros(n, np.int64)
    idx = np.zeros((n, 3), np.int64)
    kind = np.where(infeas, VERTEX, PROJ).astype(np.int64)
    circ = np.zeros(n, np.int64)
    vmax = np.asarray(scene.max_speed, np.float64)
    for i in range(n):
        S = [b for b in range(32) if (mask[i] >> b) & 1]
        L = res.lines[i]
        v = vstar[i]
        vp = vpref[i]
        tol = 1e-8 * (1.0 + vmax[i])
        chosen = None
        if not infeas[i]:
            if np.linalg.norm(v - vp) <= tol:
                chosen = ([], False)
            elif on_circ[i] and np.linalg.norm(v - vmax[i] * vp / np.linalg.norm(vp)) <= tol:
                chosen = ([], True)
            else:
                for a in S:
                    P, d = L[a, :2], L[a, 2:]
                    if np.linalg.norm(P + ((vp - P) @ d) * d - v) <= tol:
                        chosen = ([a], False)
                        break
                if chosen is None:
                    chosen = _pick(L, S, on_circ[i], v, 2, False)
        else:
            if len(S) >= 2:
                for a in S:
                    for b in S:
                        if b <= a:
                            continue
                        da, db = L[a, 2:], L[b, 2:]
                        if da @ db < 0 and abs(da[0] * db[1] - da[1] * db[0]) < 1e-9:
                            nA = np.array([-da[1], da[0]])
                            nB = np.array([-db[1], db[0]])
                            av = nB - nA
                            beta = (db[0] * L[b, 1] - db[1] * L[b, 0]) - \
                                   (da[0] * L[a, 1] - da[1] * L[a, 0])
                            pv = vp + (beta - av @ vp) / (av @ av) * av
                            if np.linalg.norm(pv - v) <= tol:
                                chosen = ([a, b], False)
                                kind[i] = VALLEY
            if chosen is None and on_circ[i]:
                for a in S:
                    if np.linalg.norm(vmax[i] * np.array([-L[a, 3], L[a, 2]]) - v) <= tol:
                        chosen = ([a], True)
                        break
            if chosen is None:
                chosen = _pick(L, S, on_circ[i], v, 3, True)
        if chosen is None:
            raise ValueError(f"agent {i}: no determining set of active boundaries")
        lines, c = chosen
        nl[i] = len(lines)
        idx[i, :len(lines)] = lines
        circ[i] = int(c)
    return nl, idx, kind, circ


def construction_bits(scene, pos, vel, nbr, idx, nl):
    """Overlap (FP32 key test) and cut-off (FP64) flags of the active lines."""
    prm = scene.params
    tau = float(np.float32(prm.time_horizon))
    n = scene.n
    cap = np.zeros((n, 3), bool)
    ov = np.zeros((n, 3), bool)
    p32 = pos.astype(np.float32)
    for i in range(n):
        for m in range(int(nl[i])):
            j = int(nbr[i, idx[i, m]])
            dx = np.float32(p32[j, 0] - p32[i, 0])
            dy = np.float32(p32[j, 1] - p32[i, 1])
            d2 = np.float32(np.float32(dx * dx) + np.float32(dy * dy))
            rs = np.float32(np.float32(scene.radius[i]) + np.float32(scene.radius[j]))
            ov[i, m] = d2 <= np.float32(rs * rs)
            if not ov[i, m]:
                q = pos[j] - pos[i]
                w = (vel[i] - vel[j]) - q / tau
                rho = float(scene.radius[i]) + float(scene.radius[j])
                wq = w @ q
                cap[i, m] = wq < 0 and wq * wq > rho * rho * (w @ w)
    return cap, ov


def preferred_velocity_np(scene, pos, wp_used, delta=None):
    """v_pref of every agent (FP64 numpy, the step's formula)."""
    g = scene.goal.astype(np.float64).copy()
    if scene.route is not None:
        rt = np.asarray(scene.route)
        r = np.nonzero(rt >= 0)[0]
        g[r] = np.asarray(scene.waypoints, np.float64)[rt[r], np.asarray(wp_used)[r]]
    dt = float(np.float32(scene.params.dt))
    e = g - pos
    gl = np.sqrt((e ** 2).sum(1))
    with np.errstate(divide="ignore", invalid="ignore"):
        sc = np.minimum(scene.max_speed.astype(np.float64) / gl, 1.0 / dt)
    vp = np.where((gl > 0)[:, None], e * sc[:, None], 0.0)
    return vp if delta is None else vp + delta


def loss(scene, pos_T, vel_traj, target_speed=5.0, weight=0.1):
    """The adjoint benchmark's loss on float64 tensors."""
    goal = torch.as_tensor(scene.goal, dtype=torch.float64)
    veh = torch.as_tensor(np.asarray(scene.type) == 1)
    term = ((pos_T - goal) ** 2).sum(-1).mean()
    # a vehicle held at zero speed (an apex of f = 0 half-planes) has no
    # speed direction; its speed term then contributes no gradient
    sp = torch.sqrt((vel_traj[:, veh] ** 2).sum(-1).clamp_min(1e-30))
    return term + weight * ((sp - target_speed) ** 2).sum()


def loss_np(scene, pos_T, vel_traj, target_speed=5.0, weight=0.1):
    veh = np.asarray(scene.type) == 1
    term = ((pos_T - scene.goal.astype(np.float64)) ** 2).sum(-1).mean()
    sp = np.sqrt((np.asarray(vel_traj)[:, veh] ** 2).sum(-1))
    return float(term + weight * ((sp - target_speed) ** 2).sum())
