"""Pins of the FP64 oracle to things other than itself (CPU only).

Each test ties one part of the oracle to an independent fact: a KKT
certificate, a dense grid search, scipy's QP/LP solvers, the head-on closed
form of the ORCA construction, the velocity-obstacle geometry sampled by brute
force, the collision-free guarantee of reciprocal avoidance (Sec. 3.1), a
kd-tree neighbour query, and exact symmetries.  A dropped term, a wrong sign,
a swapped leg or a transposed operand in the oracle fails one of them.
"""
import math

import numpy as np
import pytest
from scipy.optimize import linprog, minimize, nnls
from scipy.spatial import cKDTree

import oracle
from paper_2008_11578_gb300 import scenes


def _rand_lines(rng, n, spread=1.0):
    th = rng.uniform(0, 2 * np.pi, n)
    d = np.stack([np.cos(th), np.sin(th)], 1)
    P = rng.normal(0, spread, (n, 2))
    return np.concatenate([P, d], 1)


def _pen(lines, v):
    """det(d, P - v) for every line (positive = violated)."""
    P, d = lines[:, :2], lines[:, 2:]
    return d[:, 0] * (P[:, 1] - v[1]) - d[:, 1] * (P[:, 0] - v[0])


# ---------------------------------------------------------------- 2D LP -----

def test_lp_kkt_certificate():
    """Feasible LPs: v* is feasible and v_pref - v* lies in the normal cone of
    the active boundaries with non-negative multipliers (KKT, sufficient for a
    convex projection)."""
    rng = np.random.default_rng(10)
    checked = 0
    for _ in range(3000):
        n = int(rng.integers(0, 11))
        lines = _rand_lines(rng, n, 1.0)
        vmax = rng.uniform(0.5, 3.0)
        vp = rng.normal(0, 2.0, 2)
        v, ts, fl, cond, mask = oracle.lp(lines, vmax, vp)
        if fl & 1:
            continue
        assert not (fl & 2)
        assert np.linalg.norm(v) <= vmax * (1 + 1e-9)
        if n:
            assert _pen(lines, v).max() <= 1e-9
        cols = []
        for i in range(n):
            if abs(_pen(lines[i:i + 1], v)[0]) <= 1e-8:
                # gradient of the violated side is -n_i, n = (-d_y, d_x)
                cols.append(np.array([lines[i, 3], -lines[i, 2]]))
        if abs(np.linalg.norm(v) - vmax) <= 1e-8:
            cols.append(v.copy())
        r = vp - v
        if not cols:
            assert np.linalg.norm(r) <= 1e-9
        else:
            A = -np.stack(cols, 1)
            lam, res = nnls(A, -r)
            assert res <= 1e-7 * (1 + np.linalg.norm(r)), (n, res)
        checked += 1
    assert checked > 1000


def test_lp_dense_grid_bruteforce():
    """Tiny LPs against a dense grid search over the disc."""
    rng = np.random.default_rng(11)
    g = np.linspace(-1, 1, 1201)
    X, Y = np.meshgrid(g, g)
    for _ in range(40):
        n = int(rng.integers(1, 5))
        lines = _rand_lines(rng, n, 0.6)
        vmax = 1.0
        vp = rng.normal(0, 1.0, 2)
        v, ts, fl, _, _ = oracle.lp(lines, vmax, vp)
        if fl & 1:
            continue
        ok = X ** 2 + Y ** 2 <= vmax ** 2
        for L in lines:
            ok &= L[2] * (L[1] - Y) - L[3] * (L[0] - X) <= 0
        if ok.sum() < 10:
            continue
        dist = (X - vp[0]) ** 2 + (Y - vp[1]) ** 2
        dist[~ok] = np.inf
        j = np.unravel_index(np.argmin(dist), dist.shape)
        h = g[1] - g[0]
        fstar = (v[0] - vp[0]) ** 2 + (v[1] - vp[1]) ** 2
        assert fstar <= dist[j] + 1e-12
        # strong convexity: |v_grid - v*|^2 <= f(v_grid) - f(v*)
        assert math.hypot(X[j] - v[0], Y[j] - v[1]) <= 3 * h + math.sqrt(max(dist[j] - fstar, 0))


def test_lp_scipy_slsqp():
    rng = np.random.default_rng(12)
    n_cmp = 0
    for _ in range(150):
        n = int(rng.integers(1, 11))
        lines = _rand_lines(rng, n, 1.0)
        vmax = rng.uniform(1.0, 3.0)
        vp = rng.normal(0, 2.0, 2)
        v, ts, fl, cond, _ = oracle.lp(lines, vmax, vp)
        if fl & 1 or cond > 1e3:
            continue
        cons = [{"type": "ineq", "fun": lambda x, L=L: -(L[2] * (L[1] - x[1]) - L[3] * (L[0] - x[0]))}
                for L in lines]
        cons.append({"type": "ineq", "fun": lambda x: vmax ** 2 - x @ x})
        best = None
        for x0 in (np.zeros(2), v + 0.01):
            r = minimize(lambda x: ((x - vp) ** 2).sum(), x0, method="SLSQP",
                         constraints=cons, options=dict(ftol=1e-14, maxiter=500))
            if r.success and (best is None or r.fun < best.fun):
                best = r
        if best is None:
            continue
        assert np.abs(best.x - v).max() <= 1e-5, (best.x, v)
        n_cmp += 1
    assert n_cmp > 50


# ------------------------------------------------------ 3D LP fallback ------

def _tstar_linprog(lines, vmax, m=1440):
    """min t s.t. det(d_i, P_i - v) <= t and v in the circumscribed m-gon."""
    A, b = [], []
    for L in lines:
        # c - n.v - t <= 0  with c = det(d, P), n = (-d_y, d_x)
        c = L[2] * L[1] - L[3] * L[0]
        A.append([L[3], -L[2], -1.0])
        b.append(-c)
    R = vmax / math.cos(math.pi / m)
    for j in range(m):
        a = 2 * math.pi * j / m
        A.append([math.cos(a), math.sin(a), 0.0])
        b.append(vmax)
    r = linprog([0, 0, 1], A_ub=np.array(A), b_ub=np.array(b),
                bounds=[(-R, R), (-R, R), (None, None)], method="highs")
    assert r.status == 0
    return r.fun


def test_tstar_against_linprog():
    """Least penetration t* of infeasible sets against an LP over a fine polygon
    sandwiching the disc (error <= vmax * (1/cos(pi/m) - 1))."""
    rng = np.random.default_rng(13)
    seen = 0
    for _ in range(400):
        n = int(rng.integers(3, 11))
        lines = _rand_lines(rng, n, 0.3)
        # move every line 1.5 along its admissible normal n = (-d_y, d_x),
        # so the admissible sides face away from each other
        lines[:, :2] += 1.5 * np.stack([-lines[:, 3], lines[:, 2]], 1)
        vmax = 1.0
        v, ts, fl, _, _ = oracle.lp(lines, vmax, np.zeros(2))
        if not (fl & 1):
            continue
        lp_t = _tstar_linprog(lines, vmax)
        # the polygon contains the disc: lp_t <= ts; its excess is bounded
        assert lp_t <= ts + 1e-9
        assert ts - lp_t <= vmax * (1 / math.cos(math.pi / 1440) - 1) * 2 + 1e-9
        # the returned velocity attains t*
        assert abs(_pen(lines, v).max() - ts) <= 1e-8
        seen += 1
    assert seen > 100


def test_tstar_valley_tie_break():
    """Two opposite parallel lines that cannot both hold: every point of the
    mid-line is a minimiser, and the tie-break picks the one closest to v_pref."""
    # admissible side is left of d: line 1 (d = +x) admits y >= 0.4,
    # line 2 (d = -x) admits y <= -0.4
    lines = np.array([[0.0, 0.4, 1.0, 0.0], [0.0, -0.4, -1.0, 0.0]])
    vmax = 2.0
    for vp in ([1.0, 0.7], [-0.3, -1.2], [3.0, 0.0], [0.0, 0.0]):
        v, ts, fl, _, _ = oracle.lp(lines, vmax, np.array(vp))
        assert fl & 1
        assert abs(ts - 0.4) <= 1e-12
        # projection of vp onto the segment {y = 0, |x| <= vmax}
        assert abs(v[1]) <= 1e-12
        assert abs(v[0] - np.clip(vp[0], -vmax, vmax)) <= 1e-12


def test_tstar_three_lines_triangle():
    """Three lines bounding an inverted triangle: t* is the inradius-type
    minimax of an equilateral arrangement, attained at its centre."""
    # admissible sides point outward from the origin, distance a from it
    a = 0.5
    lines = []
    for k in range(3):
        th = 2 * np.pi * k / 3
        nrm = np.array([np.cos(th), np.sin(th)])      # admissible direction
        d = np.array([nrm[1], -nrm[0]])               # left normal of d is nrm
        lines.append([*(a * nrm), *d])
    v, ts, fl, cond, _ = oracle.lp(np.array(lines), 3.0, np.array([0.2, 0.1]))
    assert fl & 1
    assert abs(ts - a) <= 1e-12
    assert np.abs(v).max() <= 1e-12
    # all three planes attain t*; any two of them meet at 120 degrees
    assert abs(cond - 1.0 / math.sin(2 * math.pi / 3)) <= 1e-12


# ------------------------------------------- active-set conditioning -------
# The oracle reports, per agent, the condition number of the active set at
# its LP result: 1 / sin of the angle between the best-conditioned pair of
# active boundaries (lines, or a line and the speed circle's tangent), and 1
# when fewer than two boundaries are active.  The tests use it to decide
# which agents are ill-conditioned, so its value is pinned by closed forms.

@pytest.mark.parametrize("phi", [math.pi / 6, math.pi / 3, math.pi / 2, 2 * math.pi / 3,
                                 5 * math.pi / 6])
def test_active_cond_two_lines_at_a_known_angle(phi):
    """Two half-planes through the origin whose inward normals n_A, n_B meet
    at angle phi; v_pref = -(n_A + n_B) lies in the normal cone of the apex,
    so the result is the apex and the condition number is 1 / sin(phi)."""
    nA = np.array([0.0, 1.0])
    nB = np.array([-math.sin(phi), math.cos(phi)])
    # left normal of d is n: d = (n_y, -n_x)
    lines = np.array([[0.0, 0.0, nA[1], -nA[0]], [0.0, 0.0, nB[1], -nB[0]]])
    v, ts, fl, cond, mask = oracle.lp(lines, 3.0, -(nA + nB))
    assert fl & 1 == 0
    assert np.abs(v).max() <= 1e-12
    assert mask == 0b11
    assert abs(cond - 1.0 / math.sin(phi)) <= 1e-9 / math.sin(phi)


@pytest.mark.parametrize("h", [0.25, 1.0, 1.9])
def test_active_cond_line_against_speed_circle(h):
    """The half-plane y <= h cut by the speed circle |v| = R: at the corner
    v* = (sqrt(R^2 - h^2), h) the line's direction makes an angle with the
    circle's tangent whose sine is |d . v*| / R, so the condition number is
    R / sqrt(R^2 - h^2).  v_pref = v* + (0, 1) + v*/R has positive
    multipliers on both boundaries (KKT), so v* is the projection."""
    R = 2.0
    vs = np.array([math.sqrt(R * R - h * h), h])
    lines = np.array([[0.0, h, -1.0, 0.0]])          # admissible side: y <= h
    v, ts, fl, cond, mask = oracle.lp(lines, R, vs + np.array([0.0, 1.0]) + vs / R)
    assert fl & 1 == 0
    assert np.abs(v - vs).max() <= 1e-12
    assert fl & 8                                      # on the speed circle
    assert abs(cond - R / math.sqrt(R * R - h * h)) <= 1e-9 * cond


def test_active_cond_single_boundary_is_one():
    """One active line inside the disc, or the circle alone: cond = 1."""
    lines = np.array([[0.0, 0.5, -1.0, 0.0]])         # y <= 0.5
    v, _, fl, cond, mask = oracle.lp(lines, 3.0, np.array([0.3, 1.0]))
    assert np.abs(v - [0.3, 0.5]).max() <= 1e-12 and mask == 1 and cond == 1.0
    v, _, fl, cond, mask = oracle.lp(np.zeros((0, 4)), 1.5, np.array([3.0, 4.0]))
    assert np.abs(v - [0.9, 1.2]).max() <= 1e-12 and fl & 8 and cond == 1.0


# ------------------------------------------------------- ORCA lines ---------

def _two_agent_scene(pa, va, pb, vb, ra=0.5, rb=0.5, vmax=(1.5, 1.5), types=(0, 0),
                     goals=None, f=None, tau=5.0, dt=0.25):
    pos = np.array([pa, pb], np.float32)
    vel = np.array([va, vb], np.float32)
    if goals is None:
        goals = [np.array(pa) + 1000 * np.array(va) / max(np.linalg.norm(va), 1e-9),
                 np.array(pb) + 1000 * np.array(vb) / max(np.linalg.norm(vb), 1e-9)]
    p = scenes.OrcaParams(time_horizon=tau, dt=dt, max_neighbors=10)
    if f is not None:
        p.f = f
    s = scenes.Scene(pos, vel, np.array(goals, np.float32), np.array([ra, rb], np.float32),
                     np.array(vmax, np.float32), np.array(types, np.uint8), p)
    return s


@pytest.mark.parametrize("fa,fb", [(0.5, 0.5), (1.0, 0.0), (0.0, 1.0), (0.25, 0.75), (0.7, 0.3)])
def test_headon_cap_closed_form(fa, fb):
    """Head-on pair on the x axis, v_pref = current velocity, cut-off branch:
    v_A,new = s_A + f_A ((D - rho)/tau - (s_A + s_B)) along the axis."""
    sA, sB, D, rho, tau = 1.5, 1.0, 5.5, 1.0, 2.0
    assert D - rho < (sA + sB) * tau < D < 10.0
    s = _two_agent_scene([0, 0], [sA, 0], [D, 0], [-sB, 0], vmax=(sA, sB),
                         types=(0, 1), f=((0.5, fa), (fb, 0.5)), tau=tau)
    r = oracle.step(s)
    S = sA + sB
    vA = sA + fa * ((D - rho) / tau - S)
    vB = -(sB + fb * ((D - rho) / tau - S))
    assert abs(r.vel[0, 0] - vA) <= 1e-12 and abs(r.vel[0, 1]) <= 1e-12
    assert abs(r.vel[1, 0] - vB) <= 1e-12 and abs(r.vel[1, 1]) <= 1e-12
    if fa == fb == 0.5 and sA == sB:
        assert abs(vA - (D - rho) / (2 * tau)) <= 1e-12


def test_headon_symmetric_half():
    s_, D, rho, tau = 1.0, 8.5, 1.0, 4.0
    assert D - rho < 2 * s_ * tau < D
    s = _two_agent_scene([0, 0], [s_, 0], [D, 0], [-s_, 0], vmax=(s_, s_), tau=tau)
    r = oracle.step(s)
    assert abs(r.vel[0, 0] - (D - rho) / (2 * tau)) <= 1e-12
    assert abs(r.vel[1, 0] + (D - rho) / (2 * tau)) <= 1e-12


def test_headon_leg_tie_goes_right():
    """(s_A + s_B) tau >= D: leg branch; the exactly collinear input is the
    det = 0 tie, which takes the right leg, so each agent veers to its right."""
    sA = sB = 1.5
    D, rho, tau, f = 4.0, 1.0, 5.0, 0.5
    s = _two_agent_scene([0, 0], [sA, 0], [D, 0], [-sB, 0], vmax=(sA, sB))
    r = oracle.step(s)
    S = sA + sB
    ell = math.sqrt(D * D - rho * rho)
    # projection of v_pref onto the right-leg half-plane through v_A + f u
    vx = sA - f * S * rho ** 2 / D ** 2
    vy = -f * S * rho * ell / D ** 2
    assert abs(r.vel[0, 0] - vx) <= 1e-12 and abs(r.vel[0, 1] - vy) <= 1e-12
    # B mirrors A (its right is +y in world coordinates)
    assert abs(r.vel[1, 0] + vx) <= 1e-12 and abs(r.vel[1, 1] + vy) <= 1e-12


def _vo_boundary(q, rho, tau, m=200000):
    """Dense samples of the truncated cone's boundary (legs + cut-off arc)."""
    ql = np.linalg.norm(q)
    c = q / tau
    rc = rho / tau
    ang = math.asin(min(rho / ql, 1.0))
    base = math.atan2(q[1], q[0])
    pts = []
    ell = math.sqrt(max(ql * ql - rho * rho, 0.0))
    for sgn in (1, -1):
        dirv = np.array([math.cos(base + sgn * ang), math.sin(base + sgn * ang)])
        t0 = ell / tau   # tangent point distance on the cut-off circle
        tt = np.linspace(t0, t0 + 50.0, m)
        pts.append(tt[:, None] * dirv[None, :])
    # the arc facing the origin between the two tangent points
    a = np.linspace(0, 2 * np.pi, m)
    arc = c[None, :] + rc * np.stack([np.cos(a), np.sin(a)], 1)
    toward = (arc - c) @ (-q / ql) >= rc * math.cos(math.pi / 2 - ang) - 1e-12
    pts.append(arc[toward])
    return np.concatenate(pts)


def _in_vo(v, q, rho, tau):
    """v is in the truncated velocity obstacle iff |t v - q| <= rho for some
    t in (0, tau]."""
    vv = v @ v
    t = tau if vv == 0 else min(max((v @ q) / vv, 1e-12), tau)
    return np.linalg.norm(t * v - q) <= rho


def test_u_is_shortest_vector_to_vo_boundary():
    """u from the oracle equals the brute-force closest boundary point of the
    truncated velocity obstacle minus w_rel (f = 1 exposes u directly)."""
    rng = np.random.default_rng(14)
    tau, dt = 5.0, 0.25
    for _ in range(60):
        q = rng.uniform(-6, 6, 2)
        ra, rb = 0.5, rng.choice([0.5, 1.5])
        rho = ra + rb
        if np.linalg.norm(q) <= rho * 1.05:
            continue
        va = rng.uniform(-2, 2, 2)
        vb = rng.uniform(-2, 2, 2)
        L = oracle.pair_line([0, 0], va, ra, q, vb, rb, 1.0, tau, dt, False)
        u = L[:2] - va
        wrel = va - vb
        B = _vo_boundary(q, rho, tau)
        j = np.argmin(((B - wrel) ** 2).sum(1))
        u_bf = B[j] - wrel
        assert np.linalg.norm(u - u_bf) <= 2e-3, (u, u_bf)
        # the admissible side (left of d) faces away from the obstacle
        d = L[2:]
        nrm = np.array([-d[1], d[0]])
        c = wrel + u
        assert _in_vo(c - 1e-3 * nrm, q, rho, tau)
        assert not _in_vo(c + 1e-3 * nrm, q, rho, tau)
        assert abs(np.linalg.norm(d) - 1.0) <= 1e-12


def test_leg_tangency_and_cap_circle():
    rng = np.random.default_rng(15)
    tau, dt = 5.0, 0.25
    n_leg = n_cap = 0
    for _ in range(2000):
        q = rng.uniform(-8, 8, 2)
        rho = 1.0
        if np.linalg.norm(q) <= 1.05 * rho:
            continue
        va, vb = rng.uniform(-2, 2, 2), rng.uniform(-2, 2, 2)
        L = oracle.pair_line([0, 0], va, 0.5, q, vb, 0.5, 1.0, tau, dt, False)
        u, d = L[:2] - va, L[2:]
        wrel = va - vb
        x = wrel + u
        w = wrel - q / tau
        cap = (w @ q < 0) and (w @ q) ** 2 > rho ** 2 * (w @ w)
        if cap:
            # closest point is on the cut-off circle
            assert abs(np.linalg.norm(x - q / tau) - rho / tau) <= 1e-12
            n_cap += 1
        else:
            # closest point is on a leg through the origin, along d
            assert abs(d[0] * x[1] - d[1] * x[0]) <= 1e-12
            # the leg is tangent to D(q, rho): distance from q to the line = rho
            assert abs(abs(d[0] * q[1] - d[1] * q[0]) - rho) <= 1e-12
            n_leg += 1
    assert n_leg > 100 and n_cap > 100


def test_cap_leg_switch_is_continuous():
    """Sweeping w_rel across the cap/leg boundary moves the line continuously."""
    q = np.array([4.0, 0.0])
    rho, tau = 1.0, 5.0
    ell = math.sqrt(16 - 1)
    # tangent point on the upper leg at the cut-off: (ell/tau) * leg direction
    leg = np.array([ell, rho]) / 4.0
    tp = (ell / tau) * leg
    # walk along the circle's outward normal at the tangent point
    nrm = tp - q / tau
    nrm /= np.linalg.norm(nrm)
    tang = np.array([-nrm[1], nrm[0]])
    prev = None
    for s in np.linspace(-1e-3, 1e-3, 401):
        wrel = tp + 0.3 * nrm + s * tang
        L = oracle.pair_line([0, 0], wrel, 0.5, q, [0, 0], 0.5, 0.5, tau, 0.25, False)
        if prev is not None:
            assert np.abs(L - prev).max() <= 1e-4
        prev = L


def test_overlap_pair_separates_in_one_step():
    """Overlapping pair, no other constraint binding: with f = 1/2 each, the
    pair's relative velocity points apart at the rate that clears the overlap
    within dt (the overlap construction replaces tau by dt)."""
    s = _two_agent_scene([0, 0], [0, 0], [0.625, 0], [0, 0], vmax=(5.0, 5.0))
    s.goal[:] = s.pos  # v_pref = 0
    r = oracle.step(s)
    # each moves (rho - D)/(2 dt) apart
    sep = (1.0 - 0.625) / (2 * 0.25)
    assert abs(r.vel[0, 0] + sep) <= 1e-12 and abs(r.vel[1, 0] - sep) <= 1e-12
    newd = r.pos[1, 0] - r.pos[0, 0]
    assert abs(newd - 1.0) <= 1e-12


# ------------------------------------------------ preferred velocity --------

def test_lone_agent_preferred_velocity():
    s = _two_agent_scene([0, 0], [0, 0], [100, 100], [0, 0], vmax=(1.5, 1.5))
    s.goal = np.array([[30.0, 40.0], [100.1, 100.0]], np.float32)
    r = oracle.step(s)
    assert np.allclose(r.vel[0], [0.9, 1.2], atol=1e-12)       # 1.5 toward (3,4)/5
    # goal within vmax*dt: lands exactly on it (no overshoot)
    assert np.allclose(r.pos[1], [100.1, 100.0], atol=1e-12)


def test_waypoints_followed_in_order():
    wps = np.array([[[5.0, 0.0], [5.0, 5.0], [0.0, 5.0]]], np.float32)
    p = scenes.OrcaParams()
    s = scenes.Scene(np.array([[0.0, 0.0]], np.float32), np.zeros((1, 2), np.float32),
                     np.array([[0.0, 5.0]], np.float32), np.array([1.5], np.float32),
                     np.array([5.0], np.float32), np.array([1], np.uint8), p,
                     np.array([0], np.int32), wps, np.zeros(1, np.uint8))
    pos, vel, wpi, traj = oracle.rollout(s, 20, fp32_state=False)
    seq = [int(x[0]) for x in [wpi]]
    assert seq[-1] == 2
    assert np.linalg.norm(pos[0] - [0.0, 5.0]) <= 1e-9


def _routed_vehicle(wps, wp_idx, r=0.5, vmax=5.0):
    wps = np.asarray(wps, np.float32).reshape(1, -1, 2)
    return scenes.Scene(np.array([[0.0, 0.0]], np.float32), np.zeros((1, 2), np.float32),
                        wps[0, -1:, :].copy(), np.array([r], np.float32),
                        np.array([vmax], np.float32), np.array([1], np.uint8),
                        scenes.OrcaParams(), np.array([0], np.int32), wps,
                        np.array([wp_idx], np.uint8))


def test_waypoint_advance_boundary():
    """The waypoint index advances when the FP32 |wp - p|^2 <= r^2: a vehicle
    exactly r away advances (and then heads for the next waypoint), one FP32
    ulp farther it does not (and heads for the current one, capped so as not
    to overshoot: v_pref = (wp - p) / dt)."""
    r = oracle.step(_routed_vehicle([[0.5, 0.0], [0.0, 10.0], [20.0, 0.0]], 0))
    assert r.wp_idx[0] == 1
    assert np.abs(r.vel[0] - [0.0, 5.0]).max() <= 1e-12
    x = float(np.nextafter(np.float32(0.5), np.float32(1.0)))
    assert np.float32(x) * np.float32(x) > np.float32(0.25)
    r = oracle.step(_routed_vehicle([[x, 0.0], [0.0, 10.0], [20.0, 0.0]], 0))
    assert r.wp_idx[0] == 0
    assert np.abs(r.vel[0] - [x / 0.25, 0.0]).max() <= 1e-12


def test_waypoint_advances_at_most_once_per_step_and_holds_the_last():
    """Two waypoints on the agent: one advance per step.  At the last
    waypoint the index stays, even with the agent on it."""
    wps = [[0.0, 0.0], [0.0, 0.0], [0.0, 10.0]]
    r = oracle.step(_routed_vehicle(wps, 0))
    assert r.wp_idx[0] == 1
    r = oracle.step(_routed_vehicle(wps, 1))
    assert r.wp_idx[0] == 2
    assert np.abs(r.vel[0] - [0.0, 5.0]).max() <= 1e-12
    r = oracle.step(_routed_vehicle([[5.0, 0.0], [0.0, 0.0]], 1))
    assert r.wp_idx[0] == 1
    assert np.abs(r.vel[0]).max() == 0.0


# --------------------------------------------------- neighbour sets ---------

def test_neighbors_match_kdtree():
    rng = np.random.default_rng(16)
    n, k, R = 3000, 10, 10.0
    pos = rng.uniform(0, 120, (n, 2)).astype(np.float32)
    s = scenes.Scene(pos, np.zeros_like(pos), pos.copy(), np.full(n, 0.5, np.float32),
                     np.full(n, 1.5, np.float32), np.zeros(n, np.uint8),
                     scenes.OrcaParams(max_neighbors=k, neighbor_dist=R))
    r = oracle.step(s)
    tree = cKDTree(pos.astype(np.float64))
    dd, ii = tree.query(pos.astype(np.float64), k=k + 2)
    checked = 0
    for a in range(n):
        ds, js = dd[a, 1:], ii[a, 1:]
        cand = [(d, j) for d, j in zip(ds, js) if d < R and j != a][:k]
        # skip rows whose decision sits within FP32 rounding of a tie or of R
        nxt = ds[k] if len(ds) > k else np.inf
        if any(abs(d - R) < 1e-4 for d in ds) or (len(cand) == k and abs(nxt - cand[-1][0]) < 1e-4):
            continue
        assert r.cnt[a] == len(cand)
        assert list(r.nbr[a, :r.cnt[a]]) == [j for _, j in cand]
        checked += 1
    assert checked > 2900


def test_neighbor_tie_break_by_index():
    """Equal keys order by agent index (points on a lattice are exact ties)."""
    pos = np.array([[0, 0], [1, 0], [-1, 0], [0, 1], [0, -1], [2, 0]], np.float32)
    n = len(pos)
    s = scenes.Scene(pos, np.zeros_like(pos), pos.copy(), np.full(n, 0.1, np.float32),
                     np.full(n, 1.5, np.float32), np.zeros(n, np.uint8),
                     scenes.OrcaParams(max_neighbors=3))
    r = oracle.step(s, sel=[0])
    assert list(r.nbr[0]) == [1, 2, 3]


def test_cells_exact_boundaries_and_clamp():
    c = 2.0
    inv = np.float32(1.0 / c)
    xs = np.array([-5.0, 0.0, 1.999, 2.0, 3.9999, 4.0, 9.99, 10.0, 1e6], np.float32)
    pos = np.stack([xs, np.zeros_like(xs)], 1)
    cells = oracle.cells(pos, (0.0, 0.0), inv, 5, 5)
    assert list(cells) == [0, 0, 0, 1, 1, 2, 4, 4, 4]
    pos2 = np.stack([np.zeros_like(xs), xs], 1)
    assert list(oracle.cells(pos2, (0.0, 0.0), inv, 5, 5)) == [5 * c_ for c_ in [0, 0, 0, 1, 1, 2, 4, 4, 4]]


def test_rectangular_cells_exact_boundaries_and_clamp():
    """w x h cells (w = 4, h = 0.5): x uses 1/w and y 1/h, each edge exact,
    clamped to the grid; the id is cy * nx + cx.  Transposing the roles of
    the two axes would put (4, 0) in column 8 and (0, 0.5) in row 0."""
    inv = (np.float32(1.0) / np.float32(4.0), np.float32(1.0) / np.float32(0.5))
    nx, ny = 3, 8
    pts = np.array([[0.0, 0.0], [3.999, 0.0], [4.0, 0.0], [0.0, 0.4999], [0.0, 0.5],
                    [8.0, 1.0], [11.99, 3.75], [12.0, 4.0], [-1.0, -1.0], [100.0, 100.0]],
                   np.float32)
    want = [0, 0, 1, 0, nx, 2 + 2 * nx, 2 + 7 * nx, 2 + 7 * nx, 0, 2 + 7 * nx]
    assert list(oracle.cells(pts, (0.0, 0.0), inv, nx, ny)) == want
    # an origin shifts both axes: (1 + 4, -2 + 0.5) is cell (1, 1)
    assert list(oracle.cells(np.array([[5.0, -1.5]], np.float32), (1.0, -2.0), inv, nx, ny)) \
        == [1 + nx]


# ------------------------------------------------------ invariants ----------

def _spawn_non_overlapping(rng, n, side, r=0.5, gap=0.2):
    pts = []
    tries = 0
    while len(pts) < n and tries < 200000:
        tries += 1
        p = rng.uniform(0, side, 2)
        if all(np.linalg.norm(p - q) >= 2 * r + gap for q in pts):
            pts.append(p)
    return np.array(pts)


@pytest.mark.parametrize("seed", [20, 21])
def test_collision_free_invariant(seed):
    """Sec. 3.1: with f_{A|B} + f_{B|A} = 1 and both agents inside their ORCA
    half-planes, a pair that does not overlap cannot overlap after the step.
    Checked over FP64 rollouts of a two-way crossing with pedestrians and
    vehicles, k large enough that every nearby pair is mutual."""
    rng = np.random.default_rng(seed)
    n = 120
    pos = _spawn_non_overlapping(rng, n, 30.0, r=0.5, gap=2.5)
    n = len(pos)
    types = (np.arange(n) % 10 == 0).astype(np.uint8)
    rad = np.where(types == 1, 1.5, 0.5)
    left = pos[:, 0] < 15
    goal = pos.copy()
    goal[:, 0] = np.where(left, 45.0, -15.0)
    s = scenes.Scene(pos.astype(np.float32), np.zeros((n, 2), np.float32),
                     goal.astype(np.float32), rad.astype(np.float32),
                     np.where(types == 1, 3.0, 1.5).astype(np.float32), types,
                     scenes.OrcaParams(max_neighbors=64, neighbor_dist=8.0))
    P = s.pos.astype(np.float64)
    V = s.vel.astype(np.float64)
    pairs_checked = 0
    for t in range(30):
        r = oracle.step(s, pos=P, vel=V)
        nb = [set(r.nbr[a, :r.cnt[a]].tolist()) for a in range(n)]
        newP = r.pos
        for a in range(n):
            for b in nb[a]:
                if b < a or a not in nb[b]:
                    continue
                if r.flags[a] & 1 or r.flags[b] & 1:
                    continue
                rho = rad[a] + rad[b]
                if np.linalg.norm(P[b] - P[a]) <= rho:
                    continue
                assert np.linalg.norm(newP[b] - newP[a]) >= rho - 1e-9, (t, a, b)
                pairs_checked += 1
        P, V = newP, r.vel
    assert pairs_checked > 500


def test_rotation_equivariance_and_permutation():
    """A 90-degree rotation of the whole scene rotates every new velocity, and
    relabelling the agents permutes the outputs (no ties in the scene)."""
    s = scenes.open_square(300, 25.0, seed=5)
    r0 = oracle.step(s)
    rot = s.copy()
    rot.pos = np.stack([-s.pos[:, 1], s.pos[:, 0]], 1)
    rot.goal = np.stack([-s.goal[:, 1], s.goal[:, 0]], 1)
    r1 = oracle.step(rot)
    exp = np.stack([-r0.vel[:, 1], r0.vel[:, 0]], 1)
    assert np.abs(r1.vel - exp).max() <= 1e-9
    assert (r1.nbr == r0.nbr).all()
    perm = np.random.default_rng(6).permutation(s.n)
    ps = s.subset(perm)
    r2 = oracle.step(ps)
    assert np.abs(r2.vel - r0.vel[perm]).max() <= 1e-9


def test_translation_invariance():
    s = scenes.open_square(300, 25.0, seed=7)
    # positions on a 2^-10 grid so that adding 64 is exact in FP32
    s.pos = (np.round(s.pos * 1024) / 1024).astype(np.float32)
    s.goal = (np.round(s.goal * 1024) / 1024).astype(np.float32)
    r0 = oracle.step(s)
    sh = s.copy()
    sh.pos = s.pos + np.float32(64.0)
    sh.goal = s.goal + np.float32(64.0)
    r1 = oracle.step(sh)
    # every difference the step forms is unchanged by the exact shift
    assert (r1.nbr == r0.nbr).all()
    assert np.abs(r1.vel - r0.vel).max() <= 1e-9


def test_responsibility_zero_keeps_constraint_through_own_velocity():
    """f = 0 (car|person): the half-plane passes through v_A itself (Sec. 3.1)."""
    L = oracle.pair_line([0, 0], [1.0, 0.2], 1.5, [3, 0.5], [-1, 0], 0.5, 0.0, 5.0, 0.25, False)
    assert np.allclose(L[:2], [1.0, 0.2], atol=0)


def test_arrival_rule_boundaries():
    """The removal rule at its exact FP32 boundary: |g - p|^2 <= r^2 with
    each operation rounded; routed agents only at their last waypoint."""
    s = scenes.waypoint_square(n_ped=3, n_veh=1, side=10.0, n_wp=2, seed=0)
    s.radius[:] = np.float32(0.5)
    P = np.zeros((4, 2), np.float32)
    s.goal[:3] = np.array([[0.5, 0.0], [np.nextafter(np.float32(0.5), np.float32(1)), 0.0],
                           [0.3, 0.4]], np.float32)
    s.waypoints[0] = np.array([[0.0, 0.0], [0.1, 0.0]], np.float32)
    got = oracle.arrived(s, P, np.array([0, 0, 0, 0], np.uint8))
    # exactly r away: arrived; one ulp farther: not; 3-4-5 triangle scaled: d^2 = 0.25 = r^2
    assert got[:3].tolist() == [True, False, True]
    assert not got[3]                                  # on its first waypoint
    assert oracle.arrived(s, P, np.array([0, 0, 0, 1], np.uint8))[3]


def _lone_vehicle(v0, goal, turn_rate=0.0, accel=0.0):
    P = np.array([[0.0, 0.0]], np.float32)
    s = scenes.Scene(P, np.array([v0], np.float32), np.array([goal], np.float32),
                     np.array([1.5], np.float32), np.array([5.0], np.float32),
                     np.array([1], np.uint8),
                     scenes.OrcaParams(extent=(100.0, 100.0), origin=(-50.0, -50.0),
                                       vehicle_turn_rate=turn_rate, vehicle_accel=accel))
    return oracle.step(s).vel[0]


@pytest.mark.parametrize("rate", [0.3, 1.0, 2.5])
def test_vehicle_turn_limit_closed_form(rate):
    """A vehicle heading east that wants to go north at full speed turns by
    exactly theta = rate * dt: v* = 5 sin(theta) (cos theta, sin theta), the
    projection of v_pref onto the edge of the allowed wedge."""
    th = float(np.float32(rate)) * 0.25
    v = _lone_vehicle([3.0, 0.0], [0.0, 40.0], turn_rate=rate)
    exp = 5.0 * np.sin(th) * np.array([np.cos(th), np.sin(th)])
    assert np.abs(v - exp).max() <= 1e-9


def test_vehicle_accel_limit_closed_form():
    """Straight ahead at 2 m/s with 2 m/s^2: the next speed is 2 + 2 * 0.25;
    from rest it is 2 * 0.25 along the preferred velocity."""
    v = _lone_vehicle([2.0, 0.0], [40.0, 0.0], turn_rate=1.0, accel=2.0)
    assert np.abs(v - np.array([2.5, 0.0])).max() <= 1e-9
    v = _lone_vehicle([0.0, 0.0], [30.0, 40.0], turn_rate=1.0, accel=2.0)
    assert np.abs(v - 0.5 * np.array([0.6, 0.8])).max() <= 1e-9
    # limits off: the unconstrained preferred velocity
    v = _lone_vehicle([2.0, 0.0], [0.0, 40.0])
    assert np.abs(v - np.array([0.0, 5.0])).max() <= 1e-9


def test_kinematic_limits_leave_pedestrians_alone():
    s = scenes.open_square(300, 20.0, seed=7)
    s.params.vehicle_turn_rate, s.params.vehicle_accel = 0.5, 1.0
    a = oracle.step(s)
    s.params.vehicle_turn_rate, s.params.vehicle_accel = 0.0, 0.0
    b = oracle.step(s)
    assert np.array_equal(a.vel, b.vel)
