"""FP64 CPU oracle of the ORCA step (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline leg may import this package.  The CUDA library and its Python
binding never import it, and the two share no code.

``orca_oracle.c`` holds the arithmetic (plain C, FP64, OpenMP over agents).
This module compiles it with gcc and exposes it through ctypes.

What it computes (paper Sec. 3 and 3.1): per agent the k nearest neighbours,
one ORCA half-plane per neighbour placed at v_opt + f_{A|B} u, the velocity
LP (projection of the preferred velocity onto the admissible set, with the
least-penetration fallback when it is empty), and the synchronous move.

Parity pins (tests/test_oracle_pins.py) tie it to things other than itself:
KKT certificates, dense grid search, scipy's QP and LP solvers, the head-on
closed form, the ORCA collision-free invariant, kd-tree neighbour sets and
exact symmetries.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "orca_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liborca_oracle.so")
_lock = threading.Lock()
_lib = None

_CFLAGS = ["-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/_build`` (git-ignored)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cc = os.environ.get("CC", "gcc")
    subprocess.check_call([cc, *_CFLAGS, _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_D = ctypes.POINTER(ctypes.c_double)
_F = ctypes.POINTER(ctypes.c_float)
_I32 = ctypes.POINTER(ctypes.c_int32)
_U32 = ctypes.POINTER(ctypes.c_uint32)
_U8 = ctypes.POINTER(ctypes.c_uint8)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.oracle_num_threads.restype = ctypes.c_int
            L.oracle_set_num_threads.argtypes = [ctypes.c_int]
            L.oracle_cells.argtypes = [ctypes.c_int, _F, _F, ctypes.c_float,
                                       ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                       ctypes.c_int, ctypes.c_int, _I32]
            L.oracle_pair_line.argtypes = [ctypes.c_double] * 13 + [ctypes.c_int, _D]
            L.oracle_lp.argtypes = [ctypes.c_int, _D, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_double, _D, _U32]
            L.oracle_lp.restype = ctypes.c_int
            L.oracle_project.argtypes = [ctypes.c_int, _D, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, _D]
            L.oracle_project.restype = ctypes.c_int
            L.oracle_step.argtypes = (
                [ctypes.c_int] + [_D] * 8 + [_U8, _I32, _D, _D, ctypes.c_int, _U8,
                                             _D, _D, ctypes.c_double, ctypes.c_int,
                                             ctypes.c_double, ctypes.c_double, _D,
                                             ctypes.c_double, ctypes.c_double,
                                             ctypes.c_int, _I32, _D, _D, _U8, _I32,
                                             _I32, _U8, _D, _D, _D, _U32])
            L.oracle_step.restype = ctypes.c_int
            _lib = L
    return _lib


def _p(a, t):
    if a is None:
        return ctypes.cast(None, t)
    return a.ctypes.data_as(t)


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def set_num_threads(n: int) -> None:
    lib().oracle_set_num_threads(int(n))


def cells(pos, origin, inv_cell, nx, ny) -> np.ndarray:
    """Cell id cy*nx + cx of every agent (FP32 decision).

    ``inv_cell`` is fl32(1 / cell edge) for square cells, or a pair
    (fl32(1 / width), fl32(1 / height)) for rectangular ones."""
    inv = np.atleast_1d(np.asarray(inv_cell, dtype=np.float32))
    ix, iy = (inv[0], inv[0]) if inv.size == 1 else (inv[0], inv[1])
    pos = np.ascontiguousarray(pos, dtype=np.float32)
    x = np.ascontiguousarray(pos[:, 0])
    y = np.ascontiguousarray(pos[:, 1])
    out = np.empty(pos.shape[0], np.int32)
    lib().oracle_cells(pos.shape[0], _p(x, _F), _p(y, _F), float(origin[0]),
                       float(origin[1]), float(ix), float(iy), int(nx), int(ny),
                       _p(out, _I32))
    return out


def pair_line(pa, va, ra, pb, vb, rb, f, tau, dt, overlap) -> np.ndarray:
    """ORCA half-plane of one ordered pair: (P_x, P_y, d_x, d_y)."""
    out = np.zeros(4)
    lib().oracle_pair_line(float(pa[0]), float(pa[1]), float(va[0]), float(va[1]),
                           float(ra), float(pb[0]), float(pb[1]), float(vb[0]),
                           float(vb[1]), float(rb), float(f), float(tau), float(dt),
                           int(bool(overlap)), _p(out, _D))
    return out


def lp(lines, vmax, vpref):
    """Velocity LP from explicit lines (n, 4).

    Returns (v (2,), t_star, flags, cond, active_mask).
    """
    lines = np.ascontiguousarray(np.asarray(lines, dtype=np.float64).reshape(-1, 4))
    out = np.zeros(4)
    mask = np.zeros(1, np.uint32)
    fl = lib().oracle_lp(lines.shape[0], _p(lines, _D), float(vmax),
                         float(vpref[0]), float(vpref[1]), _p(out, _D), _p(mask, _U32))
    return out[:2].copy(), float(out[2]), int(fl), float(out[3]), int(mask[0])


def project(lines, t, vmax, vpref):
    """Projection of vpref onto the lines relaxed by t and the disc (or None)."""
    lines = np.ascontiguousarray(np.asarray(lines, dtype=np.float64).reshape(-1, 4))
    out = np.zeros(2)
    ok = lib().oracle_project(lines.shape[0], _p(lines, _D), float(t), float(vmax),
                              float(vpref[0]), float(vpref[1]), _p(out, _D))
    return out if ok == 1 else None


class StepResult:
    """Outputs of one oracle step for the selected agents."""

    def __init__(self, sel, v, p, wp, nbr, cnt, flags, tstar, cond, lines, mask):
        self.sel, self.vel, self.pos, self.wp_idx = sel, v, p, wp
        self.nbr, self.cnt, self.flags = nbr, cnt, flags
        self.tstar, self.cond, self.lines, self.mask = tstar, cond, lines, mask

    @property
    def infeasible(self):
        return (self.flags & 1) != 0


def step(scene, sel=None, vpref_delta=None, state=None, want_lines=False,
         pos=None, vel=None, wp_idx=None) -> StepResult:
    """One synchronous oracle step of ``scene`` for agents ``sel`` (all if None).

    ``pos``/``vel``/``wp_idx`` override the scene's state (FP64 allowed).
    """
    prm = scene.params
    P = np.asarray(scene.pos if pos is None else pos, dtype=np.float64)
    V = np.asarray(scene.vel if vel is None else vel, dtype=np.float64)
    n = P.shape[0]
    px, py = np.ascontiguousarray(P[:, 0]), np.ascontiguousarray(P[:, 1])
    vx, vy = np.ascontiguousarray(V[:, 0]), np.ascontiguousarray(V[:, 1])
    G = scene.goal.astype(np.float64)
    gx, gy = np.ascontiguousarray(G[:, 0]), np.ascontiguousarray(G[:, 1])
    rad = np.ascontiguousarray(scene.radius, dtype=np.float64)
    vm = np.ascontiguousarray(scene.max_speed, dtype=np.float64)
    ty = np.ascontiguousarray(scene.type, dtype=np.uint8)
    route = wpx = wpy = wpi = None
    n_wp = 0
    if scene.route is not None:
        route = np.ascontiguousarray(scene.route, dtype=np.int32)
        W = scene.waypoints.astype(np.float64)
        n_wp = W.shape[1]
        wpx = np.ascontiguousarray(W[..., 0].reshape(-1))
        wpy = np.ascontiguousarray(W[..., 1].reshape(-1))
        wpi = np.ascontiguousarray(scene.wp_idx if wp_idx is None else wp_idx,
                                   dtype=np.uint8)
    dvx = dvy = None
    if vpref_delta is not None:
        D = np.asarray(vpref_delta, dtype=np.float64)
        dvx, dvy = np.ascontiguousarray(D[:, 0]), np.ascontiguousarray(D[:, 1])
    if sel is None:
        sel_arr = None
        ns = n
    else:
        sel_arr = np.ascontiguousarray(sel, dtype=np.int32)
        ns = sel_arr.shape[0]
    k = int(prm.max_neighbors)
    f4 = np.ascontiguousarray(np.asarray(prm.f, dtype=np.float64).reshape(4))
    ov = np.zeros((ns, 2))
    op = np.zeros((ns, 2))
    owp = np.zeros(ns, np.uint8)
    onbr = np.zeros((ns, k), np.int32)
    ocnt = np.zeros(ns, np.int32)
    ofl = np.zeros(ns, np.uint8)
    ots = np.zeros(ns)
    ocond = np.zeros(ns)
    omask = np.zeros(ns, np.uint32)
    olines = np.zeros((ns, k, 4)) if want_lines else None
    rc = lib().oracle_step(
        n, _p(px, _D), _p(py, _D), _p(vx, _D), _p(vy, _D), _p(gx, _D), _p(gy, _D),
        _p(rad, _D), _p(vm, _D), _p(ty, _U8), _p(route, _I32), _p(wpx, _D),
        _p(wpy, _D), n_wp, _p(wpi, _U8), _p(dvx, _D), _p(dvy, _D),
        float(np.float32(prm.neighbor_dist)), k, float(np.float32(prm.time_horizon)),
        float(np.float32(prm.dt)), _p(f4, _D),
        float(np.float32(getattr(prm, "vehicle_turn_rate", 0.0))),
        float(np.float32(getattr(prm, "vehicle_accel", 0.0))), ns, _p(sel_arr, _I32), _p(ov, _D),
        _p(op, _D), _p(owp, _U8), _p(onbr, _I32), _p(ocnt, _I32), _p(ofl, _U8),
        _p(ots, _D), _p(ocond, _D), _p(olines, _D), _p(omask, _U32))
    if rc != 0:
        raise ValueError(f"oracle_step rejected its arguments ({rc})")
    return StepResult(sel_arr, ov, op, owp, onbr, ocnt, ofl, ots, ocond, olines, omask)


def arrived(scene, pos, wp_idx=None) -> np.ndarray:
    """Which agents have reached their goal and leave the scene (Sec. 4:
    agents are removed on arrival and a run ends when all have arrived).

    Agent i has arrived when |g - p|^2 <= r^2, evaluated in IEEE FP32 with
    every difference, product and the sum rounded separately (numpy float32
    arithmetic), where g is its goal, or for an agent on a route its current
    waypoint once that is the route's last one.
    """
    P = np.asarray(pos, dtype=np.float32)
    G = np.asarray(scene.goal, dtype=np.float32).copy()
    final = np.ones(P.shape[0], dtype=bool)
    if scene.route is not None:
        rt = np.asarray(scene.route)
        on = np.nonzero(rt >= 0)[0]
        W = np.asarray(scene.waypoints, dtype=np.float32)
        wi = np.asarray(wp_idx if wp_idx is not None else scene.wp_idx)[on].astype(np.int64)
        G[on] = W[rt[on], wi]
        final[on] = wi == W.shape[1] - 1
    dx = np.subtract(G[:, 0], P[:, 0], dtype=np.float32)
    dy = np.subtract(G[:, 1], P[:, 1], dtype=np.float32)
    d2 = np.add(np.multiply(dx, dx, dtype=np.float32), np.multiply(dy, dy, dtype=np.float32),
                dtype=np.float32)
    r = np.asarray(scene.radius, dtype=np.float32)
    return final & (d2 <= np.multiply(r, r, dtype=np.float32))


def rollout(scene, n_steps, vpref_delta=None, fp32_state=True):
    """Run the oracle for ``n_steps`` synchronous steps from the scene's state.

    With ``fp32_state`` the state is rounded to FP32 after every step (the
    state representation of the CUDA path); otherwise it stays FP64.
    ``vpref_delta`` has shape (n_steps, N, 2) or is None.
    Returns (pos, vel, wp_idx) after the last step and the per-step positions.
    """
    pos = scene.pos.astype(np.float64)
    vel = scene.vel.astype(np.float64)
    wpi = None if scene.wp_idx is None else scene.wp_idx.copy()
    traj = []
    for t in range(n_steps):
        d = None if vpref_delta is None else vpref_delta[t]
        r = step(scene, pos=pos, vel=vel, wp_idx=wpi, vpref_delta=d)
        pos, vel = r.pos, r.vel
        if fp32_state:
            pos = pos.astype(np.float32).astype(np.float64)
            vel = vel.astype(np.float32).astype(np.float64)
        if wpi is not None:
            wpi = r.wp_idx.copy()
        traj.append((pos.copy(), vel.copy()))
    return pos, vel, wpi, traj
