"""Python binding of liborca: argument marshalling only.

Functions named like the C entry points (``orca_workspace_bytes``,
``orca_scene_create``, ``orca_step`` ...) forward to the C ABI with device
pointers taken from torch tensors; :class:`DeviceScene` bundles the tensors
of one scene.  Every step of the ORCA update runs in liborca's kernels;
torch provides device memory and the current stream only.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import _lib
from ._lib import OrcaAgents, OrcaError, OrcaParams, check


def _torch():
    import torch
    return torch


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream_handle(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


LP_WORK_UNITS = 2   # orca_params.debug_flags: the paper's work-unit batch LP
BARRIER_TIMEOUT_TEST = 4   # orca_params.debug_flags: failure-detection test hook
LP_ENUMERATION = 8   # orca_params.debug_flags: active-set enumeration LP (comparison)
LP_WARP = 16   # orca_params.debug_flags: warp-cooperative LP (comparison)
CHECKED = 32   # orca_params.debug_flags: steps certify their results on the device


def make_params(p, cell_size: float | None = None, block_size: int = 0,
                flags: int = 0, cell_height: float | None = None) -> OrcaParams:
    """orca_params from a :class:`scenes.OrcaParams` (grid from its box).

    ``cell_size`` is the cell width; ``cell_height`` its height (None: the
    width, unless neither is given and the params fix a height)."""
    c, h = p.cell_dims(cell_size, cell_height)
    nx, ny = p.grid_dims(cell_size, cell_height)
    f = np.asarray(p.f, dtype=np.float32).reshape(2, 2)
    cp = OrcaParams()
    cp.neighbor_dist = float(p.neighbor_dist)
    cp.time_horizon = float(p.time_horizon)
    cp.dt = float(p.dt)
    cp.max_neighbors = int(p.max_neighbors)
    for a in range(2):
        for b in range(2):
            cp.f[a][b] = float(f[a, b])
    cp.cell_size = c
    cp.cell_height = h
    cp.origin_x = float(p.origin[0])
    cp.origin_y = float(p.origin[1])
    cp.grid_nx = int(nx)
    cp.grid_ny = int(ny)
    cp.block_size = int(block_size)
    cp.debug_flags = int(flags)
    cp.vehicle_turn_rate = float(getattr(p, "vehicle_turn_rate", 0.0))
    cp.vehicle_accel = float(getattr(p, "vehicle_accel", 0.0))
    return cp


# ------------------------------------------------------------- C names ------

def orca_status_string(status: int) -> str:
    return _lib.load().orca_status_string(int(status)).decode()


def orca_abi_version() -> int:
    return int(_lib.load().orca_abi_version())


def orca_workspace_bytes(params: OrcaParams, n_agents: int) -> int:
    out = ctypes.c_size_t(0)
    check(_lib.load().orca_workspace_bytes(ctypes.byref(params), int(n_agents),
                                           ctypes.byref(out)), "orca_workspace_bytes")
    return int(out.value)


def orca_scene_create(params: OrcaParams, agents: OrcaAgents, workspace, ws_bytes: int):
    h = ctypes.c_void_p()
    check(_lib.load().orca_scene_create(ctypes.byref(params), ctypes.byref(agents),
                                        _ptr(workspace), int(ws_bytes), ctypes.byref(h)),
          "orca_scene_create")
    return h


def orca_scene_set_debug(handle, cell=None, nbr=None, cnt=None, flags=None, tstar=None):
    check(_lib.load().orca_scene_set_debug(handle, _ptr(cell), _ptr(nbr), _ptr(cnt),
                                           _ptr(flags), _ptr(tstar)), "orca_scene_set_debug")


def orca_scene_set_solve_events(handle, begin=None, end=None):
    """Bracket the solve kernel of every following step with two
    ``torch.cuda.Event(enable_timing=True)`` (or None to stop)."""
    for ev in (begin, end):
        if ev is not None and ev.cuda_event == 0:
            ev.record()     # torch creates the CUDA event at its first record
    b = None if begin is None else ctypes.c_void_p(begin.cuda_event)
    e = None if end is None else ctypes.c_void_p(end.cuda_event)
    check(_lib.load().orca_scene_set_solve_events(handle, b, e), "orca_scene_set_solve_events")


def orca_scene_set_bin_events(handle, begin=None, end=None):
    """Bracket the binning kernel (cell keys, scan, scatter) of every following
    step with two torch CUDA events (or None to stop)."""
    for ev in (begin, end):
        if ev is not None and ev.cuda_event == 0:
            ev.record()
    b = None if begin is None else ctypes.c_void_p(begin.cuda_event)
    e = None if end is None else ctypes.c_void_p(end.cuda_event)
    check(_lib.load().orca_scene_set_bin_events(handle, b, e), "orca_scene_set_bin_events")


def orca_scene_set_counters(handle, counters=None):
    """Accumulate work tallies and phase clock cycles into ``counters``
    (int64[13] on the device; the layout is in orca.h)."""
    check(_lib.load().orca_scene_set_counters(handle, _ptr(counters)), "orca_scene_set_counters")


_cudart = None


def event_elapsed_ms(begin, end) -> float:
    """Milliseconds between two torch CUDA events recorded by liborca (torch's
    own elapsed_time only accepts events it recorded itself)."""
    global _cudart
    if _cudart is None:
        _cudart = ctypes.CDLL("libcudart.so.13")
        _cudart.cudaEventElapsedTime.argtypes = [ctypes.POINTER(ctypes.c_float),
                                                 ctypes.c_void_p, ctypes.c_void_p]
        _cudart.cudaEventElapsedTime.restype = ctypes.c_int
    ms = ctypes.c_float(0.0)
    rc = _cudart.cudaEventElapsedTime(ctypes.byref(ms), ctypes.c_void_p(begin.cuda_event),
                                      ctypes.c_void_p(end.cuda_event))
    if rc != 0:
        raise RuntimeError(f"cudaEventElapsedTime failed ({rc})")
    return float(ms.value)


def orca_step(handle, n_steps: int, vpref_delta=None, stream=None):
    check(_lib.load().orca_step(handle, int(n_steps), _ptr(vpref_delta),
                                _stream_handle(stream)), "orca_step")


def orca_scene_graph_capture(handle, n_steps: int, vpref_delta=None):
    check(_lib.load().orca_scene_graph_capture(handle, int(n_steps), _ptr(vpref_delta)),
          "orca_scene_graph_capture")


def orca_scene_graph_launch(handle, stream=None):
    check(_lib.load().orca_scene_graph_launch(handle, _stream_handle(stream)),
          "orca_scene_graph_launch")


def orca_step_launch_count(handle, n_steps: int) -> int:
    return int(_lib.load().orca_step_launch_count(handle, int(n_steps)))


def orca_scene_sync_status(handle) -> int:
    return int(_lib.load().orca_scene_sync_status(handle))


def orca_scene_destroy(handle) -> None:
    _lib.load().orca_scene_destroy(handle)


def orca_step_noalloc(params: OrcaParams, agents: OrcaAgents, n_steps: int,
                      vpref_delta=None, stream=None, synchronize: bool = False) -> int:
    """orca_step without a scene or workspace, for callers that cannot
    allocate device memory; scratch comes from a fixed 2 MiB area inside the
    library, shared by all calls (serialise calls that could overlap on the
    GPU).  Returns the C status (0 = ok) instead of raising, so callers can
    tell a too-large scene (ORCA_ERR_CAPACITY) from other errors."""
    return int(_lib.load().orca_step_noalloc(ctypes.byref(params), ctypes.byref(agents),
                                             int(n_steps), _ptr(vpref_delta),
                                             _stream_handle(stream), int(bool(synchronize))))


def orca_scene_remove_arrived(handle, kept_index=None, stream=None) -> int:
    """Remove arrived agents in place; returns the new agent count."""
    n = ctypes.c_int(0)
    check(_lib.load().orca_scene_remove_arrived(handle, ctypes.byref(n), _ptr(kept_index),
                                                _stream_handle(stream)),
          "orca_scene_remove_arrived")
    return int(n.value)


def orca_scene_set_debug_active(handle, act=None):
    """Record every agent's LP active set (uint32[N] on the device)."""
    check(_lib.load().orca_scene_set_debug_active(handle, _ptr(act)),
          "orca_scene_set_debug_active")


def orca_adjoint_workspace_bytes(handle, n_steps: int, ckpt_every: int) -> int:
    out = ctypes.c_size_t(0)
    check(_lib.load().orca_adjoint_workspace_bytes(handle, int(n_steps), int(ckpt_every),
                                                   ctypes.byref(out)),
          "orca_adjoint_workspace_bytes")
    return int(out.value)


def orca_rollout(handle, n_steps: int, ckpt_every: int, vpref_delta, adj_ws, adj_bytes: int,
                 vel_traj=None, stream=None):
    check(_lib.load().orca_rollout(handle, int(n_steps), int(ckpt_every), _ptr(vpref_delta),
                                   _ptr(adj_ws), int(adj_bytes), _ptr(vel_traj),
                                   _stream_handle(stream)), "orca_rollout")


def orca_adjoint(handle, n_steps: int, ckpt_every: int, vpref_delta, adj_ws, adj_bytes: int,
                 dl_dpos, dl_dvel_traj=None, dl_dvpref_delta=None, dl_dwaypoints=None,
                 dl_dpos0=None, dl_dvel0=None, stream=None):
    check(_lib.load().orca_adjoint(handle, int(n_steps), int(ckpt_every), _ptr(vpref_delta),
                                   _ptr(adj_ws), int(adj_bytes), _ptr(dl_dpos),
                                   _ptr(dl_dvel_traj), _ptr(dl_dvpref_delta),
                                   _ptr(dl_dwaypoints), _ptr(dl_dpos0), _ptr(dl_dvel0),
                                   _stream_handle(stream)), "orca_adjoint")


def orca_step_vjp(handle, adj_ws, adj_bytes: int, pos, vel, wp_idx, vpref_delta, dl_dpos_next,
                  dl_dvel_next, dl_dpos, dl_dvel, dl_dvpref_delta=None, dl_dwaypoints=None,
                  stream=None):
    check(_lib.load().orca_step_vjp(handle, _ptr(adj_ws), int(adj_bytes), _ptr(pos), _ptr(vel),
                                    _ptr(wp_idx), _ptr(vpref_delta), _ptr(dl_dpos_next),
                                    _ptr(dl_dvel_next), _ptr(dl_dpos), _ptr(dl_dvel),
                                    _ptr(dl_dvpref_delta), _ptr(dl_dwaypoints),
                                    _stream_handle(stream)), "orca_step_vjp")


def orca_adjoint_launch_count(handle, n_steps: int, ckpt_every: int) -> int:
    return int(_lib.load().orca_adjoint_launch_count(handle, int(n_steps), int(ckpt_every)))


def _params_array(params_list):
    arr = (OrcaParams * len(params_list))()
    for i, p in enumerate(params_list):
        arr[i] = p
    return arr


def _offsets_array(offsets):
    return (ctypes.c_int * len(offsets))(*[int(o) for o in offsets])


def orca_batch_workspace_bytes(params_list, offsets) -> int:
    out = ctypes.c_size_t(0)
    check(_lib.load().orca_batch_workspace_bytes(_params_array(params_list), len(params_list),
                                                 _offsets_array(offsets), ctypes.byref(out)),
          "orca_batch_workspace_bytes")
    return int(out.value)


def orca_batch_create(params_list, offsets, agents: OrcaAgents, workspace, ws_bytes: int):
    h = ctypes.c_void_p()
    check(_lib.load().orca_batch_create(_params_array(params_list), len(params_list),
                                        _offsets_array(offsets), ctypes.byref(agents),
                                        _ptr(workspace), int(ws_bytes), ctypes.byref(h)),
          "orca_batch_create")
    return h


def orca_batch_set_debug(handle, cell=None, nbr=None, cnt=None, flags=None, tstar=None):
    check(_lib.load().orca_batch_set_debug(handle, _ptr(cell), _ptr(nbr), _ptr(cnt),
                                           _ptr(flags), _ptr(tstar)), "orca_batch_set_debug")


def orca_step_batched(handle, n_steps: int, vpref_delta=None, stream=None):
    check(_lib.load().orca_step_batched(handle, int(n_steps), _ptr(vpref_delta),
                                        _stream_handle(stream)), "orca_step_batched")


def orca_batch_launch_count(handle, n_steps: int) -> int:
    return int(_lib.load().orca_batch_launch_count(handle, int(n_steps)))


def orca_batch_graph_capture(handle, n_steps: int, vpref_delta=None):
    check(_lib.load().orca_batch_graph_capture(handle, int(n_steps), _ptr(vpref_delta)),
          "orca_batch_graph_capture")


def orca_batch_graph_launch(handle, stream=None):
    check(_lib.load().orca_batch_graph_launch(handle, _stream_handle(stream)),
          "orca_batch_graph_launch")


def orca_batch_sync_status(handle) -> int:
    return int(_lib.load().orca_batch_sync_status(handle))


def orca_batch_destroy(handle) -> None:
    _lib.load().orca_batch_destroy(handle)


# ------------------------------------------------------------- scene --------

class DeviceScene:
    """One scene's agent arrays and workspace on the GPU, behind liborca.

    ``scene`` is a :class:`scenes.Scene` (numpy, caller order).  The device
    tensors ``pos``, ``vel`` and ``wp_idx`` are updated in place by
    :meth:`step`; ``goal``, ``radius``, ``max_speed``, ``type``, ``route``
    and ``waypoints`` are read-only inputs.  ``pos`` and ``vel`` are the two
    halves of one tensor, ``state`` (shape (2, n, 2)), so the evolving state
    moves between host and device in a single copy each way.
    """

    def __init__(self, scene, device="cuda", cell_size=None, block_size=0, debug=False,
                 flags=0, cell_height=None):
        torch = _torch()
        self.device = torch.device(device)
        self.scene = scene
        self.n = scene.n
        self.k = int(scene.params.max_neighbors)
        dev = self.device

        def t(a, dt=None):
            return torch.as_tensor(np.ascontiguousarray(a), device=dev, dtype=dt)

        # positions and velocities share one allocation ([0] = pos, [1] = vel),
        # so the evolving state moves between host and device in one copy
        self.state = torch.empty((2, self.n, 2), dtype=torch.float32, device=dev)
        self.pos, self.vel = self.state[0], self.state[1]
        self.pos.copy_(t(scene.pos, torch.float32).reshape(self.n, 2))
        self.vel.copy_(t(scene.vel, torch.float32).reshape(self.n, 2))
        self.goal = t(scene.goal, torch.float32)
        self.radius = t(scene.radius, torch.float32)
        self.max_speed = t(scene.max_speed, torch.float32)
        self.type = t(scene.type, torch.uint8)
        self.route = self.waypoints = self.wp_idx = None
        if scene.route is not None:
            self.route = t(scene.route, torch.int32)
            self.waypoints = t(scene.waypoints.reshape(-1, 2), torch.float32)
            self.wp_idx = t(scene.wp_idx, torch.uint8)
        self.params = make_params(scene.params, cell_size, block_size, flags, cell_height)
        self.ws_bytes = orca_workspace_bytes(self.params, self.n)
        self.workspace = torch.empty(max(self.ws_bytes, 256), dtype=torch.uint8, device=dev)
        a = OrcaAgents()
        a.n_agents = self.n
        a.pos, a.vel, a.goal = _ptr(self.pos), _ptr(self.vel), _ptr(self.goal)
        a.radius, a.max_speed, a.type = _ptr(self.radius), _ptr(self.max_speed), _ptr(self.type)
        a.route = _ptr(self.route)
        a.waypoints = _ptr(self.waypoints)
        a.n_routes = 0 if scene.route is None else int(scene.waypoints.shape[0])
        a.n_waypoints = 0 if scene.route is None else int(scene.waypoints.shape[1])
        a.wp_idx = _ptr(self.wp_idx)
        self._agents = a
        self.handle = orca_scene_create(self.params, a, self.workspace, self.ws_bytes)
        self.dbg = None
        if debug:
            self.enable_debug()

    def enable_debug(self, active=False):
        """Per-agent diagnostics of the last step (``self.dbg``); with
        ``active`` also the LP active set (``self.dbg["act"]``, int32 view of
        the packed uint32 words)."""
        torch = _torch()
        n, k, dev = self.n, max(self.k, 1), self.device
        self.dbg = dict(cell=torch.full((n,), -1, dtype=torch.int32, device=dev),
                        nbr=torch.full((n, k), -1, dtype=torch.int32, device=dev),
                        cnt=torch.zeros(n, dtype=torch.int32, device=dev),
                        flags=torch.zeros(n, dtype=torch.uint8, device=dev),
                        tstar=torch.zeros(n, dtype=torch.float32, device=dev))
        orca_scene_set_debug(self.handle, **self.dbg)
        if active:
            self.dbg["act"] = torch.zeros(n, dtype=torch.int32, device=dev)
            orca_scene_set_debug_active(self.handle, self.dbg["act"])

    def set_state(self, pos=None, vel=None, wp_idx=None):
        torch = _torch()
        if pos is not None:
            self.pos.copy_(torch.as_tensor(pos, dtype=torch.float32))
        if vel is not None:
            self.vel.copy_(torch.as_tensor(vel, dtype=torch.float32))
        if wp_idx is not None and self.wp_idx is not None:
            self.wp_idx.copy_(torch.as_tensor(wp_idx, dtype=torch.uint8))

    def step(self, n_steps: int = 1, vpref_delta=None, stream=None):
        if vpref_delta is not None:
            assert vpref_delta.dtype == _torch().float32 and vpref_delta.is_contiguous()
            assert vpref_delta.numel() == 2 * n_steps * self.n
        orca_step(self.handle, n_steps, vpref_delta, stream)

    def remove_arrived(self):
        """Remove the agents at their goal (the paper's removal on arrival).

        The kept agents are compacted to the front of every device array;
        ``self.n`` becomes their count (the tensors keep their size, rows
        ``self.n:`` are stale).  Returns the previous indices of the kept
        agents (numpy int32)."""
        torch = _torch()
        kept = torch.empty(max(self.n, 1), dtype=torch.int32, device=self.device)
        self.n = orca_scene_remove_arrived(self.handle, kept)
        if self.dbg is not None:
            self.enable_debug(active="act" in self.dbg)
        return kept[:self.n].cpu().numpy()

    def capture(self, n_steps: int, vpref_delta=None):
        """Record ``n_steps`` steps into the scene's CUDA graph."""
        orca_scene_graph_capture(self.handle, n_steps, vpref_delta)

    def replay(self, stream=None):
        """Launch the recorded graph on ``stream`` (torch's current one)."""
        orca_scene_graph_launch(self.handle, stream)

    def launch_count(self, n_steps: int) -> int:
        return orca_step_launch_count(self.handle, n_steps)

    def sync_status(self) -> int:
        return orca_scene_sync_status(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            orca_scene_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class DeviceBatch:
    """Many independent scenes advanced together by one launch per phase.

    ``scene_list`` holds :class:`scenes.Scene` objects; their agents are
    concatenated (scene 0 first) into the device tensors ``pos``, ``vel`` ...
    and ``offsets[s]:offsets[s + 1]`` is scene ``s``'s slice.  Routes are
    re-based onto the concatenated waypoint rows.  ``cell_sizes`` and
    ``cell_heights`` (one per scene, or None for each scene's default) only
    change speed, never results.
    """

    def __init__(self, scene_list, device="cuda", cell_sizes=None, block_size=0, debug=False,
                 cell_heights=None):
        torch = _torch()
        self.device = torch.device(device)
        dev = self.device
        self.scenes = list(scene_list)
        S = len(self.scenes)
        if S == 0:
            raise ValueError("a batch needs at least one scene")
        sizes = [sc.n for sc in self.scenes]
        self.offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        self.n = int(self.offsets[-1])
        if cell_sizes is None:
            cell_sizes = [None] * S
        if cell_heights is None:
            cell_heights = [None] * S
        self.params_list = [make_params(sc.params, c, block_size, 0, h)
                            for sc, c, h in zip(self.scenes, cell_sizes, cell_heights)]
        self.kmax = max(int(p.max_neighbors) for p in self.params_list)

        def cat(get, dtype):
            return torch.as_tensor(np.ascontiguousarray(np.concatenate(
                [get(sc) for sc in self.scenes])), device=dev, dtype=dtype)

        self.pos = cat(lambda sc: sc.pos.reshape(-1, 2), torch.float32)
        self.vel = cat(lambda sc: sc.vel.reshape(-1, 2), torch.float32)
        self.goal = cat(lambda sc: sc.goal.reshape(-1, 2), torch.float32)
        self.radius = cat(lambda sc: sc.radius, torch.float32)
        self.max_speed = cat(lambda sc: sc.max_speed, torch.float32)
        self.type = cat(lambda sc: sc.type, torch.uint8)
        self.route = self.waypoints = self.wp_idx = None
        routed = [sc for sc in self.scenes if sc.route is not None]
        n_wp = 0
        n_routes = 0
        if routed:
            n_wp = int(routed[0].waypoints.shape[1])
            if any(int(sc.waypoints.shape[1]) != n_wp for sc in routed):
                raise ValueError("all routed scenes of a batch need the same waypoint count")
            rows, routes, row0 = [], [], 0
            for sc in self.scenes:
                if sc.route is None:
                    routes.append(np.full(sc.n, -1, np.int32))
                else:
                    r = sc.route.astype(np.int64)
                    routes.append(np.where(r >= 0, r + row0, -1).astype(np.int32))
                    rows.append(sc.waypoints.reshape(-1, n_wp, 2))
                    row0 += sc.waypoints.shape[0]
            n_routes = row0
            self.route = torch.as_tensor(np.concatenate(routes), device=dev, dtype=torch.int32)
            self.waypoints = torch.as_tensor(np.ascontiguousarray(
                np.concatenate(rows).reshape(-1, 2)), device=dev, dtype=torch.float32)
            self.wp_idx = cat(lambda sc: sc.wp_idx if sc.wp_idx is not None
                              else np.zeros(sc.n, np.uint8), torch.uint8)
        self.ws_bytes = orca_batch_workspace_bytes(self.params_list, self.offsets)
        self.workspace = torch.empty(max(self.ws_bytes, 256), dtype=torch.uint8, device=dev)
        a = OrcaAgents()
        a.n_agents = self.n
        a.pos, a.vel, a.goal = _ptr(self.pos), _ptr(self.vel), _ptr(self.goal)
        a.radius, a.max_speed, a.type = _ptr(self.radius), _ptr(self.max_speed), _ptr(self.type)
        a.route = _ptr(self.route)
        a.waypoints = _ptr(self.waypoints)
        a.n_routes = n_routes
        a.n_waypoints = n_wp
        a.wp_idx = _ptr(self.wp_idx)
        self._agents = a
        self.handle = orca_batch_create(self.params_list, self.offsets, a, self.workspace,
                                        self.ws_bytes)
        self.dbg = None
        if debug:
            self.enable_debug()

    def enable_debug(self):
        torch = _torch()
        n, k, dev = self.n, max(self.kmax, 1), self.device
        self.dbg = dict(cell=torch.full((n,), -1, dtype=torch.int32, device=dev),
                        nbr=torch.full((n, k), -1, dtype=torch.int32, device=dev),
                        cnt=torch.zeros(n, dtype=torch.int32, device=dev),
                        flags=torch.zeros(n, dtype=torch.uint8, device=dev),
                        tstar=torch.zeros(n, dtype=torch.float32, device=dev))
        orca_batch_set_debug(self.handle, **self.dbg)

    def scene_slice(self, s: int) -> slice:
        return slice(int(self.offsets[s]), int(self.offsets[s + 1]))

    def step(self, n_steps: int = 1, vpref_delta=None, stream=None):
        orca_step_batched(self.handle, n_steps, vpref_delta, stream)

    def capture(self, n_steps: int, vpref_delta=None):
        """Record ``n_steps`` batched steps into the batch's CUDA graph."""
        orca_batch_graph_capture(self.handle, n_steps, vpref_delta)

    def replay(self, stream=None):
        orca_batch_graph_launch(self.handle, stream)

    def launch_count(self, n_steps: int) -> int:
        return orca_batch_launch_count(self.handle, n_steps)

    def sync_status(self) -> int:
        return orca_batch_sync_status(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            orca_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
