"""Host-side checks of the C ABI (no GPU needed, no compute calls).

The library must load, export every function include/orca.h declares, and
reject bad arguments on the host before touching the device.
"""
import ctypes
import os
import re

import pytest

from paper_2008_11578_gb300 import _lib, api, scenes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    txt = open(os.path.join(ROOT, "include", header)).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(orca_[a-z0-9_]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported():
    L = _lib.load()
    names = _declared("orca.h")
    assert "orca_step" in names and "orca_scene_create" in names
    for n in names:
        assert hasattr(L, n), n
        assert n in _lib.SIGNATURES, f"{n} has no ctypes signature"


def test_version_and_status_strings():
    assert api.orca_abi_version() == 5
    assert api.orca_status_string(0) == "ok"
    assert "non-finite" in api.orca_status_string(4)
    assert "invariant" in api.orca_status_string(6)
    assert api.orca_status_string(99) == "unknown status"


def _params(**kw):
    p = api.make_params(scenes.OrcaParams())
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def test_workspace_bytes_and_parameter_validation():
    b1 = api.orca_workspace_bytes(_params(), 1000)
    b2 = api.orca_workspace_bytes(_params(), 2000)
    assert 0 < b1 < b2 and b1 % 256 == 0
    assert api.orca_workspace_bytes(_params(), 0) > 0
    L = _lib.load()
    out = ctypes.c_size_t()
    for bad, code in [(dict(dt=0.0), 1), (dict(neighbor_dist=-1.0), 1),
                      (dict(time_horizon=float("nan")), 1), (dict(cell_size=0.0), 1),
                      (dict(max_neighbors=-1), 1), (dict(max_neighbors=33), 5),
                      (dict(grid_nx=0), 1), (dict(grid_nx=1 << 14, grid_ny=1 << 14), 5),
                      (dict(block_size=48), 1), (dict(block_size=256), 1),
                      (dict(debug_flags=1), 1), (dict(debug_flags=128), 1),
                      (dict(debug_flags=10), 1), (dict(debug_flags=14), 1),
                      (dict(debug_flags=18), 1), (dict(debug_flags=24), 1),
                      (dict(debug_flags=34), 1), (dict(debug_flags=64), 1),
                      (dict(cell_height=-1.0), 1), (dict(cell_height=float("nan")), 1),
                      (dict(cell_height=float("inf")), 1)]:
        p = _params(**bad)
        assert L.orca_workspace_bytes(ctypes.byref(p), 10, ctypes.byref(out)) == code, bad
    for good in (2, 4, 6, 8, 12, 16, 20, 32, 36):   # one scheme/checked flag, and/or the test hook
        p = _params(debug_flags=good)
        assert L.orca_workspace_bytes(ctypes.byref(p), 10, ctypes.byref(out)) == 0, good
    for h in (0.0, 0.25, 8.0):   # 0 = square cells
        p = _params(cell_height=h)
        assert L.orca_workspace_bytes(ctypes.byref(p), 10, ctypes.byref(out)) == 0, h
    p = _params()
    assert L.orca_workspace_bytes(ctypes.byref(p), -1, ctypes.byref(out)) == 1
    assert L.orca_workspace_bytes(None, 10, ctypes.byref(out)) == 1


def test_create_rejects_bad_arguments_on_host():
    L = _lib.load()
    p = _params()
    h = ctypes.c_void_p()
    a = _lib.OrcaAgents()
    a.n_agents = 10
    # null agent arrays
    assert L.orca_scene_create(ctypes.byref(p), ctypes.byref(a), ctypes.c_void_p(4096),
                               1 << 20, ctypes.byref(h)) == 1
    fake = 1 << 40      # never dereferenced: validation fails before any access
    for f in ("pos", "vel", "goal", "radius", "max_speed", "type"):
        setattr(a, f, fake)
    need = api.orca_workspace_bytes(p, 10)
    # misaligned / missing / small workspace
    assert L.orca_scene_create(ctypes.byref(p), ctypes.byref(a), ctypes.c_void_p(fake + 8),
                               need, ctypes.byref(h)) == 1
    assert L.orca_scene_create(ctypes.byref(p), ctypes.byref(a), None, need,
                               ctypes.byref(h)) == 1
    assert L.orca_scene_create(ctypes.byref(p), ctypes.byref(a), ctypes.c_void_p(fake),
                               need - 256, ctypes.byref(h)) == 1
    # misaligned float2 array
    a.pos = fake + 4
    assert L.orca_scene_create(ctypes.byref(p), ctypes.byref(a), ctypes.c_void_p(fake),
                               need, ctypes.byref(h)) == 1
    a.pos = fake
    # a route without waypoints
    a.route = fake
    assert L.orca_scene_create(ctypes.byref(p), ctypes.byref(a), ctypes.c_void_p(fake),
                               need, ctypes.byref(h)) == 1
    a.route = None
    # bad parameters
    q = _params(max_neighbors=40)
    assert L.orca_scene_create(ctypes.byref(q), ctypes.byref(a), ctypes.c_void_p(fake),
                               need, ctypes.byref(h)) == 5
    assert L.orca_scene_create(ctypes.byref(p), ctypes.byref(a), ctypes.c_void_p(fake),
                               need, None) == 1


def test_null_handles():
    L = _lib.load()
    assert L.orca_step(None, 1, None, None) == 1
    assert L.orca_step_launch_count(None, 1) == -1
    assert L.orca_scene_sync_status(None) == 1
    assert L.orca_scene_set_debug(None, None, None, None, None, None) == 1
    L.orca_scene_destroy(None)


def test_batch_validation_on_host():
    L = _lib.load()
    plist = [_params(), _params(grid_nx=10, grid_ny=10), _params()]
    out = ctypes.c_size_t()
    off = api._offsets_array([0, 5, 5, 12])
    arr = api._params_array(plist)
    assert L.orca_batch_workspace_bytes(arr, 3, off, ctypes.byref(out)) == 0
    one = ctypes.c_size_t()
    assert L.orca_workspace_bytes(ctypes.byref(plist[0]), 12, ctypes.byref(one)) == 0
    assert out.value > one.value and out.value % 256 == 0
    # offsets must start at 0 and not decrease
    assert L.orca_batch_workspace_bytes(arr, 3, api._offsets_array([1, 5, 5, 12]),
                                        ctypes.byref(out)) == 1
    assert L.orca_batch_workspace_bytes(arr, 3, api._offsets_array([0, 6, 5, 12]),
                                        ctypes.byref(out)) == 1
    assert L.orca_batch_workspace_bytes(arr, 0, off, ctypes.byref(out)) == 1
    # every scene shares the launch shape
    bad = api._params_array([_params(), _params(block_size=64), _params()])
    assert L.orca_batch_workspace_bytes(bad, 3, off, ctypes.byref(out)) == 1
    # per-scene parameter errors surface with their own code
    bad = api._params_array([_params(), _params(max_neighbors=40), _params()])
    assert L.orca_batch_workspace_bytes(bad, 3, off, ctypes.byref(out)) == 5
    # the cell total of all scenes is bounded
    big = api._params_array([_params(grid_nx=1 << 13, grid_ny=1 << 13)] * 3)
    assert L.orca_batch_workspace_bytes(big, 3, off, ctypes.byref(out)) == 5
    # create: offsets must end at n_agents
    a = _lib.OrcaAgents()
    a.n_agents = 13
    fake = 1 << 40
    for f in ("pos", "vel", "goal", "radius", "max_speed", "type"):
        setattr(a, f, fake)
    h = ctypes.c_void_p()
    assert L.orca_batch_create(arr, 3, off, ctypes.byref(a), ctypes.c_void_p(fake), 1 << 30,
                               ctypes.byref(h)) == 1
    a.n_agents = 12
    assert L.orca_batch_create(arr, 3, off, ctypes.byref(a), ctypes.c_void_p(fake + 16),
                               1 << 30, ctypes.byref(h)) == 1
    assert L.orca_batch_create(arr, 3, off, ctypes.byref(a), ctypes.c_void_p(fake), 256,
                               ctypes.byref(h)) == 1
    assert L.orca_step_batched(None, 1, None, None) == 1
    assert L.orca_batch_launch_count(None, 1) == -1
    assert L.orca_batch_graph_capture(None, 1, None) == 1
    assert L.orca_batch_graph_launch(None, None) == 1
    assert L.orca_scene_graph_capture(None, 1, None) == 1
    assert L.orca_scene_graph_launch(None, None) == 1
    assert L.orca_batch_sync_status(None) == 1
    L.orca_batch_destroy(None)


def test_removal_rejects_null_arguments():
    L = _lib.load()
    n = ctypes.c_int()
    assert L.orca_scene_remove_arrived(None, ctypes.byref(n), None, None) == 1


def test_rectangular_cell_parameters():
    """Cell width and height reach orca_params and size the grid: a width
    alone means square cells, a height of 0 in the scene's parameters too."""
    p = scenes.OrcaParams(extent=(50.0, 30.0), cell_size=2.0)
    cp = api.make_params(p, 4.0, cell_height=0.5)
    assert (cp.cell_size, cp.cell_height, cp.grid_nx, cp.grid_ny) == (4.0, 0.5, 13, 60)
    cp = api.make_params(p, 3.0)
    assert (cp.cell_size, cp.cell_height, cp.grid_nx, cp.grid_ny) == (3.0, 3.0, 17, 10)
    cp = api.make_params(p)
    assert (cp.cell_size, cp.cell_height, cp.grid_nx, cp.grid_ny) == (2.0, 2.0, 25, 15)
    p.cell_height = 1.5
    cp = api.make_params(p)
    assert (cp.cell_size, cp.cell_height, cp.grid_nx, cp.grid_ny) == (2.0, 1.5, 25, 20)
