"""Build and load liborca (the CUDA library) and declare its C ABI for ctypes.

The library is compiled in-tree with nvcc for sm_103a only and loaded from
``paper_2008_11578_gb300/_build/liborca.so``.  There is no fallback: if the
library cannot be built or loaded, every entry point raises.
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_PKG)
_CSRC = os.path.join(_PKG, "csrc")
_INCLUDE = os.path.join(_ROOT, "include")
BUILD_DIR = os.path.join(_PKG, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liborca.so")

ARCH_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-shared",
              "-cudart", "shared", "-Xcompiler", "-fno-strict-aliasing"]

_SOURCES = ["orca_capi.cu"]

_lock = threading.Lock()
_lib = None


def _nvcc() -> str:
    cand = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: liborca cannot be built")
    return cand


def _deps():
    files = [os.path.join(_INCLUDE, "orca.h")]
    for f in os.listdir(_CSRC):
        if f.endswith((".cu", ".cuh", ".h")):
            files.append(os.path.join(_CSRC, f))
    return files


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile liborca.so for sm_103a (cross-compiles without a GPU)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if not force and os.path.exists(LIB_PATH):
        t = os.path.getmtime(LIB_PATH)
        if all(os.path.getmtime(f) <= t for f in _deps()):
            return LIB_PATH
    cuda_lib = os.path.join(os.path.dirname(os.path.dirname(_nvcc())), "lib64")
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = [_nvcc(), *ARCH_FLAGS, *NVCC_FLAGS, f"-I{_INCLUDE}", f"-I{_CSRC}",
           *[os.path.join(_CSRC, s) for s in _SOURCES], "-o", tmp,
           "-Xlinker", f"-rpath,{cuda_lib}"]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.check_call(cmd)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class OrcaParams(ctypes.Structure):
    _fields_ = [("neighbor_dist", ctypes.c_float), ("time_horizon", ctypes.c_float),
                ("dt", ctypes.c_float), ("max_neighbors", ctypes.c_int),
                ("f", (ctypes.c_float * 2) * 2), ("cell_size", ctypes.c_float),
                ("origin_x", ctypes.c_float), ("origin_y", ctypes.c_float),
                ("grid_nx", ctypes.c_int), ("grid_ny", ctypes.c_int),
                ("block_size", ctypes.c_int), ("debug_flags", ctypes.c_uint),
                ("vehicle_turn_rate", ctypes.c_float), ("vehicle_accel", ctypes.c_float),
                ("cell_height", ctypes.c_float)]


class OrcaAgents(ctypes.Structure):
    _fields_ = [("n_agents", ctypes.c_int), ("pos", ctypes.c_void_p),
                ("vel", ctypes.c_void_p), ("goal", ctypes.c_void_p),
                ("radius", ctypes.c_void_p), ("max_speed", ctypes.c_void_p),
                ("type", ctypes.c_void_p), ("route", ctypes.c_void_p),
                ("waypoints", ctypes.c_void_p), ("n_routes", ctypes.c_int),
                ("n_waypoints", ctypes.c_int), ("wp_idx", ctypes.c_void_p)]


# every symbol the header declares, with (restype, argtypes)
_V = ctypes.c_void_p
_I = ctypes.c_int
SIGNATURES = {
    "orca_status_string": (ctypes.c_char_p, [_I]),
    "orca_abi_version": (_I, []),
    "orca_workspace_bytes": (_I, [ctypes.POINTER(OrcaParams), _I, ctypes.POINTER(ctypes.c_size_t)]),
    "orca_scene_create": (_I, [ctypes.POINTER(OrcaParams), ctypes.POINTER(OrcaAgents), _V,
                               ctypes.c_size_t, ctypes.POINTER(_V)]),
    "orca_scene_set_debug": (_I, [_V, _V, _V, _V, _V, _V]),
    "orca_scene_set_solve_events": (_I, [_V, _V, _V]),
    "orca_scene_set_bin_events": (_I, [_V, _V, _V]),
    "orca_scene_set_counters": (_I, [_V, _V]),
    "orca_step": (_I, [_V, _I, _V, _V]),
    "orca_step_launch_count": (_I, [_V, _I]),
    "orca_scene_graph_capture": (_I, [_V, _I, _V]),
    "orca_scene_graph_launch": (_I, [_V, _V]),
    "orca_scene_sync_status": (_I, [_V]),
    "orca_scene_destroy": (None, [_V]),
    "orca_scene_set_debug_active": (_I, [_V, _V]),
    "orca_scene_remove_arrived": (_I, [_V, ctypes.POINTER(ctypes.c_int), _V, _V]),
    "orca_adjoint_workspace_bytes": (_I, [_V, _I, _I, ctypes.POINTER(ctypes.c_size_t)]),
    "orca_rollout": (_I, [_V, _I, _I, _V, _V, ctypes.c_size_t, _V, _V]),
    "orca_adjoint": (_I, [_V, _I, _I, _V, _V, ctypes.c_size_t, _V, _V, _V, _V, _V, _V, _V]),
    "orca_adjoint_launch_count": (_I, [_V, _I, _I]),
    "orca_step_vjp": (_I, [_V, _V, ctypes.c_size_t] + [_V] * 10 + [_V]),
    "orca_batch_workspace_bytes": (_I, [ctypes.POINTER(OrcaParams), _I,
                                       ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_size_t)]),
    "orca_batch_create": (_I, [ctypes.POINTER(OrcaParams), _I, ctypes.POINTER(ctypes.c_int),
                               ctypes.POINTER(OrcaAgents), _V, ctypes.c_size_t,
                               ctypes.POINTER(_V)]),
    "orca_batch_set_debug": (_I, [_V, _V, _V, _V, _V, _V]),
    "orca_step_batched": (_I, [_V, _I, _V, _V]),
    "orca_batch_launch_count": (_I, [_V, _I]),
    "orca_batch_graph_capture": (_I, [_V, _I, _V]),
    "orca_batch_graph_launch": (_I, [_V, _V]),
    "orca_batch_sync_status": (_I, [_V]),
    "orca_batch_destroy": (None, [_V]),
    "orca_step_noalloc": (_I, [ctypes.POINTER(OrcaParams), ctypes.POINTER(OrcaAgents), _I, _V,
                               _V, _I]),
}
NOALLOC_SCRATCH_BYTES = 2 << 20

STATUS = {0: "ORCA_OK", 1: "ORCA_ERR_INVALID_ARG", 2: "ORCA_ERR_CUDA",
          3: "ORCA_ERR_TIMEOUT", 4: "ORCA_ERR_NONFINITE", 5: "ORCA_ERR_CAPACITY",
          6: "ORCA_ERR_CHECK"}
MAX_NEIGHBORS = 32


class OrcaError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {STATUS.get(status, status)}")


def load(path: str | None = None):
    """Load liborca (building it first when needed) and declare signatures."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or build()
            L = ctypes.CDLL(p, mode=ctypes.RTLD_GLOBAL)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def check(status: int, what: str) -> None:
    if status != 0:
        raise OrcaError(status, what)
