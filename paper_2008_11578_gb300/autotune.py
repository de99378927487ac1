"""Autotuner of the launch shape: grid cell size and solve-kernel block size.

Neither knob changes any result.  The neighbour search is exact for every
cell size (the ring stencil grows until the k-th key is certified), and each
agent's arithmetic does not depend on the block it runs in, so every
candidate produces bit-identical states; the tuner only times candidates on
a copy of the state and keeps the fastest.  The neighbour cap is a compile-
time choice (16 or 32 slots, the smallest that holds k).

Candidates: cell size = alpha x the scene's default cell size, for each
alpha in ``alphas``, times each block size in ``blocks``.  Each candidate
runs ``warmup`` untimed steps and ``steps`` timed steps (CUDA events on the
launching stream) from the scene's initial state.
"""
from __future__ import annotations

import dataclasses

from . import api
from ._lib import OrcaError

DEFAULT_ALPHAS = (0.375, 0.5, 0.75, 1.0, 1.5, 2.0)
DEFAULT_BLOCKS = (64, 128)


@dataclasses.dataclass
class TuneResult:
    alpha: float
    block_size: int
    ms_per_step: float
    table: list          # (alpha, block_size, ms_per_step or None if rejected)

    def cell_sizes(self, scene_list):
        return [self.alpha * float(sc.params.cell_size) for sc in scene_list]


def _time_steps(obj, steps, warmup):
    import torch
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        obj.step(1)
    b = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    b.record(stream)
    obj.step(steps)
    e.record(stream)
    torch.cuda.synchronize()
    return b.elapsed_time(e) / steps


def _tune(make, alphas, blocks, steps, warmup):
    table = []
    best = None
    for a in alphas:
        for bs in blocks:
            try:
                obj = make(a, bs)
            except OrcaError:          # grid too fine for the cell limit
                table.append((a, bs, None))
                continue
            ms = _time_steps(obj, steps, warmup)
            obj.close()
            table.append((a, bs, ms))
            if best is None or ms < best[2]:
                best = (a, bs, ms)
    if best is None:
        raise RuntimeError("no autotuner candidate could be created")
    return TuneResult(best[0], best[1], best[2], table)


def tune_scene(scene, device="cuda", alphas=DEFAULT_ALPHAS, blocks=DEFAULT_BLOCKS,
               steps=3, warmup=1) -> TuneResult:
    """Fastest (cell size, block size) for one scene."""
    base = float(scene.params.cell_size)
    return _tune(lambda a, bs: api.DeviceScene(scene, device, cell_size=a * base,
                                               block_size=bs),
                 alphas, blocks, steps, warmup)


def tune_batch(scene_list, device="cuda", alphas=DEFAULT_ALPHAS, blocks=DEFAULT_BLOCKS,
               steps=3, warmup=1) -> TuneResult:
    """Fastest (cell-size factor, block size) for a batch; every scene's cell
    is alpha x its own default cell size."""
    bases = [float(sc.params.cell_size) for sc in scene_list]
    return _tune(lambda a, bs: api.DeviceBatch(scene_list, device,
                                               cell_sizes=[a * c for c in bases],
                                               block_size=bs),
                 alphas, blocks, steps, warmup)
