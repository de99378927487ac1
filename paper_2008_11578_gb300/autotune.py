"""Autotuner of the launch shape: grid cell shape and solve-kernel block size.

None of the knobs changes any result.  The neighbour search is exact for
every cell width and height (it scans each x-sorted grid row outward from the
agent until the k-th key is certified), and each agent's arithmetic does not
depend on the block it runs in, so every candidate produces bit-identical
states; the tuner only times candidates on a copy of the state and keeps the
fastest.  The neighbour cap is a compile-time choice (16 or 32 slots, the
smallest that holds k).

Candidates: cell height = alpha x the scene's default cell size for each
alpha in ``alphas``, cell width = aspect x height for each aspect in
``aspects`` (thin, wide cells: the search looks at most one row height
beyond the k-th nearest neighbour, while wide cells keep the cell count
down), times each block size in ``blocks``.  Each candidate runs ``warmup``
untimed steps and ``steps`` timed steps (CUDA events on the launching
stream) from the scene's initial state.
"""
from __future__ import annotations

import dataclasses

from . import api
from ._lib import OrcaError

DEFAULT_ALPHAS = (0.375, 0.5, 0.75, 1.0, 1.5, 2.0)
DEFAULT_ASPECTS = (1.0, 2.0, 4.0, 8.0)
DEFAULT_BLOCKS = (64, 128)


@dataclasses.dataclass
class TuneResult:
    alpha: float         # cell height / the scene's default cell size
    aspect: float        # cell width / cell height
    block_size: int
    ms_per_step: float
    table: list          # (alpha, aspect, block_size, ms_per_step or None if rejected)

    def cell_heights(self, scene_list):
        return [self.alpha * float(sc.params.cell_size) for sc in scene_list]

    def cell_sizes(self, scene_list):
        """Cell widths."""
        return [self.aspect * h for h in self.cell_heights(scene_list)]


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


def _tune(make, alphas, aspects, blocks, steps, warmup):
    table = []
    best = None
    for a in alphas:
        for asp in aspects:
            for bs in blocks:
                try:
                    obj = make(a, asp, bs)
                except OrcaError:          # grid too fine for the cell limit
                    table.append((a, asp, bs, None))
                    continue
                ms = _time_steps(obj, steps, warmup)
                obj.close()
                table.append((a, asp, bs, ms))
                if best is None or ms < best[3]:
                    best = (a, asp, bs, ms)
    if best is None:
        raise RuntimeError("no autotuner candidate could be created")
    return TuneResult(best[0], best[1], best[2], best[3], table)


def tune_scene(scene, device="cuda", alphas=DEFAULT_ALPHAS, aspects=DEFAULT_ASPECTS,
               blocks=DEFAULT_BLOCKS, steps=3, warmup=1) -> TuneResult:
    """Fastest (cell height, cell width, block size) for one scene."""
    base = float(scene.params.cell_size)
    return _tune(lambda a, asp, bs: api.DeviceScene(scene, device, cell_size=asp * a * base,
                                                    cell_height=a * base, block_size=bs),
                 alphas, aspects, blocks, steps, warmup)


def tune_batch(scene_list, device="cuda", alphas=DEFAULT_ALPHAS, aspects=DEFAULT_ASPECTS,
               blocks=DEFAULT_BLOCKS, steps=3, warmup=1) -> TuneResult:
    """Fastest (height factor, aspect, block size) for a batch; every scene's
    cell height is alpha x its own default cell size."""
    bases = [float(sc.params.cell_size) for sc in scene_list]
    return _tune(lambda a, asp, bs: api.DeviceBatch(scene_list, device,
                                                    cell_sizes=[asp * a * c for c in bases],
                                                    cell_heights=[a * c for c in bases],
                                                    block_size=bs),
                 alphas, aspects, blocks, steps, warmup)
