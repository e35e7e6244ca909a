"""Launch autotuner for a bed or batch handle.

Times a few steps for each candidate launch setting (persistent CTAs per SM, sort period)
on a copy of the parcel state with CUDA events on the handle's stream, and keeps the
fastest. The settings change no result beyond the summation grouping of the deposits.
"""
from __future__ import annotations

import itertools

import torch


def autotune(bed, parcels: dict, gas, steps: int = 10, grids=(0, 2, 3), sorts=(5, 10, 20),
             obj_shape=None):
    """Pick (grid_per_sm, sort_every) for `bed` (mppic.Bed or mppic.Batch) and apply it.

    Returns {"best": (grid, sort), "ms_per_step": {(grid, sort): ms}}.
    """
    stream = bed.stream
    timings = {}
    for g, srt in itertools.product(grids, sorts):
        bed.tune(g, srt)
        work = {k: v.clone() for k, v in parcels.items()}
        bed.step(work, gas, srt)                       # settle any first-use work
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n = max(steps, srt)
        e0.record(stream)
        bed.step(work, gas, n)
        e1.record(stream)
        e1.synchronize()
        bed.check()
        timings[(g, srt)] = e0.elapsed_time(e1) / n
        del work
    best = min(timings, key=timings.get)
    bed.tune(*best)
    return {"best": best, "ms_per_step": timings}
