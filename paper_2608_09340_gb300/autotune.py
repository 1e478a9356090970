"""Launch-parameter autotuner for the packet walk.

Times short pilot runs (a fraction of each model's packets, under ids that
the real run does not use) for every candidate (block size, refill
threshold, CTAs per SM) and returns the fastest. Pilot tallies are
discarded (the tallies are reset afterwards), so tuning does not change
what a later run accumulates.
"""
from __future__ import annotations

import itertools

DEFAULT_SPACE = {
    "block": (256, 512),
    "refill_min": (1, 4, 16),
    "ctas_per_sm": (0, 1),          # 0: as many as fit
}

# The batched launch runs CTAs of at most 256 threads.
BATCH_SPACE = {
    "block": (128, 256),
    "refill_min": (1, 4, 16),
    "ctas_per_sm": (0, 1),
}

PILOT_FIRST_ID = 1 << 48            # pilot packets use ids far from any real run


def _candidates(space):
    keys = list(space)
    for vals in itertools.product(*(space[k] for k in keys)):
        yield dict(zip(keys, vals))


def _time(fn):
    import torch
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


PILOT_SET_STRIDE = 1 << 40           # pilot set r starts at PILOT_FIRST_ID + r * stride


def tune_batch(batch, packets, fraction: float = 0.2, space=None, seed: int = 12345, repeats: int = 2):
    """Best {block, refill_min, ctas_per_sm} for `batch` (a Batch) and the
    per-model packet counts `packets`; returns (best, timings). Each
    candidate is timed on `repeats` disjoint pilot sets and ranked by the
    sum: a pilot's time is set largely by its few longest packets, so one
    set alone ranks close candidates by chance."""
    space = space or BATCH_SPACE
    pilot = [max(1, int(n * fraction)) for n in packets]
    timings = []
    for cand in _candidates(space):
        try:                            # a block the walk does not support raises: skip it
            ms = 0.0
            for r in range(repeats):
                first = [PILOT_FIRST_ID + r * PILOT_SET_STRIDE] * len(pilot)
                ms += _time(lambda: batch.run(pilot, first_ids=first, seed=seed, **cand))
        except Exception:
            continue
        timings.append((ms, cand))
    for g in batch.grids:
        g.reset()
    timings.sort(key=lambda t: t[0])
    return timings[0][1], timings


def tune_grid(grid, n: int, fraction: float = 0.05, space=None, seed: int = 12345):
    """Best launch parameters for krl_run_packets on one grid."""
    space = space or DEFAULT_SPACE
    pilot = max(1, int(n * fraction))
    timings = []
    for cand in _candidates(space):
        try:
            ms = _time(lambda: grid.run(n=pilot, first=PILOT_FIRST_ID, seed=seed, want_stats=False, **cand))
        except Exception:
            continue
        timings.append((ms, cand))
    grid.reset()
    timings.sort(key=lambda t: t[0])
    return timings[0][1], timings
