"""Properties of the sampler tables that the CUDA walk's search shortcuts
rely on, checked on the oracle's tables (the device builds the same tables,
element by element: tests/test_gpu_tables.py).

* The row guide: |x| is binned by the top bits of its float32 encoding (16
  bins per octave, from 0.25 to 512); the walk takes the largest row whose
  node is at or below the bin's lower edge and steps up at most once. That
  is exact only if no bin holds two nodes.
* The row inversions walk a row's ln CDF from a guide entry without bound
  checks: they stop inside the row because every row starts below the
  smallest ln(xi) (xi >= 2^-24) and ends at ln 1 = 0, above the largest.
"""
import math

import numpy as np
import pytest

from oracle import tables as T

ROW_GUIDE_N = 176
ROW_GUIDE_SHIFT = 19


def _edges():
    base = int(np.float32(0.25).view(np.uint32)) >> ROW_GUIDE_SHIFT
    return np.array([np.uint32((t + base) << ROW_GUIDE_SHIFT) for t in range(ROW_GUIDE_N + 1)],
                    dtype=np.uint32).view(np.float32)


def test_row_guide_bins_hold_at_most_one_node():
    xs = np.asarray(T.usampler_xnodes(), dtype=np.float32)
    e = _edges()
    assert e[0] == 0.25 and e[-1] == 512.0 and xs[-1] < e[-1]
    assert xs[1] > e[0]                     # below the first bin every |x| is in row 0
    for t in range(ROW_GUIDE_N):
        inside = int(((xs >= e[t]) & (xs < e[t + 1])).sum())
        assert inside <= 1, (t, e[t], e[t + 1])


def test_row_guide_lookup_equals_the_bracket():
    """The guide plus one step up gives the largest node <= |x| for every
    |x| (a dense sweep in float32, including every node and its neighbours)."""
    xs = np.asarray(T.usampler_xnodes(), dtype=np.float32)
    e = _edges()
    guide = np.array([max(i for i in range(len(xs) - 1) if xs[i] <= e[t]) for t in range(ROW_GUIDE_N)])
    base = int(np.float32(0.25).view(np.uint32)) >> ROW_GUIDE_SHIFT
    probe = np.concatenate([np.linspace(0, 320, 200001, dtype=np.float32), xs,
                            np.nextafter(xs, np.float32(0)), np.nextafter(xs, np.float32(1e9))]).astype(np.float32)
    t = (probe.view(np.uint32) >> ROW_GUIDE_SHIFT).astype(np.int64) - base
    t = np.clip(t, 0, ROW_GUIDE_N - 1)
    i = guide[t]
    up = (i < len(xs) - 2) & (xs[np.minimum(i + 1, len(xs) - 1)] <= probe)
    row = i + up
    want = np.clip(np.searchsorted(xs, probe, side="right") - 1, 0, len(xs) - 2)
    assert np.array_equal(row, want)


@pytest.mark.parametrize("a", [1e-4, 4.7e-4, 1e-2, 0.149])
def test_sampler_rows_bound_the_search(a):
    _, lnc = T.usampler_table(a)
    lnc = np.asarray(lnc, dtype=np.float32)
    smallest = math.log(2.0 ** -24)
    assert np.all(lnc[:, 0] < smallest)
    assert np.all(lnc[:, -1] == 0.0)
    assert np.all(np.diff(lnc, axis=1) >= 0)
