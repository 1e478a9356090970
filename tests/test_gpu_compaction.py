"""Packets moved between lanes (the tail compaction of the persistent walk)
continue exactly as they would have in their old lane: per-packet records and
integer tallies are bit-identical across launch shapes, which give different
lane assignments, different tails and different compaction patterns."""
import numpy as np
import pytest

import workloads as W
from _gpu_common import gpu_run, need_gpu

pytestmark = pytest.mark.gpu

SHAPES = [dict(), dict(block=256, refill_min=16, ctas_per_sm=1), dict(block=64, ctas_per_sm=1),
          dict(block=128, refill_min=4)]


def _same(a, b):
    ra, rb = a["records"], b["records"]
    for f in ("status", "nscat", "ncross", "cell0"):
        assert np.array_equal(ra[f], rb[f]), f
    assert np.array_equal(ra["x"].view(np.uint32), rb["x"].view(np.uint32))
    for k in ("spec_n", "scatmap", "stats_tally"):
        if a[k] is not None:
            assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_records_independent_of_launch_shape(prec):
    """Static sphere with a heavy-tailed scattering count (most of a launch's
    packets end long before the last ones, so every shape compacts)."""
    krl = need_gpu()
    p = W.sphere(vmax_kms=0.0, tau0=3e3, n=16, n_packets=6000)
    pr = krl.KRL_PREC_FP32 if prec == "fp32" else krl.KRL_PREC_FP64
    runs = [gpu_run(krl, p, pr, **s) for s in SHAPES]
    for r in runs[1:]:
        _same(runs[0], r)
    st = runs[0]["stats_tally"]
    assert st[0] == 6000 == st[1]


def test_rich_walk_records_independent_of_launch_shape():
    """Rich-tally walk (emissivity, J, excitation, destruction): records and
    the escape histogram exact, floating-point tallies equal up to the order
    of their atomic additions."""
    krl = need_gpu()
    p = W.envelope(n=16, n_ch=16, n_packets=3000)
    runs = [gpu_run(krl, p, krl.KRL_PREC_FP32, **s) for s in SHAPES[:3]]
    for r in runs[1:]:
        _same(runs[0], r)
        for k in ("exc", "J", "emiss"):
            a, b = runs[0][k].astype(np.float64), r[k].astype(np.float64)
            assert np.abs(a - b).sum() <= 1e-5 * np.abs(a).sum(), k
