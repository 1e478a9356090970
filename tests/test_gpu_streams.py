"""Runs of one grid in flight on several streams at once (each takes its own
scratch slot) give exactly the tallies of the same packets run serially."""
import numpy as np
import pytest

import workloads as W
from _gpu_common import need_gpu

pytestmark = pytest.mark.gpu


def test_concurrent_runs_match_serial():
    krl = need_gpu()
    import torch
    p = W.sphere(vmax_kms=200.0, tau0=1e5, n=32, n_packets=40000)
    out = []
    for concurrent in (False, True):
        g = krl.Grid(p)
        try:
            streams = [torch.cuda.Stream() for _ in range(3)]
            chunks = [(0, 13000), (13000, 14000), (27000, 13000)]
            for k, (lo, n) in enumerate(chunks):
                s = streams[k] if concurrent else torch.cuda.current_stream()
                for st_ in streams:
                    st_.wait_stream(torch.cuda.current_stream())
                g.run(n=n, first=lo, want_stats=False, stream=s)
            torch.cuda.synchronize()
            out.append({k: g.tally(k).cpu().numpy() for k in ("spec_n", "scatmap", "stats")})
        finally:
            g.close()
    a, b = out
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    assert a["stats"][0] == 40000 == a["stats"][1]
