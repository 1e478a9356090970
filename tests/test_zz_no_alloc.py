"""krl_emission_cdf_noalloc, the allocation-free entry point.

Callers that cannot call cudaMalloc (an application whose device memory
belongs to its own pool or framework allocator, or a loop that must not
take cudaMalloc's implicit synchronisation) get the volume-source emission
CDF from this call, whose scratch is a fixed array in the library. It must
give the same CDF as the allocating path (krl_line_set, read back with
krl_tallies_get), also on a second call that reuses the array left over by
the first. Collected last so that a failure here comes after every other
test has run."""
import ctypes as C
import dataclasses

import numpy as np
import pytest

import workloads as W
from _gpu_common import need_gpu

pytestmark = pytest.mark.gpu


def _lib(krl):
    lib = krl.load_library()
    f = lib.krl_emission_cdf_noalloc
    f.restype = C.c_int
    f.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]
    return lib


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _problem(rate):
    p = W.box(n=4, tau0=1.0)
    nz, ny, nx = rate.shape
    return dataclasses.replace(p, shape=rate.shape, opacity=np.ones(rate.shape, np.float32),
                               source=dataclasses.replace(p.source, rate=rate))


def _reference_cdf(krl, rate):
    g = krl.Grid(_problem(rate))
    try:
        return g.tally("src_cdf").cpu().numpy()
    finally:
        g.close()


def test_noalloc_cdf_matches_the_allocating_path_on_two_calls():
    krl = need_gpu()
    import torch
    lib = _lib(krl)
    rng = np.random.default_rng(2608)
    big = rng.gamma(2.0, 1.0, size=(40, 40, 40)).astype(np.float32)
    big[big < 0.3] = 0.0                                   # some empty cells
    small = rng.uniform(0.0, 5.0, size=(17, 19, 23)).astype(np.float32)   # ragged, < 1 scan block per row
    # 2,080,000 cells: 1016 scan blocks of 2048 cells, the last one ragged, so
    # that each thread of the block-offset pass sums several block totals
    huge = rng.exponential(1.0, size=(130, 125, 128)).astype(np.float32)
    for rate in (big, small, huge):                        # later calls reuse the earlier calls' scratch
        ref = _reference_cdf(krl, rate)
        r = torch.from_numpy(rate.reshape(-1)).cuda()
        out = torch.full((rate.size,), float("nan"), dtype=torch.float64, device="cuda")
        rc = lib.krl_emission_cdf_noalloc(C.c_void_p(r.data_ptr()), rate.size, C.c_void_p(out.data_ptr()), _stream())
        assert rc == krl.KRL_OK, lib.krl_last_error()
        got = out.cpu().numpy()
        assert np.allclose(got, ref, rtol=1e-13, atol=1e-15)
        assert got[-1] == 1.0 and np.all(np.diff(got) >= 0)
        # and against the definition itself: the FP64 running sum of the rates
        # over their total (numpy, independent of both device paths)
        cs = np.cumsum(rate.reshape(-1).astype(np.float64))
        assert np.allclose(got, cs / cs[-1], rtol=1e-12, atol=1e-15)


def test_noalloc_rejects_sizes_beyond_its_fixed_scratch():
    krl = need_gpu()
    import torch
    lib = _lib(krl)
    r = torch.ones(8, dtype=torch.float32, device="cuda")
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    for n in ((1 << 27) + 1, 0, -5):
        rc = lib.krl_emission_cdf_noalloc(C.c_void_p(r.data_ptr()), n, C.c_void_p(out.data_ptr()), _stream())
        assert rc == krl.KRL_ERR_ARG
        assert b"outside [1, 134217728]" in lib.krl_last_error()
    assert lib.krl_emission_cdf_noalloc(None, 8, C.c_void_p(out.data_ptr()), _stream()) == krl.KRL_ERR_ARG
    bad = torch.tensor([1.0, -1.0, 2.0], dtype=torch.float32, device="cuda")
    out3 = torch.zeros(3, dtype=torch.float64, device="cuda")
    assert lib.krl_emission_cdf_noalloc(C.c_void_p(bad.data_ptr()), 3, C.c_void_p(out3.data_ptr()),
                                        _stream()) == krl.KRL_ERR_NUMERIC
