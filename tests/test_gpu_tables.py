"""The device-built FP64 tables (stored float32) equal the oracle's
element by element (Sec. 2.1.1, Eq. riia-table, the ph_mode 2 Voigt slice)."""
import dataclasses

import numpy as np
import pytest

import workloads as W
from oracle import tables as OT
from _gpu_common import need_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("a", [1e-2, 4.7e-4, 0.149, 1e-4, 1.55e-13])
def test_tables_match_oracle(a):
    krl = need_gpu()
    p = W.thin_slab()
    p.line = dataclasses.replace(p.line, a_fixed=a)
    g = krl.Grid(p)
    try:
        lnH = g.tally("voigt").cpu().numpy()
        H0 = g.tally("H0").cpu().numpy()[0]
        usx = g.tally("us_x").cpu().numpy()
        lnc = g.tally("us_lncdf").cpu().numpy().reshape(40, 251)
        rt = g.tally("rtab").cpu().numpy().reshape(40, 200, 201)
        assert abs(g.info.a - a) < 1e-15
    finally:
        g.close()
    ref_lnH, ref_H0 = OT.voigt_table(a)
    assert np.allclose(lnH, ref_lnH, rtol=3e-7, atol=1e-7)
    assert abs(H0 / ref_H0 - 1) < 2e-7
    rx, rlnc = OT.usampler_table(a)
    assert np.array_equal(usx, rx) or np.allclose(usx, rx, rtol=2e-7, atol=0)
    assert np.allclose(lnc, rlnc, rtol=1e-6, atol=1e-6)
    rrt = OT.rtable(a)
    assert np.allclose(rt, rrt, rtol=1e-5, atol=1e-9 * rrt.max())


def test_cell_records_and_source_cdf():
    """Per-cell records {alpha0 dx, V/b} (Eq. sigma0, Sec. 2.2.1), destruction
    probabilities (Eq. eps) and the emission CDF, vs the oracle's derivation."""
    krl = need_gpu()
    import oracle
    p = W.envelope(n=16, n_ch=8, n_packets=10)
    g = krl.Grid(p)
    try:
        cells = g.tally("cells").cpu().numpy().reshape(-1, 4)
        eps = g.tally("eps").cpu().numpy()
        cdf = g.tally("src_cdf").cpu().numpy()
        info = g.info
    finally:
        g.close()
    d = oracle.derive(p)
    assert abs(info.b_cms / d["b"] - 1) < 1e-14
    assert np.allclose(cells[:, 0], d["tau0"], rtol=1e-7, atol=0)
    assert np.allclose(cells[:, 1:], d["vel"], rtol=1e-7, atol=1e-7)
    assert np.allclose(eps, d["eps"], rtol=1e-7, atol=0)
    assert np.allclose(cdf, d["cdf"], rtol=1e-13, atol=1e-15)
    assert cdf[-1] == 1.0
