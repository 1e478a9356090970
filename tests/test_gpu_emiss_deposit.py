"""Two-stage emissivity deposit of the FP32 walk (Eq. scat-line): the walk
records each segment, then one warp per segment adds that segment's channels
for every camera. Checked against the deposit inside the walk on the same
packets (identical walks; the cube equal up to the order of the FP32 atomic
additions), with a segment buffer that overflows part way (the walk deposits
the rest), on a moving grid and a static one (the two instantiations of the
second stage), and through the R_IIA wing limit (Eq. riia-inf, |x_com| >=
120) against the oracle."""
import dataclasses
import math

import numpy as np
import pytest

import oracle
import workloads as W
from _gpu_common import agreement, gpu_run, need_gpu, rel_l1

pytestmark = pytest.mark.gpu


def _wing_slab(n_packets=20000):
    """The thin slab's line-centre beam (travelling along +x in the slab
    layer, camera along +z, g = 0) with the slab cells beyond the first
    column moving at -130 b along x: the beam, emitted at rest, meets them at
    x_com = 130, in the wing limit of the redistribution kernel. Channels
    cover x_out in [120, 140]."""
    p = W.thin_slab(n_packets=n_packets)
    vel = np.zeros_like(p.vel_cms)
    vel[0, 1, :, 1:] = -130e5                  # b = 1 km/s
    return dataclasses.replace(p, name="thin_slab_wing", vel_cms=vel, channels=(-140e5, 20e5 / 32, 32))


def _static_envelope():
    p = W.envelope(n=16, n_ch=16, n_packets=20000)
    return dataclasses.replace(p, name="envelope_static", vel_cms=None)


CASES = {
    "envelope_moving": W.envelope(n=16, n_ch=16, n_packets=20000),
    "envelope_static": _static_envelope(),
    "thin_slab_wing": _wing_slab(),
}


def _same_cube(a, b):
    a = a.astype(np.float64)
    b = b.astype(np.float64)
    assert np.abs(a - b).sum() <= 1e-5 * np.abs(a).sum()
    assert np.allclose(a, b, rtol=1e-3, atol=1e-6 * np.abs(a).max())


@pytest.mark.parametrize("name", list(CASES))
def test_two_stage_matches_in_walk_deposit(name):
    krl = need_gpu()
    p = CASES[name]
    runs = {r: gpu_run(krl, p, krl.KRL_PREC_FP32, emiss_records=r) for r in (-1, 0, 1000)}
    base = runs[-1]
    assert base["emiss"] is not None and np.abs(base["emiss"]).sum() > 0
    for r in (0, 1000):
        out = runs[r]
        for f in base["records"].dtype.names:
            assert np.array_equal(out["records"][f], base["records"][f]), (r, f)
        assert np.array_equal(out["spec_n"], base["spec_n"])
        _same_cube(base["emiss"], out["emiss"])
        for k in ("exc", "J"):
            if base[k] is not None:
                assert np.allclose(out[k], base[k], rtol=1e-9, atol=1e-12 * np.abs(base[k]).max())


def test_wing_limit_against_the_oracle():
    """FP64 walk in lockstep and the FP32 two-stage deposit, both against the
    oracle's cube: every segment beyond the first column deposits through
    Eq. riia-inf."""
    krl = need_gpu()
    p = CASES["thin_slab_wing"]
    ref = oracle.run(p, records=True)
    re_ = ref["emiss"].astype(np.float64)
    assert re_.sum() > 0
    f64 = gpu_run(krl, p, krl.KRL_PREC_FP64)
    ok = agreement(f64["records"], ref["records"])
    assert ok.mean() >= 0.999
    e64 = f64["emiss"].reshape(re_.shape).astype(np.float64)
    if ok.all():
        assert np.allclose(e64, re_, rtol=1e-3, atol=1e-6 * re_.max())
    assert rel_l1(e64, re_) < 1e-3, rel_l1(e64, re_)
    f32 = gpu_run(krl, p, krl.KRL_PREC_FP32)
    assert agreement(f32["records"], ref["records"], strict=False).mean() >= 0.999
    e32 = f32["emiss"].reshape(re_.shape).astype(np.float64)
    assert rel_l1(e32, re_) < 1e-3, rel_l1(e32, re_)
    # the wing cells carry the deposit: x_out - x_com spans the channel band
    ncell = p.shape[0] * p.shape[1] * p.shape[2]
    per_cell = re_.reshape(ncell, -1).sum(axis=1).reshape(p.shape)
    assert per_cell[1, :, 1:].sum() > 0.5 * per_cell.sum()


def test_emiss_records_is_validated():
    krl = need_gpu()
    g = krl.Grid(CASES["envelope_moving"])
    try:
        with pytest.raises(krl.KrlError):
            g.run(n=10, emiss_records=-2)
    finally:
        g.close()


def test_channel_sum_is_the_path_length_estimator():
    """The two-stage cube summed over channels (times the channel width in
    x and 4 pi) equals alpha0 times the excitation tally, per camera and
    cell, and the scattering map agrees with it within counting noise (the
    oracle's pin of the same identity is in test_oracle_walk.py)."""
    krl = need_gpu()
    p = W.box(tau0=2.0, n=8, T_K=100.0, n_packets=200_000, tallies=("emiss", "exc", "scatmap"))
    b = math.sqrt(2.0 * 1.380649e-16 * 100.0 / (W.HYDROGEN_AMU * 1.66053906660e-24))
    p = dataclasses.replace(p, channels=(-14.0 * b, 0.25 * b, 112),
                            cameras=((0.0, 0.0), (math.pi / 2, 0.0), (math.pi / 3, 1.0)))
    out = gpu_run(krl, p, krl.KRL_PREC_FP32, records=False)
    em = out["emiss"].reshape(3, p.ncell, 112).astype(np.float64)
    S = em.sum(axis=2) * 0.25 * 4.0 * math.pi
    P = p.opacity.reshape(-1).astype(np.float64) * out["exc"]
    assert np.all(np.abs(S.sum(axis=1) / P.sum() - 1.0) < 1e-3)
    assert np.all(np.abs(S / P - 1.0) < 5e-3)
    n_scat = float(out["scatmap"].sum())
    assert abs(n_scat - P.sum()) < 4.0 * math.sqrt(n_scat), (n_scat, P.sum())

