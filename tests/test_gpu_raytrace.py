"""GPU channel-map ray trace against the FP64 oracle trace on the same
emissivity (criterion: max |I - I_ref| / max(|I_ref|, 1e-3 max I_ref) <= 1e-5),
and the full two-step chain on the thin moving slab (Eq. thin-slab)."""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import raytrace as RT
from _gpu_common import need_gpu

pytestmark = pytest.mark.gpu


def _crit(got, ref):
    ref = np.asarray(ref, dtype=np.float64)
    den = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max())
    return np.max(np.abs(np.asarray(got, dtype=np.float64) - ref) / den)


def test_raytrace_matches_fp64_on_the_mc_emissivity():
    krl = need_gpu()
    import torch
    p = W.envelope(n=16, n_ch=16, n_packets=20000)
    g = krl.Grid(p)
    try:
        g.run(precision=krl.KRL_PREC_FP32, want_stats=False)
        em = g.tally("emiss").reshape(len(p.cameras), p.ncell, p.channels[2])
        jline = torch.from_numpy((1e-3 * p.source.rate.reshape(-1)).astype(np.float32)).cuda()
        for m in range(len(p.cameras)):
            for jl in (None, jline):
                ref = RT.trace_maps(oracle, p, em[m].cpu().numpy(), camera=m, npix_x=24, npix_y=20, fov=17.0,
                                    jline=None if jl is None else jl.cpu().numpy())
                assert np.abs(ref).max() > 0
                # with the per-camera extinction cube, and without (profile per segment)
                for ns in (False, True):
                    maps = g.raytrace(m, 24, 20, fov_cells=17.0, jline=jl, no_scratch=ns).cpu().numpy()
                    assert _crit(maps, ref) <= 1e-5, (m, jl is None, ns, _crit(maps, ref))
        # an explicit direction with a caller emissivity buffer
        th, ph = math.radians(30.0), math.radians(70.0)
        maps = g.raytrace(-1, 9, 11, fov_cells=20.0, emiss=em[0].contiguous(), theta=th, phi=ph).cpu().numpy()
        q = W.envelope(n=16, n_ch=16, n_packets=1)
        q.cameras = ((th, ph),)
        ref = RT.trace_maps(oracle, q, em[0].cpu().numpy(), camera=0, npix_x=9, npix_y=11, fov=20.0)
        assert _crit(maps, ref) <= 1e-5
    finally:
        g.close()


def test_thin_slab_two_step_chain():
    """MC emissivity + ray trace through the face-on camera: the image carries
    the volume-integrated emissivity (thin slab), peaked at v = -v_z with the
    thermal shape of Eq. thin-slab."""
    krl = need_gpu()
    p = W.thin_slab(n_packets=200000)
    g = krl.Grid(p)
    try:
        g.run(precision=krl.KRL_PREC_FP32, want_stats=False)
        em = g.tally("emiss").cpu().numpy().reshape(p.ncell, -1).astype(np.float64)
        npx = 32
        fov = float(p.shape[2])
        maps = g.raytrace(0, npx, npx, fov_cells=fov).cpu().numpy().astype(np.float64)
        b = g.info.b_cms
    finally:
        g.close()
    pix_area = (fov / npx) ** 2
    img = maps.sum(axis=(1, 2)) * pix_area          # integrated over the image
    vol = em.sum(axis=0)                            # volume-integrated emissivity
    assert np.allclose(img, vol, rtol=0.01)
    vmin, dv, nch = p.channels
    v = vmin + (np.arange(nch) + 0.5) * dv
    shape = np.exp(-((v + 1e5) / b) ** 2)
    assert abs(v[np.argmax(img)] + 1e5) <= dv
    assert np.max(np.abs(img / img.sum() - shape / shape.sum())) / np.max(shape / shape.sum()) < 0.02


@pytest.mark.parametrize("n_ch,offset", [(3, 0), (8, 0), (20, 0), (33, 0), (64, 0), (64, 1), (100, 0), (128, 0)])
def test_channel_counts_and_lane_groups(n_ch, offset):
    """Every lanes-per-ray variant of the trace (1 .. 32 lanes, 4 channels
    each; ragged channel counts, and channel counts that fill every lane,
    read as one 16-byte vector per lane) and the per-segment fallback, on a
    random emissivity through a moving envelope, against the FP64 trace.
    offset = 1: the emissivity starts 4 bytes past a 16-byte boundary, so a
    full channel count takes the unvectorised reads."""
    krl = need_gpu()
    import torch
    p = W.envelope(n=12, n_ch=n_ch, n_packets=1)
    rng = np.random.default_rng(n_ch)
    em_host = rng.random((p.ncell, n_ch), dtype=np.float32)
    buf = torch.zeros(p.ncell * n_ch + 4, dtype=torch.float32, device="cuda")
    em = buf[offset:offset + p.ncell * n_ch].view(p.ncell, n_ch)
    em.copy_(torch.from_numpy(em_host))
    assert (em.data_ptr() % 16 == 0) == (offset == 0)
    th, ph = math.radians(40.0), math.radians(25.0)
    q = W.envelope(n=12, n_ch=n_ch, n_packets=1)
    q.cameras = ((th, ph),)
    ref = RT.trace_maps(oracle, q, em.cpu().numpy(), camera=0, npix_x=13, npix_y=11, fov=14.0)
    g = krl.Grid(p)
    try:
        for ns in (False, True):
            maps = g.raytrace(-1, 13, 11, fov_cells=14.0, emiss=em, theta=th, phi=ph, no_scratch=ns).cpu().numpy()
            assert maps.shape == (n_ch, 11, 13)
            assert _crit(maps, ref) <= 1e-5, (n_ch, ns, _crit(maps, ref))
    finally:
        g.close()


def test_full_size_maps_against_fp64_on_sampled_pixels():
    """The benchmark's imaging workload at full size: the 256^3 rotating,
    infalling envelope, 64 channels over +-5 km/s, its emissivity cube
    filled by 1e6 Monte Carlo packets, channel maps of 1024^2 pixels at the
    three inclinations. For each camera, 8 pixel rows spread over the image
    (64 pixels each, every 16th) against the FP64 oracle trace on the same
    emissivity cube (Eq. imaging-formal, imaging-alphas): the criterion
    max |I - I_ref| / max(|I_ref|, 1e-3 max I_ref) <= 1e-5, and the plain
    relative error of every sampled pixel brighter than 1e-7 of the
    camera's peak, reported and held below 1e-4."""
    krl = need_gpu()
    import torch
    from _gpu_common import report
    p = W.envelope(n=256, n_ch=64, n_packets=1_000_000)
    npx = 1024
    rows = [int(npx * (k + 0.5) / 8) for k in range(8)]
    cols = list(range(8, npx, 16))
    pix = [(ix, iy) for iy in rows for ix in cols]
    g = krl.Grid(p)
    try:
        g.run(want_stats=False)
        torch.cuda.synchronize()
        em = g.tally("emiss").reshape(len(p.cameras), p.ncell, p.channels[2])
        for m in range(len(p.cameras)):
            maps = g.raytrace(m, npx, npx, fov_cells=256.0).cpu().numpy()
            got = np.stack([maps[:, iy, ix] for ix, iy in pix], axis=1)
            ref_maps = RT.trace_maps(oracle, p, em[m].cpu().numpy(), camera=m, npix_x=npx, npix_y=npx,
                                     fov=256.0, pixels=pix)
            ref = np.stack([ref_maps[:, iy, ix] for ix, iy in pix], axis=1)
            peak = np.abs(maps).max()
            crit = _crit(got, ref)
            bright = np.abs(ref) > 1e-7 * peak
            rel = float(np.max(np.abs(got[bright] - ref[bright]) / np.abs(ref[bright]))) if bright.any() else 0.0
            report("raytrace_full_size_vs_fp64", camera=m, pixels=len(pix), criterion=crit,
                   plain_rel_bright=rel, bright_fraction=float(bright.mean()))
            assert ref.max() > 0
            assert crit <= 1e-5, (m, crit)
            assert rel <= 1e-4, (m, rel)
    finally:
        g.close()
