"""Pins of the oracle's channel-map ray trace (Eq. imaging-formal,
Eq. imaging-alphas) against closed forms."""
import math

import numpy as np

import workloads as W
from oracle import raytrace as RT


def _cube(n=6, tau=0.0, nch=5):
    p = W.envelope(n=n, n_ch=nch, n_packets=1)
    p.opacity_kind = "tau"
    p.opacity = np.full((n, n, n), tau, np.float32)
    p.vel_cms = None
    return p


def test_thin_limit_is_the_line_integral(oracle_mod):
    """alpha = 0: I = sum of j over the chord; face-on through a cube the chord
    is the side length."""
    p = _cube(tau=0.0)
    ncell, nch = 6 ** 3, p.channels[2]
    j = np.arange(1, nch + 1, dtype=np.float64)[None, :] * np.ones((ncell, 1))
    maps = RT.trace_maps(oracle_mod, p, j, camera=0, npix_x=4, npix_y=4, fov=6.0)   # camera 0: theta = 0
    assert np.allclose(maps, 6.0 * np.arange(1, nch + 1)[:, None, None], rtol=1e-12)


def test_uniform_source_function(oracle_mod):
    """Constant S in a uniform static cube (j_k = S alpha_k): I = S (1 - e^{-tau_k})
    with tau_k = alpha0 H(a, x_k) L along the ray."""
    from oracle import tables as T
    tau_cell = 0.7
    p = _cube(tau=tau_cell)
    d = oracle_mod.derive(p)
    tb = oracle_mod.line_tables(float(d["a"]), False)
    vmin, dv, nch = p.channels
    xk = -(vmin + (np.arange(nch) + 0.5) * dv) / d["b"]
    H = T.voigt_lookup(xk, d["a"], tb["voigt_lnH"], tb["voigt_H0"])
    S = 2.5
    alpha = float(np.float32(tau_cell)) * H
    j = np.tile(S * alpha, (6 ** 3, 1))
    for cam in range(3):
        maps = RT.trace_maps(oracle_mod, p, j, camera=cam, npix_x=3, npix_y=3, fov=2.0)
        n, _, _ = RT.camera_basis(*p.cameras[cam])
        L = 6.0 / max(abs(n))               # chord through the centre region along n
        if abs(max(abs(n)) - 1) < 1e-12:
            expect = S * (1 - np.exp(-alpha * L))
            assert np.allclose(maps[:, 1, 1], expect, rtol=1e-10)
        assert np.all(maps <= S * (1 + 1e-12)) and np.all(maps >= 0)


def test_segments_cover_the_chord(oracle_mod):
    n, u, v = RT.camera_basis(math.radians(45.0), 0.3)
    cells, lens = RT.ray_segments(oracle_mod, (8, 8, 8), (False,) * 3, np.array([4.0, 4.0, 4.0]), n)
    t = [(0.0 - 4.0) / c if c < 0 else (8.0 - 4.0) / c for c in n]
    # the chord through the centre is twice the distance to the first face
    assert abs(lens.sum() - 2 * min(t)) < 1e-9
