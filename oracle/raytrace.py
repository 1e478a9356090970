"""FP64 oracle of the channel-map ray trace (Sec. 2.2.2, Eq. imaging-formal,
Eq. imaging-alphas).

TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg may import this module.

Orthographic camera (reading): pixel-centred parallel rays along the camera
direction n_cam, image axes u = e_theta, v = e_phi of (theta, phi), image
centred on the box centre, width fov cells, I_in = 0 where the ray enters.
Per cell segment of length dl and channel k with gas-frame frequency
x_k = -(v_k / b) - n_cam . V / b:

    alpha_k = alpha0 H(a, x_k) + alpha_abs,   dtau = alpha_k dl,
    I_out = I_in exp(-dtau) + S_k (1 - exp(-dtau)),
    S_k = (j_sca,k + j_line H(a, x_k) / sqrt(pi)) / alpha_k,

written as I_out = I_in e^{-dtau} + j_k dl (1 - e^{-dtau}) / dtau so that
an empty cell (alpha = 0) adds j dl. alpha_abs is the continuum absorption
(zero without one): the two-step scheme applies it in this formal solution
(Sec. 3.2), the continuum adding extinction but no emission. The cell walk
is the oracle's own (orc_trace in transport.c).
"""
from __future__ import annotations

import math

import numpy as np

from . import tables as T

SQRT_PI = math.sqrt(math.pi)


def camera_basis(theta: float, phi: float):
    n = np.array([math.sin(theta) * math.cos(phi), math.sin(theta) * math.sin(phi), math.cos(theta)])
    u = np.array([math.cos(theta) * math.cos(phi), math.cos(theta) * math.sin(phi), -math.sin(theta)])
    v = np.array([-math.sin(phi), math.cos(phi), 0.0])
    return n, u, v


def _entry(shape, P, n):
    """Parameter interval [t0, t1] where P + t n lies inside the box."""
    nz, ny, nx = shape
    hi = np.array([nx, ny, nz], dtype=np.float64)
    t0, t1 = -np.inf, np.inf
    for d in range(3):
        if n[d] != 0.0:
            a, b = (0.0 - P[d]) / n[d], (hi[d] - P[d]) / n[d]
            t0, t1 = max(t0, min(a, b)), min(t1, max(a, b))
        elif not (0.0 <= P[d] < hi[d]):
            return None
    return (t0, t1) if t1 > t0 else None


def ray_segments(oracle_mod, shape, periodic, P, n):
    """(cells, lengths) of the ray P + t n, t increasing, through the box."""
    iv = _entry(shape, P, n)
    if iv is None:
        return np.zeros(0, np.int64), np.zeros(0)
    nz, ny, nx = shape
    X = np.clip(P + iv[0] * n, 0.0, np.array([nx, ny, nz], dtype=np.float64))
    return oracle_mod.trace(shape, (False, False, False), X, n)


def trace_maps(oracle_mod, problem, emiss, camera: int, npix_x: int, npix_y: int, fov: float,
               jline=None, pixels=None):
    """Channel maps [n_ch][npix_y][npix_x] (FP64) for the given emissivity
    [ncell][n_ch] (raw code units). `pixels`: optional list of (ix, iy) to
    compute only those (others stay 0)."""
    d = oracle_mod.derive(problem)
    tb = oracle_mod.line_tables(float(d["a"]), False)
    lnH, H0 = tb["voigt_lnH"], tb["voigt_H0"]
    vmin, dv, nch = problem.channels
    b = d["b"]
    th, ph = problem.cameras[camera]
    n, u, v = camera_basis(th, ph)
    nz, ny, nx = problem.shape
    C = np.array([nx, ny, nz], dtype=np.float64) / 2.0
    x0 = -(vmin + (np.arange(nch) + 0.5) * dv) / b          # -v_k / b
    vel = d["vel"]
    tau0 = d["tau0"]
    tau_abs = d["tau_abs"]                                   # continuum opacity, or None
    em = np.asarray(emiss).reshape(-1, nch)                 # rows taken to FP64 one segment at a time
    jl = None if jline is None else np.asarray(jline, dtype=np.float64).reshape(-1)
    pix_h = fov / npix_x
    out = np.zeros((nch, npix_y, npix_x))
    todo = pixels if pixels is not None else [(i, j) for j in range(npix_y) for i in range(npix_x)]
    for (ix, iy) in todo:
        uc = (ix + 0.5) * pix_h - 0.5 * fov
        vc = (iy + 0.5) * pix_h - 0.5 * pix_h * npix_y
        P = C + uc * u + vc * v
        cells, lens = ray_segments(oracle_mod, problem.shape, problem.periodic, P, n)
        I = np.zeros(nch)
        for c, dl in zip(cells, lens):                      # along n: far side first
            vn = 0.0 if vel is None else float(n @ vel[c])
            xk = x0 - vn
            H = T.voigt_lookup(xk, d["a"], lnH, H0)
            alpha = tau0[c] * H
            if tau_abs is not None:                         # line plus continuum extinction
                alpha = alpha + tau_abs[c]
            dtau = alpha * dl
            j = em[c].astype(np.float64)
            if jl is not None:
                j = j + jl[c] * H / SQRT_PI
            e = np.exp(-dtau)
            with np.errstate(invalid="ignore", divide="ignore"):
                f = np.where(dtau > 1e-12, -np.expm1(-dtau) / dtau, 1.0 - 0.5 * dtau)
            I = I * e + j * dl * f
        out[:, iy, ix] = I
    return out
