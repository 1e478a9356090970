"""O-exact: the static-slab walk with every table replaced by direct FP64
evaluation, to measure the table error of the tabulated method (reported,
not gated: the comparison is statistical).

TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg may import this module.

What differs from the tabulated oracle walk (transport.c):
  * H(a, x) is the Faddeeva function's real part, Re w(x + i a) (scipy),
    instead of the interpolated Voigt slice;
  * the parallel velocity of the scattering atom is drawn exactly from
    p(u | x) ~ exp(-u^2) / ((u - x)^2 + a^2) (Sec. 2.1.1) by rejection
    sampling, instead of inverting the tabulated log-CDF;
  * the slab is continuous (no cells; the medium is uniform, so the cell
    walk of the tabulated oracle changes nothing but rounding);
  * random numbers come from numpy's PCG64, since the comparison is
    statistical.
The rest is the same method: exponential free paths, isotropic emission and
scattering directions, x_out = x_in + u_par (g - 1) + u_perp sin(gamma) with
u_perp ~ N(0, 1/2) (Eq. riia-scatter), escape through either face.

The exact sampler (x >= 0; x < 0 by u -> -u). For a split point s, either
s <= x, with envelope
  u <  s:  exp(-u^2) L(s)            (|u - x| >= x - s, so L(u) <= L(s)),
  u >= s:  c(s) L(u), c(s) = exp(-max(s, 0)^2)  (exp(-u^2) <= c(s)),
where L(u) = 1 / ((u - x)^2 + a^2); or s = -inf, envelope L(u) alone. The
first piece is drawn as a Gaussian N(0, 1/2) over all u (so its mass is
L(s) sqrt(pi); draws at u >= s are rejected), the second as a Lorentzian
truncated to u >= s (u = x + a tan(theta), theta uniform); a proposal is
accepted with probability (target restricted to its piece) / envelope.
Every choice of s gives exactly p(u | x); s only sets the acceptance rate,
so each draw takes the s of a short candidate list with the smallest
envelope mass.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import wofz

_SQRT_PI = math.sqrt(math.pi)
_FRACTIONS = np.array([0.0, 0.25, 0.5, 0.7, 0.8, 0.9, 0.95, 0.98, 0.99])


def voigt_H(a: float, x):
    """H(a, x) = Re w(x + i a)."""
    return wofz(np.asarray(x, dtype=np.float64) + 1j * a).real


def _envelope(x, a, s):
    """Masses of the two envelope pieces for split s (s = -inf: Lorentzian
    only) at x >= 0."""
    with np.errstate(over="ignore", invalid="ignore"):
        # the Gaussian piece's envelope is exp(-u^2) L(s) over all u (its
        # proposals at u >= s are rejected), so its mass is L(s) sqrt(pi)
        gauss = np.where(np.isfinite(s), _SQRT_PI / ((x - s) ** 2 + a * a), 0.0)
        th = np.where(np.isfinite(s), np.arctan((s - x) / a), -math.pi / 2)
        c = np.exp(-np.maximum(np.where(np.isfinite(s), s, 0.0), 0.0) ** 2)
        lor = c * (math.pi / 2 - th) / a
    return gauss, lor, th, c


def sample_upar(x, a: float, rng: np.random.Generator) -> np.ndarray:
    """Exact draws of u_par from p(u | x), one per element of x."""
    x = np.asarray(x, dtype=np.float64)
    sgn = np.where(x < 0.0, -1.0, 1.0)
    ax = np.abs(x)
    # split point per element: the candidate with the smallest envelope mass
    cand = np.concatenate([np.full((1, ax.size), -np.inf), _FRACTIONS[:, None] * ax[None, :]])
    g, l, _, _ = _envelope(ax[None, :], a, cand)
    s = cand[np.argmin(g + l, axis=0), np.arange(ax.size)]
    mg, ml, th_s, c = _envelope(ax, a, s)
    p_gauss = mg / (mg + ml)
    out = np.empty_like(ax)
    todo = np.arange(ax.size)
    while todo.size:
        xs, ss, ts, cs, pg = ax[todo], s[todo], th_s[todo], c[todo], p_gauss[todo]
        n = todo.size
        u = np.empty(n)
        acc = np.zeros(n, dtype=bool)
        pick_g = rng.random(n) < pg
        # Gaussian piece: N(0, 1/2); accept below s with L(u) / L(s)
        ig = np.nonzero(pick_g)[0]
        if ig.size:
            ug = rng.normal(0.0, math.sqrt(0.5), ig.size)
            ok = ug < ss[ig]
            lu = 1.0 / ((ug - xs[ig]) ** 2 + a * a)
            ls = 1.0 / ((xs[ig] - ss[ig]) ** 2 + a * a)
            ok &= rng.random(ig.size) * ls < lu
            u[ig] = ug
            acc[ig] = ok
        # Lorentzian piece: theta uniform on (theta_s, pi/2); accept with exp(-u^2) / c(s)
        il = np.nonzero(~pick_g)[0]
        if il.size:
            th = ts[il] + (math.pi / 2 - ts[il]) * rng.random(il.size)
            ul = xs[il] + a * np.tan(th)
            ok = rng.random(il.size) * cs[il] < np.exp(-ul * ul)
            u[il] = ul
            acc[il] = ok
        out[todo[acc]] = u[acc]
        todo = todo[~acc]
    return sgn * out


def slab_spectrum(tau0: float, a: float, n_packets: int, seed: int, bins: tuple) -> np.ndarray:
    """Escaped-photon counts of the static slab (half-thickness line-centre
    depth tau0, line-centre photons emitted isotropically at the midplane)
    on (lo, hi, n) bins of x, plus under- and overflow: [n + 2]."""
    rng = np.random.default_rng(seed)
    lo, hi, nb = bins
    z = np.zeros(n_packets)                     # height above the midplane, in units of the half-thickness
    mu = 2.0 * rng.random(n_packets) - 1.0
    x = np.zeros(n_packets)
    counts = np.zeros(nb + 2, dtype=np.int64)
    live = np.arange(n_packets)
    while live.size:
        zl, ml, xl = z[live], mu[live], x[live]
        tau = -np.log(rng.random(live.size))
        zn = zl + ml * tau / (tau0 * voigt_H(a, xl))
        esc = np.abs(zn) >= 1.0
        if esc.any():
            xe = xl[esc]
            k = np.where(xe < lo, 0, np.where(xe >= hi, nb + 1,
                                              1 + np.minimum(((xe - lo) / (hi - lo) * nb).astype(np.int64), nb - 1)))
            np.add.at(counts, k, 1)
        keep = ~esc
        live, zl, ml, xl, zn = live[keep], zl[keep], ml[keep], xl[keep], zn[keep]
        if not live.size:
            break
        # scattering at zn: atom velocity, new direction, outgoing frequency
        upar = sample_upar(xl, a, rng)
        mu2 = 2.0 * rng.random(live.size) - 1.0
        dphi = 2.0 * math.pi * rng.random(live.size)
        g = ml * mu2 + np.sqrt(np.maximum(0.0, 1.0 - ml * ml)) * np.sqrt(np.maximum(0.0, 1.0 - mu2 * mu2)) * np.cos(dphi)
        uperp = rng.normal(0.0, math.sqrt(0.5), live.size)
        x[live] = xl + upar * (g - 1.0) + uperp * np.sqrt(np.maximum(0.0, 1.0 - g * g))
        z[live] = zn
        mu[live] = mu2
    return counts
