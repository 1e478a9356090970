"""FP64 oracle: line physics and sampling tables, written from the paper.

TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg may import this module. The product path never does.

Everything here is plain FP64 numpy/scipy. Tables are rounded to float32 at
the end because the method stores its sampling tables in single precision
after building them in double precision (Sec. 2.3, 2.3.1).

Contents and the passages they follow:

* ``doppler_b``, ``nu_D``, ``damping_a``   - Sec. 2.1, Eq. xdef and the
  definition a = A_ul / (4 pi nu_D).
* ``sigma0``                               - Eq. sigma0.
* ``epsilon``                              - Eq. eps.
* ``voigt_H``                              - the Voigt function H(a, x)
  (Sec. 2.1), as Re w(x + i a) with scipy's Faddeeva routine.
* ``voigt_table`` / ``voigt_lookup``       - the 1-D log-frequency Voigt table
  of ph_mode 2 (Sec. 2.2.1, 2.3.1). Grid and interpolation are a reading
  (the paper gives only "5000 points in logarithmic frequency").
* ``voigt2d_*`` / ``blend_*``              - the ph_mode 1 two-dimensional
  Voigt table and the ph_mode 3 core-wing blend (Sec. 2.3.1).
* ``usampler_*``                           - the velocity sampler p(u_par | x_in)
  (Sec. 2.1.1): 40 x-nodes, 251 u-nodes on [-6, 6], log of the normalised
  cumulative distribution.
* ``rtable`` / ``r_lookup`` / ``r_inf``    - the discrete R_IIA kernel table
  (Eq. riia-table) and its asymptotic form (Eq. riia-inf).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import wofz

# Physical constants (CGS, CODATA 2018).
K_B = 1.380649e-16
C_LIGHT = 2.99792458e10
AMU = 1.66053906660e-24
SQRT_PI = math.sqrt(math.pi)

# ---------------------------------------------------------------- line physics


def doppler_b(T_K: float, mass_amu: float) -> float:
    """Thermal Doppler width b = (2 k T / m)^(1/2) [cm/s] (Sec. 2.1)."""
    return math.sqrt(2.0 * K_B * T_K / (mass_amu * AMU))


def nu_D(nu0: float, b: float) -> float:
    """Doppler frequency width nu_D = nu0 b / c (Eq. xdef)."""
    return nu0 * b / C_LIGHT


def damping_a(A_ul: float, nu0: float, b: float) -> float:
    """Damping parameter a = A_ul / (4 pi nu_D) (Sec. 2.1)."""
    return A_ul / (4.0 * math.pi * nu_D(nu0, b))


def sigma0(g_u: float, g_l: float, A_ul: float, nu0: float, b: float) -> float:
    """Line-centre cross section per lower-level molecule (Eq. sigma0):
    sigma0 = (g_u/g_l) A c^3 / (8 pi^{3/2} nu0^3 b)."""
    return (g_u / g_l) * A_ul * C_LIGHT ** 3 / (8.0 * math.pi ** 1.5 * nu0 ** 3 * b)


def epsilon(k_ul: float, n_coll, A_ul: float):
    """Collisional destruction probability per scattering (Eq. eps)."""
    q = k_ul * np.asarray(n_coll, dtype=np.float64)
    return q / (A_ul + q)


# ---------------------------------------------------------------- Voigt


def voigt_H(a: float, x):
    """Voigt function H(a, x) = (a/pi) int exp(-y^2) / ((x-y)^2 + a^2) dy,
    evaluated as the real part of the Faddeeva function w(x + i a)."""
    return wofz(np.asarray(x, dtype=np.float64) + 1j * a).real


VOIGT_N = 5000
VOIGT_LOG10_MIN = -4.0
VOIGT_LOG10_MAX = 3.0


def voigt_table(a: float):
    """ph_mode 2 Voigt slice at one damping parameter (reading): 5000 nodes
    uniform in log10|x| over [-4, 3]; the table holds ln H at the nodes,
    stored as float32. Returns (lnH[5000] float32, H(a,0) as float32)."""
    l = VOIGT_LOG10_MIN + (VOIGT_LOG10_MAX - VOIGT_LOG10_MIN) * np.arange(VOIGT_N) / (VOIGT_N - 1)
    lnH = np.log(voigt_H(a, 10.0 ** l)).astype(np.float32)
    return lnH, np.float32(voigt_H(a, 0.0))


def voigt_lookup(x, a: float, lnH, H0):
    """Table lookup of H(a, x): H(a,0) below |x| = 1e-4; the wing series
    a / (sqrt(pi) x^2) (1 + 3/(2 x^2)) above |x| = 1e3; otherwise linear
    interpolation of ln H in log10|x| between the bracketing nodes."""
    ax = np.abs(np.asarray(x, dtype=np.float64))
    out = np.empty_like(ax)
    lo = ax < 1e-4
    hi = ax > 1e3
    mid = ~(lo | hi)
    out[lo] = float(H0)
    xh = ax[hi]
    out[hi] = a / (SQRT_PI * xh * xh) * (1.0 + 1.5 / (xh * xh))
    t = (np.log10(ax[mid]) - VOIGT_LOG10_MIN) * ((VOIGT_N - 1) / (VOIGT_LOG10_MAX - VOIGT_LOG10_MIN))
    i = np.clip(np.floor(t).astype(np.int64), 0, VOIGT_N - 2)
    f = t - i
    L = np.asarray(lnH, dtype=np.float64)
    out[mid] = np.exp((1.0 - f) * L[i] + f * L[i + 1])
    return out


# ---------------------------------------------------------------- ph_mode 1 and 3 profiles
#
# Sec. 2.3.1 describes three photon modes. ph_mode 2 is the slice above.
# ph_mode 1 keeps a two-dimensional Voigt table (64 logarithmically spaced
# damping parameters by 512 frequency points) in global memory; its grid
# and interpolation are readings (the paper gives only the counts): a nodes
# uniform in log10 a over [-6, 0], x nodes uniform in log10|x| over [-4, 3],
# the table holds ln H, looked up bilinearly in (log10 a, log10|x|).
# ph_mode 3 replaces the tabulated profile by a blend of the Doppler core
# exp(-x^2) and the damping wing a / (sqrt(pi) (x^2 + a^2)) with the switch
# w = [1 + tanh(2|x| - 2 u0)] / 2 at the crossing point u0 of the two.

V2_NA = 64
V2_NX = 512
V2_LA_MIN = -6.0
V2_LA_MAX = 0.0


def voigt2d_anodes():
    return 10.0 ** (V2_LA_MIN + (V2_LA_MAX - V2_LA_MIN) * np.arange(V2_NA) / (V2_NA - 1))


def voigt2d_xnodes():
    return 10.0 ** (VOIGT_LOG10_MIN + (VOIGT_LOG10_MAX - VOIGT_LOG10_MIN) * np.arange(V2_NX) / (V2_NX - 1))


def voigt2d_table():
    """ln H(a_j, x_i) at the ph_mode 1 nodes, [64, 512], stored as float32."""
    A = voigt2d_anodes()
    X = voigt2d_xnodes()
    tab = np.empty((V2_NA, V2_NX))
    for j, a in enumerate(A):
        tab[j] = np.log(voigt_H(a, X))
    return tab.astype(np.float32)


def voigt2d_weights(a: float):
    """Row j and weight w of damping parameter a on the table's a axis:
    log10 a = (1 - w) log10 a_j + w log10 a_{j+1}. a must lie in [1e-6, 1]."""
    if not (10.0 ** V2_LA_MIN <= a <= 10.0 ** V2_LA_MAX):
        raise ValueError(f"a = {a} outside the ph_mode 1 table [1e-6, 1]")
    s = (math.log10(a) - V2_LA_MIN) * ((V2_NA - 1) / (V2_LA_MAX - V2_LA_MIN))
    j = min(max(int(math.floor(s)), 0), V2_NA - 2)
    return j, s - j


def voigt2d_lookup(x, a: float, tab):
    """ph_mode 1 lookup of H(a, x): bilinear in (log10 a, log10|x|) of ln H;
    |x| below the first node uses the first node; the wing series
    a / (sqrt(pi) x^2) (1 + 3/(2 x^2)) above |x| = 1e3."""
    j, w = voigt2d_weights(a)
    ax = np.abs(np.asarray(x, dtype=np.float64))
    out = np.empty_like(ax)
    hi = ax > 1e3
    xh = ax[hi]
    out[hi] = a / (SQRT_PI * xh * xh) * (1.0 + 1.5 / (xh * xh))
    m = ~hi
    t = (np.log10(np.maximum(ax[m], 10.0 ** VOIGT_LOG10_MIN)) - VOIGT_LOG10_MIN) * \
        ((V2_NX - 1) / (VOIGT_LOG10_MAX - VOIGT_LOG10_MIN))
    t = np.maximum(t, 0.0)
    i = np.clip(np.floor(t).astype(np.int64), 0, V2_NX - 2)
    f = t - i
    T0 = np.asarray(tab[j], dtype=np.float64)
    T1 = np.asarray(tab[j + 1], dtype=np.float64)
    lo_row = (1.0 - f) * T0[i] + f * T0[i + 1]
    hi_row = (1.0 - f) * T1[i] + f * T1[i + 1]
    out[m] = np.exp((1.0 - w) * lo_row + w * hi_row)
    return out


def blend_u0(a: float) -> float:
    """Crossing point u0 > 0 of the core exp(-u^2) and the wing
    a / (sqrt(pi) (u^2 + a^2)) that separates core from wing: the larger
    root of g(u) = -u^2 - ln(a / (sqrt(pi) (u^2 + a^2))). g is largest at
    u* = sqrt(1 - a^2) and falls without bound beyond it, so the root is
    bracketed by [u*, 30] when g(u*) > 0 (a below about 0.8)."""
    from scipy.optimize import brentq

    def g(u):
        return -u * u - math.log(a / (SQRT_PI * (u * u + a * a)))

    if not (0.0 < a < 1.0):
        raise ValueError("ph_mode 3 needs 0 < a < 1")
    us = math.sqrt(1.0 - a * a)
    if g(us) <= 0.0:
        raise ValueError(f"core and wing do not cross for a = {a}")
    return brentq(g, us, 30.0, xtol=1e-15, rtol=1e-15, maxiter=200)


def blend_H(x, a: float, u0: float):
    """ph_mode 3 profile: (1 - w) exp(-x^2) + w a / (sqrt(pi) (x^2 + a^2)),
    w = [1 + tanh(2|x| - 2 u0)] / 2."""
    ax = np.abs(np.asarray(x, dtype=np.float64))
    w = 0.5 * (1.0 + np.tanh(2.0 * ax - 2.0 * u0))
    return (1.0 - w) * np.exp(-ax * ax) + w * a / (SQRT_PI * (ax * ax + a * a))


# ---------------------------------------------------------------- USampler

US_NX = 40
US_NU = 251
US_UMIN = -6.0
US_DU = 0.048
US_LNFLOOR = math.log(1e-30)


def usampler_xnodes():
    """Incoming-frequency nodes (reading of Sec. 2.1.1): 18 uniform nodes
    |x| = 8 i / 18, i = 0..17, then 22 log-spaced nodes from 8 to 300."""
    uni = 8.0 * np.arange(18) / 18.0
    logp = 8.0 * (300.0 / 8.0) ** (np.arange(22) / 21.0)
    return np.concatenate([uni, logp])


def usampler_unodes():
    """Atom-velocity nodes u_j = -6 + 0.048 j, j = 0..250."""
    return US_UMIN + US_DU * np.arange(US_NU)


def usampler_masses(x: float, a: float):
    """Probability mass of p(u | x) ~ exp(-u^2) / (a^2 + (x-u)^2) in each
    u-cell [u_j, u_j+1] (Sec. 2.1.1). Reading: the Lorentz factor is a spike
    of width a that a 0.048 grid cannot sample, so each cell's mass is the
    exact integral of the Lorentz factor times the second-order Taylor
    expansion of exp(-u^2) about the cell midpoint m:
      exp(-m^2) [I0 - 2 m I1 + (2 m^2 - 1) I2],  Ik = int (u - m)^k L(u) du.
    Returns (midpoints[250], unnormalised masses[250])."""
    u = usampler_unodes()
    lo, hi = u[:-1], u[1:]
    m = 0.5 * (lo + hi)
    h = hi - lo
    dl, dh = lo - x, hi - x
    # atan(dh/a) - atan(dl/a); for a cell on one side of x the difference of
    # two near-equal angles is taken as atan(h a / (a^2 + dl dh)), which does
    # not cancel when a is tiny
    same_side = dl * dh > 0
    I0 = np.where(same_side, np.arctan(np.where(same_side, h * a / (a * a + dl * dh), 0.0)),
                  np.arctan(dh / a) - np.arctan(dl / a)) / a
    Jx = 0.5 * np.log((a * a + (hi - x) ** 2) / (a * a + (lo - x) ** 2))   # int (u - x) L du
    I1 = Jx + (x - m) * I0
    I2 = h - a * a * I0 + 2.0 * (x - m) * Jx + (x - m) ** 2 * I0
    return m, np.exp(-m * m) * (I0 - 2.0 * m * I1 + (2.0 * m * m - 1.0) * I2)


def usampler_table(a: float):
    """ln of the normalised cumulative distribution at the 251 u-nodes for
    each of the 40 x-nodes, floored at ln(1e-30), stored as float32.
    Returns (xnodes[40] float32, lncdf[40, 251] float32)."""
    xs = usampler_xnodes()
    out = np.empty((US_NX, US_NU))
    for i, x in enumerate(xs):
        _, m = usampler_masses(x, a)
        cs = np.cumsum(m)
        c = np.concatenate([[0.0], cs]) / cs[-1]
        out[i] = np.log(np.maximum(c, 1e-30))
    return xs.astype(np.float32), out.astype(np.float32)


def _largest_le(nodes, v):
    """Largest index i with nodes[i] <= v (nodes ascending)."""
    return int(np.searchsorted(nodes, v, side="right")) - 1


def usampler_sample(x: float, xi: float, xnodes, lncdf) -> float:
    """Draw u_par for incoming gas-frame frequency x from one uniform xi by
    inverting each bracketing row (binary search + linear interpolation of
    u against ln CDF), then interpolating the two u values linearly in |x|;
    x < 0 by the symmetry u -> -u. Valid for |x| <= 300."""
    X = np.asarray(xnodes, dtype=np.float64)
    ax = abs(x)
    i = min(max(_largest_le(X, ax), 0), US_NX - 2)
    t = (ax - X[i]) / (X[i + 1] - X[i])
    L = math.log(xi)
    us = []
    for row in (i, i + 1):
        c = np.asarray(lncdf[row], dtype=np.float64)
        j = min(max(_largest_le(c, L), 0), US_NU - 2)
        us.append(US_UMIN + US_DU * j + US_DU * (L - c[j]) / (c[j + 1] - c[j]))
    u = (1.0 - t) * us[0] + t * us[1]
    return -u if x < 0 else u


# ---------------------------------------------------------------- R_IIA table

R_ND = 201          # Delta nodes, -10 .. 10 step 0.1
R_NX = 200          # |x_in| nodes, uniform on [0, 120]
R_NG = 40           # g nodes, uniform on [-1, 1]
R_DMAX = 10.0
R_DSTEP = 0.1
R_XMAX = 120.0
R_SMIN = 0.1        # smallest Gaussian width (the g = +-1 nodes, reading)


def rtable_axes():
    d = -R_DMAX + R_DSTEP * np.arange(R_ND)
    x = R_XMAX * np.arange(R_NX) / (R_NX - 1)
    g = -1.0 + 2.0 * np.arange(R_NG) / (R_NG - 1)
    return d, x, g


def gauss(y, s):
    """Normalised Gaussian of standard deviation s."""
    return np.exp(-0.5 * (y / s) ** 2) / (math.sqrt(2.0 * math.pi) * s)


def rtable(a: float):
    """Discrete R_IIA kernel (Eq. riia-table):
    R(D; |x|, g) = sum_k p_k G[D - u_k (g - 1); 2^{-1/2} sin(gamma)],
    with p_k the normalised sampler masses at |x| and u_k the cell
    midpoints; width floored at 0.1 where sin(gamma) -> 0 (g = +-1).
    Returns float32 array [g=40][x=200][D=201]."""
    d, xs, gs = rtable_axes()
    out = np.empty((R_NG, R_NX, R_ND))
    for jx, x in enumerate(xs):
        um, m = usampler_masses(x, a)
        p = m / m.sum()
        for kg, g in enumerate(gs):
            s = max(math.sqrt(max(0.0, 1.0 - g * g)) / math.sqrt(2.0), R_SMIN)
            out[kg, jx] = (p[None, :] * gauss(d[:, None] - um[None, :] * (g - 1.0), s)).sum(axis=1)
    return out.astype(np.float32)


def r_inf(D, g):
    """Asymptotic kernel for |x_in| >= 120 (Eq. riia-inf); the denominator
    (g-1)^2 + sin^2(gamma) = 2 (1 - g) is floored like the table widths."""
    v = max(1.0 - g, R_SMIN * R_SMIN)
    D = np.asarray(D, dtype=np.float64)
    return np.exp(-D * D / (2.0 * v)) / math.sqrt(2.0 * math.pi * v)


def r_lookup(D: float, x: float, g: float, rtab) -> float:
    """Trilinear lookup of R(D; x, g); zero for |D| > 10; the symmetry
    R(D; -x, g) = R(-D; x, g); Eq. riia-inf for |x| >= 120."""
    if x < 0.0:
        D, x = -D, -x
    if abs(D) > R_DMAX:
        return 0.0
    if x >= R_XMAX:
        return float(r_inf(D, g))
    fd = (D + R_DMAX) / R_DSTEP
    fx = x * (R_NX - 1) / R_XMAX
    fg = (g + 1.0) * (R_NG - 1) / 2.0
    i = min(max(int(math.floor(fd)), 0), R_ND - 2)
    j = min(max(int(math.floor(fx)), 0), R_NX - 2)
    k = min(max(int(math.floor(fg)), 0), R_NG - 2)
    wd, wx, wg = fd - i, fx - j, fg - k
    T = rtab
    acc = 0.0
    for dk, ck in ((0, 1.0 - wg), (1, wg)):
        for dj, cj in ((0, 1.0 - wx), (1, wx)):
            row = T[k + dk, j + dj]
            acc += ck * cj * ((1.0 - wd) * float(row[i]) + wd * float(row[i + 1]))
    return acc
