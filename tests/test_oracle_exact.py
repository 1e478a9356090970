"""The tabulated method against O-exact (oracle/exact.py: the slab walk with
the Voigt function evaluated directly and the atom's parallel velocity drawn
exactly by rejection): the exact sampler follows the quadrature CDF of
p(u | x) (Sec. 2.1.1), and the tabulated oracle's escaped spectrum is the
exact walk's within the Monte Carlo noise, i.e. the table error of the
method is below the noise at this packet count."""
import math

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.special import wofz

import oracle
import workloads as W
from oracle import exact as E


@pytest.mark.parametrize("a", [4.7e-4, 0.01, 0.149])
@pytest.mark.parametrize("x", [0.0, 0.6, 2.8, 6.0, -20.0])
def test_exact_sampler_follows_the_quadrature_cdf(a, x):
    n = 20000
    u = np.sort(E.sample_upar(np.full(n, x), a, np.random.default_rng(11)))
    Z = math.pi * wofz(x + 1j * a).real / a             # int exp(-u^2) / ((u - x)^2 + a^2) du
    f = lambda v: math.exp(-v * v) / ((v - x) ** 2 + a * a)
    idx = np.arange(100, n, 200)
    dev = 0.0
    for i in idx:
        t = u[i]
        F = quad(f, -np.inf, min(t, x), limit=400)[0]
        if t > x:
            F += quad(f, x, t, limit=400)[0]
        dev = max(dev, abs(F / Z - (i + 0.5) / n))
    assert dev < 1.95 / math.sqrt(n), dev             # the 0.1 % Kolmogorov-Smirnov bound


@pytest.mark.parametrize("tau0,a,nz,n,bins", [
    (500.0, 0.01, 64, 4000, (-20.0, 20.0, 80)),
    (2000.0 / math.sqrt(math.pi), 0.149, 128, 3000, (-30.0, 30.0, 120)),   # Sec. 3.1's slab at tau_m = 2000
])
def test_tabulated_walk_matches_the_exact_walk(tau0, a, nz, n, bins):
    """Static slab, line-centre photons at the midplane: a core-dominated
    case (a = 0.01) and the paper's damped slab (a = 0.149, whose photons
    escape through the core-wing transition). Two-sample chi^2 of the
    spectra p > 1e-3 and mean |x| within 4 sigma."""
    from _gpu_common import chi2_two_sample
    ex = E.slab_spectrum(tau0, a, n, 2, bins)
    tab = oracle.run(W.slab(tau0=tau0, a=a, nz=nz, n_packets=n, bins=bins))["spec_c"]
    assert ex.sum() == tab.sum() == n
    assert chi2_two_sample(ex[1:-1], tab[1:-1])[2] > 1e-3
    lo, hi, nb = bins
    x = lo + (np.arange(nb) + 0.5) * (hi - lo) / nb
    stats = []
    for c in (ex[1:-1].astype(np.float64), tab[1:-1].astype(np.float64)):
        m = (np.abs(x) * c).sum() / c.sum()
        sd = math.sqrt(((np.abs(x) - m) ** 2 * c).sum() / c.sum())
        stats.append((m, sd))
    sig = math.sqrt(stats[0][1] ** 2 + stats[1][1] ** 2) / math.sqrt(n)
    assert abs(stats[0][0] - stats[1][0]) < 4.0 * sig, (stats, sig)
