"""Pins of the oracle's continuum absorption (Sec. 2.2.1 and Eq. scat-line:
the packet weight decays as exp(-dtau_e) along a segment, whose tallies
take the mean weight (1 - exp(-dtau_e))/dtau_e; Sec. 3.2's dusty slab)
against closed forms of pure absorption, the weight budget and the
invariance of the walk itself."""
import math

import numpy as np
import pytest
from scipy.special import expn

import oracle
import workloads as W


@pytest.mark.parametrize("tau_a", [0.1, 1.0, 3.0])
def test_pure_absorption_escape_fraction_is_E2(tau_a):
    """No line opacity: a packet from the midplane with direction cosine mu
    escapes with weight exp(-tau_a/|mu|), so f_esc = E_2(tau_a), with
    per-packet variance E_2(2 tau_a) - E_2(tau_a)^2."""
    n = 20000
    r = oracle.run(W.dusty_slab(tau_a, tau0=0.0, n_packets=n))
    f = r["spec_w"].sum() / n
    sig = math.sqrt((expn(2, 2 * tau_a) - expn(2, tau_a) ** 2) / n)
    assert abs(f - expn(2, tau_a)) < 4.5 * sig, (f, expn(2, tau_a), sig)
    assert r["stats"][4] == 0                       # no scatterings


def test_segment_factor_against_layer_closed_form():
    """Mean weight along segments: in the pure-absorption slab (kappa per
    cell width) the expected sum of w ds over the layer between heights z1
    and z2 above the midplane is, per packet, (E_2(kappa z1) - E_2(kappa
    z2)) / (2 kappa) on each side. The excitation tally multiplies it by
    the profile value at the packet's (line-centre) frequency, H(a, 0)."""
    n, nz, tau_a = 40000, 16, 2.0
    p = W.dusty_slab(tau_a, tau0=0.0, nz=nz, n_packets=n, tallies=("exc",))
    r = oracle.run(p)
    H0 = oracle.line_tables(0.015, False)["voigt_H0"]
    kappa = tau_a / (nz / 2)
    exc = r["exc"].reshape(nz) / (n * H0)
    for layer in range(nz // 2):
        z1, z2 = layer, layer + 1
        want = (expn(2, kappa * z1) - expn(2, kappa * z2)) / (2 * kappa)
        up, down = exc[nz // 2 + layer], exc[nz // 2 - 1 - layer]
        assert up == pytest.approx(want, rel=0.03), (layer, up, want)
        assert down == pytest.approx(want, rel=0.03), (layer, down, want)


def test_weight_budget_is_exact():
    """Every unit of emitted weight escapes, is absorbed, or falls below the
    cut: sum(spec_w) + sum(absw) = N up to the cut weights and rounding."""
    n = 2000
    r = oracle.run(W.dusty_slab(0.05, tau0=1e4, n_packets=n, bins=(-30.0, 30.0, 60)))
    tot = r["spec_w"].sum() + r["absw"].sum()
    cut = int(r["stats"][6]) * oracle.WEIGHT_CUT
    assert abs(tot - n) <= cut + 1e-9 * n
    assert r["stats"][0] == r["stats"][1] + r["stats"][2] + r["stats"][3] + r["stats"][6]


def test_absorption_only_reweights_the_walk():
    """The continuum changes weights, never decisions: packet by packet the
    walk (scatterings, crossings, final frequency, status) is the walk
    without absorption, until a weight falls below the cut."""
    n = 1500
    base = W.slab(tau0=1e4, a=0.015, T_K=10.0, n_packets=n, bins=(-30.0, 30.0, 60))
    dusty = W.dusty_slab(0.2, tau0=1e4, n_packets=n, bins=(-30.0, 30.0, 60))
    r0 = oracle.run(base, records=True)
    r1 = oracle.run(dusty, records=True)
    a, b = r0["records"], r1["records"]
    live = b["status"] != oracle.ABSORBED
    assert live.mean() > 0.5
    for f in ("nscat", "ncross", "status", "cell0", "x"):
        assert np.array_equal(a[f][live], b[f][live]), f
    assert np.all(b["nscat"][~live] <= a["nscat"][~live])
    # escaped weights: each escaping packet lost weight, none gained
    assert r1["spec_w"].sum() < r0["spec_w"].sum() == n


def test_escape_fraction_falls_with_absorption_depth():
    n = 1500
    f = []
    for tau_a in (1e-3, 1e-2, 1e-1):
        r = oracle.run(W.dusty_slab(tau_a, tau0=1e4, n_packets=n, bins=(-30.0, 30.0, 60)))
        f.append(r["spec_w"].sum() / n)
    assert 1.0 > f[0] > f[1] > f[2] > 0.0
