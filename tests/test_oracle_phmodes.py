"""Pins of the oracle's ph_mode 1 (two-dimensional Voigt table) and ph_mode 3
(core-wing blend) profiles (Sec. 2.3.1), against the exact Voigt function
(scipy's Faddeeva routine), the crossing-point definition, the limits the
blend is built from, and the C walk's own lookups."""
import math

import numpy as np
import pytest

import oracle
from oracle import tables as T

A_VALUES = [1e-4, 4.7e-4, 1e-2, 0.149]


@pytest.fixture(scope="module")
def tab():
    return T.voigt2d_table()


def test_table_grid_and_nodes(tab):
    A = T.voigt2d_anodes()
    X = T.voigt2d_xnodes()
    assert tab.shape == (64, 512) and tab.dtype == np.float32
    assert A[0] == pytest.approx(1e-6, rel=1e-12) and A[-1] == pytest.approx(1.0, rel=1e-12)
    assert X[0] == pytest.approx(1e-4, rel=1e-12) and X[-1] == pytest.approx(1e3, rel=1e-12)
    assert np.allclose(np.diff(np.log10(A)), 6.0 / 63) and np.allclose(np.diff(np.log10(X)), 7.0 / 511)
    # every stored node is ln H(a_j, x_i) rounded to float32
    for j in (0, 17, 40, 63):
        exact = np.log(T.voigt_H(A[j], X))
        assert np.abs(tab[j].astype(np.float64) - exact).max() <= 4e-7 * np.abs(exact).max() + 1e-7


def test_lookup_on_nodes_reproduces_the_table(tab):
    A = T.voigt2d_anodes()
    X = T.voigt2d_xnodes()
    for j in (3, 30, 62):
        a = float(A[j])
        got = T.voigt2d_lookup(X[5:500:37], a, tab)
        want = np.exp(tab[j, 5:500:37].astype(np.float64))
        assert np.allclose(got, want, rtol=1e-6)


@pytest.mark.parametrize("a", A_VALUES)
def test_lookup_error_against_exact_voigt(tab, a):
    """Bilinear interpolation of ln H on the coarse grid: the error against
    the exact H stays at the level set by the node spacing (0.0137 dex in x,
    0.095 dex in a): below 0.3% in the core, and up to 1-2% (the level at
    which the paper finds its two exact modes to agree) in the core-wing
    transition, where ln H bends sharply and the transition point moves
    between neighbouring a nodes."""
    x = np.concatenate([np.linspace(0.0, 10.0, 4001), np.geomspace(10.0, 2e3, 500)])
    rel = np.abs(T.voigt2d_lookup(x, a, tab) / T.voigt_H(a, x) - 1.0)
    assert rel.max() < 0.02, rel.max()
    core = np.abs(x) < 2.0
    assert rel[core].max() < 3e-3, rel[core].max()
    wing = np.abs(x) > 8.0
    assert rel[wing].max() < 1e-3, rel[wing].max()


@pytest.mark.parametrize("a", A_VALUES)
def test_lookup_normalisation(tab, a):
    """int H dx = sqrt(pi) (the Voigt normalisation) within the table error."""
    x = np.linspace(0.0, 1e3, 2_000_001)
    h = T.voigt2d_lookup(x, a, tab)
    integral = 2.0 * np.trapezoid(h, x) + 2.0 * a / (math.sqrt(math.pi) * 1e3)   # + wing beyond 1e3
    assert integral == pytest.approx(math.sqrt(math.pi), rel=3e-3)


def test_a_outside_the_table_is_rejected():
    for a in (5e-7, 1.5):
        with pytest.raises(ValueError):
            T.voigt2d_weights(a)


@pytest.mark.parametrize("a", [1e-6, 1e-4, 4.7e-4, 1e-2, 0.149, 0.5])
def test_blend_crossing_point(a):
    """u0 is where core and wing are equal, and it is the outer crossing:
    the core is larger just inside it and the wing larger outside."""
    u0 = T.blend_u0(a)
    core = lambda u: math.exp(-u * u)
    wing = lambda u: a / (math.sqrt(math.pi) * (u * u + a * a))
    assert core(u0) == pytest.approx(wing(u0), rel=1e-12)
    assert u0 > math.sqrt(1.0 - a * a)
    assert core(u0 * 0.98) > wing(u0 * 0.98)
    for u in (u0 * 1.02, u0 * 1.5, 10.0, 25.0):
        assert wing(u) > core(u)


@pytest.mark.parametrize("a", [1e-4, 1e-2, 0.149])
def test_blend_limits(a):
    """Core limit exp(-x^2) well inside u0, wing limit a / (sqrt(pi) x^2)
    far outside, the mean of the two at u0, and exact agreement with the
    true Voigt in the far wing, where both are the Lorentzian."""
    u0 = T.blend_u0(a)
    # (at x -> 0 the wing term 1/(sqrt(pi) a) is large enough for tiny a
    # that even the switch's residual weight there shows; start at 0.5)
    x_in = np.linspace(0.5, u0 - 2.0, 50)
    assert np.allclose(T.blend_H(x_in, a, u0), np.exp(-x_in ** 2), rtol=2e-3, atol=0)
    x_out = np.geomspace(u0 + 3.0, 1e3, 50)
    wing = a / (math.sqrt(math.pi) * (x_out ** 2 + a * a))
    assert np.allclose(T.blend_H(x_out, a, u0), wing, rtol=1e-4)
    assert T.blend_H(u0, a, u0) == pytest.approx(math.exp(-u0 * u0), rel=1e-12)
    far = np.geomspace(50.0, 1e3, 20)
    assert np.allclose(T.blend_H(far, a, u0), T.voigt_H(a, far), rtol=2e-3)
    assert np.allclose(T.blend_H(-far, a, u0), T.blend_H(far, a, u0))


def test_blend_is_rough_in_the_transition():
    """The approximation the paper offers only as a demonstration: tens of
    per cent off the true profile between core and wing."""
    a = 4.7e-4
    u0 = T.blend_u0(a)
    x = np.linspace(u0 - 1.0, u0 + 1.0, 201)
    rel = np.abs(T.blend_H(x, a, u0) / T.voigt_H(a, x) - 1.0)
    assert rel.max() > 0.1


@pytest.mark.parametrize("mode", [1, 3])
@pytest.mark.parametrize("a", [4.7e-4, 0.149])
def test_c_walk_lookups_match(tab, mode, a):
    L = oracle.c_lookups(a, ph_mode=mode)
    x = np.concatenate([[0.0, 5e-5, 1e-4], np.linspace(-12.0, 12.0, 301), [500.0, 999.0, 1001.0, 4e4]])
    got = np.array([L.voigt(float(v)) for v in x])
    want = T.voigt2d_lookup(x, a, tab) if mode == 1 else T.blend_H(x, a, T.blend_u0(a))
    assert np.allclose(got, want, rtol=1e-13, atol=0)


def _neufeld_mean_abs_x(a_tau_lc):
    """Mean |x| of the Neufeld slab profile P(x) ~ x^2 / cosh(sqrt(pi^3/54)
    x^3 / (a tau0)) (line-centre tau0): with y = c x^3 / (a tau0),
    E|x| = (a tau0 / c)^{1/3} (2/pi) int_0^inf y^{1/3} sech(y) dy."""
    from scipy.integrate import quad
    c = math.sqrt(math.pi ** 3 / 54.0)
    I = quad(lambda y: y ** (1.0 / 3.0) / math.cosh(y), 0.0, 60.0, limit=200)[0]
    return (a_tau_lc / c) ** (1.0 / 3.0) * 2.0 / math.pi * I


def test_walk_modes_on_a_damped_slab():
    """The paper's E1 slab (a = 0.149, mean depth tau_m = 2000, i.e. line-
    centre tau0 = tau_m / sqrt(pi)), 4000 packets: ph_mode 1 and 2 give the
    same spectrum within the Monte Carlo noise (and nearly the same walks,
    packet by packet, on the same random streams), both near the Neufeld
    mean |x|; ph_mode 3 shifts the spectrum (its core-wing transition is
    off by tens of per cent)."""
    import dataclasses
    import workloads as W
    from scipy.stats import chi2_contingency
    tau_lc = 2000.0 / math.sqrt(math.pi)
    p = W.slab(tau0=tau_lc, a=0.149, nz=128, n_packets=4000, bins=(-20.0, 20.0, 80))
    x = np.linspace(-20.0, 20.0, 81)[:-1] + 0.25
    out = {}
    for m in (2, 1, 3):
        q = dataclasses.replace(p, line=dataclasses.replace(p.line, ph_mode=m))
        r = oracle.run(q, records=True)
        c = r["spec_c"][1:-1].astype(np.float64)
        assert r["spec_c"][0] == 0 and r["spec_c"][-1] == 0
        out[m] = (c, (np.abs(x) * c).sum() / c.sum(), r["records"])
    mean_pred = _neufeld_mean_abs_x(0.149 * tau_lc)
    for m in (1, 2):
        assert out[m][1] == pytest.approx(mean_pred, rel=0.08), (m, out[m][1], mean_pred)
    same = (out[1][2]["nscat"] == out[2][2]["nscat"]).mean()
    assert same > 0.5, same
    keep = (out[1][0] + out[2][0]) >= 20
    _, pv, _, _ = chi2_contingency(np.stack([out[1][0][keep], out[2][0][keep]]))
    assert pv > 0.01, pv
    assert abs(out[3][1] / out[2][1] - 1.0) > 0.05, (out[3][1], out[2][1])
