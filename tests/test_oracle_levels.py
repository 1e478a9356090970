"""Pins of the oracle's statistical-equilibrium solve and of the Lambda
iteration's excitation rate (Sec. 2.1.3)."""
import math

import numpy as np

from oracle import levels as LV


def test_collisions_alone_give_boltzmann():
    """Detailed balance: with A = 0 and Gamma = 0 the solve returns the
    Boltzmann populations at T exactly."""
    lev = LV.rotor()
    lev.A[:] = 0.0
    n_mol = np.array([1.0, 3.5e-2, 7.0])
    pops = LV.solve(lev, 20.0, np.array([1e3, 1e2, 1e5]), n_mol, {})
    ref = LV.boltzmann(lev, 20.0, n_mol)
    assert np.allclose(pops, ref, rtol=1e-12)


def test_two_level_closed_form():
    """Eq. boltzmann for two levels, with radiation and collisions."""
    lev = LV.rotor(n_lev=2, A1=3e-6, k_ul=2e-11)
    for G, nc in ((0.0, 1e3), (1e-6, 1e2), (5e-5, 1e6)):
        p = LV.solve_cell(lev, 15.0, nc, 2.0, {(1, 0): G})
        ratio = LV.two_level_ratio(G, 2e-11, nc, 3e-6, 3.0, 1.0, lev.E_K[1], 15.0)
        assert abs(p[1] / p[0] / ratio - 1) < 1e-12
        assert abs(p.sum() - 2.0) < 1e-12


def test_strong_radiation_saturates_and_weak_density_subthermal():
    lev = LV.rotor()
    # huge Gamma on every line: populations approach the statistical weights
    G = {tr: 1e3 for tr in lev.transitions()}
    p = LV.solve_cell(lev, 20.0, 1.0, 1.0, G)
    w = lev.g / lev.g.sum()
    assert np.allclose(p, w, rtol=2e-3)
    # no collisions, no radiation field: everything decays to the ground state
    p = LV.solve_cell(lev, 20.0, 0.0, 1.0, {})
    assert abs(p[0] - 1.0) < 1e-12 and np.all(p[1:] < 1e-12)


def test_rotor_line_frequencies():
    lev = LV.rotor()
    # B/k = 2.77 K puts J = 1-0 at 2 B = 115.4 GHz
    assert abs(lev.nu(1, 0) / 115.4e9 - 1) < 1e-3
    assert lev.transitions() == [(1, 0), (2, 1), (3, 2), (4, 3)]


def test_gamma_thin_limit_at_the_centre_of_an_emitting_cube():
    """The Lambda iteration's excitation rate (the path-length estimator
    (L / N) sigma0 sum(w ds H) / V_cell). An optically thin uniform cube
    (depth 2e-7) emitting n_u A per unit volume with the thermal profile:
    at its centre Gamma = n_u A sigma0 <H> <d>, where <H> = int e^{-x^2} /
    sqrt(pi) H(a, x) dx (Faddeeva quadrature; 1/sqrt(2) as a -> 0) and <d> =
    h E[1/max|n_i|] is the mean distance from the centre to the surface of
    a cube of half-side h (quadrature over directions). The 8 central cells,
    2e6 packets: counting error ~0.5 %."""
    import workloads as W
    import oracle
    from numpy.polynomial.legendre import leggauss
    from scipy.integrate import quad
    from scipy.special import wofz
    from oracle import tables as T
    n = 16
    shape = (n, n, n)
    nm = np.full(shape, 1e-9, np.float32)
    spec = W.LevelSpec()
    p = W.Problem(name="thin_cube", shape=shape, cell_cm=1e15, periodic=(False, False, False),
                  opacity_kind="n_l", opacity=nm.copy(), T_K=20.0,
                  line=W.Line(115.27e9, spec.mass_amu, spec.A1, 3.0, 1.0, spec.k_ul, 0.0),
                  source=W.Source(W.SOURCE_VOLUME, profile=W.PROFILE_GAUSSIAN, rate=nm.copy()),
                  n_coll=np.full(shape, 1.0, np.float32), tallies=("exc",), n_packets=1)
    lev = LV.rotor(2, spec.B_K, spec.A1, spec.k_ul, spec.mass_amu)
    pops0 = LV.boltzmann(lev, p.T_K, nm.reshape(-1).astype(np.float64))
    G = LV.gamma_rates(oracle, p, lev, pops0, pops0, 2_000_000, 4)[(1, 0)].reshape(shape)
    b = T.doppler_b(p.T_K, lev.mass_amu)
    a = T.damping_a(lev.A[1, 0], lev.nu(1, 0), b)
    s0 = T.sigma0(lev.g[1], lev.g[0], lev.A[1, 0], lev.nu(1, 0), b)
    assert nm[0, 0, 0] * s0 * n * p.cell_cm < 1e-6                      # thin
    H_em = quad(lambda x: 2.0 * np.exp(-x * x) / np.sqrt(np.pi) * wofz(x + 1j * a).real, 0.0, 12.0, limit=200)[0]
    mx, mw = leggauss(1000)
    mu, wmu = 0.5 * (mx + 1.0), 0.5 * mw
    ph, wph = (np.pi / 8) * (mx + 1.0), (np.pi / 8) * mw
    M, P = np.meshgrid(mu, ph, indexing="ij")
    st = np.sqrt(1.0 - M * M)
    inv_max = 1.0 / np.maximum(np.maximum(st * np.cos(P), st * np.sin(P)), M)
    d_mean = (n / 2) * p.cell_cm * float((wmu[:, None] * wph[None, :] * inv_max).sum() / (np.pi / 4))
    want = pops0[0, 1] * lev.A[1, 0] * s0 * H_em * d_mean
    got = G[n // 2 - 1:n // 2 + 1, n // 2 - 1:n // 2 + 1, n // 2 - 1:n // 2 + 1].mean()
    assert abs(got / want - 1.0) < 0.03, got / want

