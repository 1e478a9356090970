"""Pins of the oracle's statistical-equilibrium solve (Sec. 2.1.3)."""
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
