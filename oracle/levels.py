"""FP64 oracle of statistical equilibrium and the Lambda iteration
(Sec. 2.1.3, Eq. boltzmann, Eq. eps).

TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg may import this module.

Rates for each level pair u > l (energies E in K, degeneracies g):
  collisions  C_ul = k_ul n_coll,  C_lu = (g_u/g_l) C_ul exp(-(E_u - E_l)/T)
              (detailed balance);
  radiation   l -> u: Gamma_lu (the absorption rate per lower-level molecule,
              from the Monte Carlo excitation tally),
              u -> l: A_ul + (g_l/g_u) Gamma_lu (spontaneous plus stimulated,
              B_ul = (g_l/g_u) B_lu).
Steady state: for every level i, sum_j n_j R_ji = n_i sum_j R_ij, with the
last equation replaced by sum_i n_i = n_mol; solved with numpy.linalg.solve.

Lambda iteration (Sec. 2.1.3): start from collisional equilibrium (the
Boltzmann populations at T, which the collision-only rates give by detailed
balance); the emission of every line is frozen at those populations
(volume source proportional to n_u A_ul); each cycle sets each line's
opacity from the current lower-level population, runs the Monte Carlo pass,
turns the excitation tally into Gamma, and re-solves the populations.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import tables as T

H_PLANCK = 6.62607015e-27


@dataclasses.dataclass
class Levels:
    E_K: np.ndarray          # [n] level energies / k_B
    g: np.ndarray            # [n] degeneracies
    A: np.ndarray            # [n, n] A[u, l] for u > l, else 0
    k_coll: np.ndarray       # [n, n] k[u, l] for u > l (cm^3 s^-1)
    mass_amu: float

    @property
    def n(self):
        return len(self.E_K)

    def transitions(self):
        """Radiative pairs (u, l) with A > 0, in order of (l, u)."""
        return [(u, l) for l in range(self.n) for u in range(l + 1, self.n) if self.A[u, l] > 0]

    def nu(self, u, l):
        return (self.E_K[u] - self.E_K[l]) * T.K_B / H_PLANCK


def boltzmann(lev: Levels, T_K: float, n_mol):
    """LTE populations [ncell, n]."""
    w = lev.g * np.exp(-(lev.E_K - lev.E_K[0]) / T_K)
    f = w / w.sum()
    return np.asarray(n_mol, dtype=np.float64)[:, None] * f[None, :]


def rate_matrix(lev: Levels, T_K: float, n_coll: float, gamma: dict):
    """R[i, j] = rate coefficient from level i to level j (per molecule in i)."""
    n = lev.n
    R = np.zeros((n, n))
    for u in range(n):
        for l in range(u):
            Cul = lev.k_coll[u, l] * n_coll
            Clu = lev.g[u] / lev.g[l] * Cul * math.exp(-(lev.E_K[u] - lev.E_K[l]) / T_K)
            G = gamma.get((u, l), 0.0)
            R[u, l] += lev.A[u, l] + lev.g[l] / lev.g[u] * G + Cul
            R[l, u] += G + Clu
    return R


def solve_cell(lev: Levels, T_K: float, n_coll: float, n_mol: float, gamma: dict):
    R = rate_matrix(lev, T_K, n_coll, gamma)
    n = lev.n
    M = R.T - np.diag(R.sum(axis=1))        # dn_i/dt = sum_j n_j R[j, i] - n_i sum_j R[i, j]
    M[-1, :] = 1.0
    rhs = np.zeros(n)
    rhs[-1] = n_mol
    return np.linalg.solve(M, rhs)


def solve(lev: Levels, T_K: float, n_coll, n_mol, gamma_cells: dict):
    """Populations [ncell, n] given Gamma[(u, l)] -> array [ncell]."""
    n_coll = np.asarray(n_coll, dtype=np.float64)
    n_mol = np.asarray(n_mol, dtype=np.float64)
    out = np.empty((n_mol.size, lev.n))
    for c in range(n_mol.size):
        out[c] = solve_cell(lev, T_K, float(n_coll[c]), float(n_mol[c]),
                            {k: float(v[c]) for k, v in gamma_cells.items()})
    return out


def two_level_ratio(Gamma, k_ul, n_coll, A, g_u, g_l, dE_K, T_K):
    """Eq. boltzmann: n_u / n_l for a two-level system."""
    k_lu = g_u / g_l * k_ul * math.exp(-dE_K / T_K)
    return (Gamma + k_lu * n_coll) / (A + g_l / g_u * Gamma + k_ul * n_coll)


def rotor(n_lev: int = 5, B_K: float = 2.77, A1: float = 1e-7, k_ul: float = 1e-11, mass_amu: float = 28.0):
    """Linear rotor: E_J = B J (J + 1), g_J = 2J + 1, A_{J -> J-1} = A1 J^3,
    k_ul = k_ul for every pair u > l."""
    J = np.arange(n_lev)
    A = np.zeros((n_lev, n_lev))
    k = np.zeros((n_lev, n_lev))
    for u in range(1, n_lev):
        A[u, u - 1] = A1 * u ** 3
        for l in range(u):
            k[u, l] = k_ul
    return Levels(E_K=B_K * J * (J + 1.0), g=2.0 * J + 1.0, A=A, k_coll=k, mass_amu=mass_amu)


def gamma_rates(oracle_mod, problem, lev: Levels, pops, pops0, packets_per_line: int, seed: int, cycle: int = 0,
                nthreads=None):
    """Gamma_lu per cell for every radiative pair (u, l): one pass of the
    oracle's FP64 walk per line, with the line's opacity from the lower-level
    populations `pops` and its emission frozen at `pops0` (a volume source of
    n_u A_ul per cell, thermal profile), packet ids starting at
    (cycle * n_lines + line) * N. The path-length estimator: Gamma =
    (L / N) sigma0 sum(w ds H) / V_cell, with L = sum n_u A_ul V_cell the
    line's photon rate and ds in cm (the excitation tally holds ds in cell
    widths, hence one factor dx against V_cell = dx^3)."""
    import dataclasses as dc
    trans = lev.transitions()
    dx = problem.cell_cm
    gam = {}
    for t, (u, l) in enumerate(trans):
        rate = (pops0[:, u] * lev.A[u, l]).astype(np.float32)
        line = dc.replace(problem.line, nu0_hz=lev.nu(u, l), mass_amu=lev.mass_amu, A_ul=lev.A[u, l],
                          g_u=lev.g[u], g_l=lev.g[l], k_ul=lev.k_coll[u, l], a_fixed=0.0)
        q = dc.replace(problem, opacity_kind="n_l",
                       opacity=pops[:, l].astype(np.float32).reshape(problem.shape), line=line,
                       source=dc.replace(problem.source, kind="volume", profile="gaussian",
                                         rate=rate.reshape(problem.shape)),
                       tallies=("exc",), spectrum=(-40.0, 40.0, 80), channels=None, cameras=())
        r = oracle_mod.run(q, n=packets_per_line, first=(cycle * len(trans) + t) * packets_per_line, seed=seed,
                           nthreads=nthreads)
        b = T.doppler_b(problem.T_K, lev.mass_amu)
        s0 = T.sigma0(lev.g[u], lev.g[l], lev.A[u, l], lev.nu(u, l), b)
        lum = float(np.sum(pops0[:, u] * lev.A[u, l])) * dx ** 3
        gam[(u, l)] = lum / packets_per_line * s0 * r["exc"] / dx ** 2
    return gam


def lambda_iterate(oracle_mod, problem, n_mol, lev: Levels, n_iter: int, packets_per_line: int, seed: int,
                   pops=None, nthreads=None):
    """The Lambda iteration with the oracle's FP64 walk, following the same
    packet ids per cycle and line ((cycle * n_lines + line) * N), so that a
    device run with the same inputs follows the same random streams.
    Returns (populations [ncell, n], per-cycle max change / n_mol)."""
    n_mol = np.asarray(n_mol, dtype=np.float32).astype(np.float64).reshape(-1)
    n_coll = np.asarray(problem.n_coll, dtype=np.float32).astype(np.float64).reshape(-1)
    pops = boltzmann(lev, problem.T_K, n_mol) if pops is None else np.array(pops, dtype=np.float64)
    pops0 = pops.copy()
    changes = []
    for it in range(n_iter):
        gam = gamma_rates(oracle_mod, problem, lev, pops, pops0, packets_per_line, seed, it, nthreads)
        new = solve(lev, problem.T_K, n_coll, n_mol, gam)
        with np.errstate(invalid="ignore", divide="ignore"):
            ch = np.where(n_mol[:, None] > 0, np.abs(new - pops) / n_mol[:, None], 0.0)
        changes.append(float(ch.max()))
        pops = new
    return pops, changes
