"""Statistical equilibrium on the GPU (FP64 per-cell solves) against numpy on
the same rates (populations within 1e-4 relative, the stated bar), and the
Lambda iteration against the oracle's on a small non-LTE cloud."""
import numpy as np
import pytest

import oracle
import workloads as W
from oracle import levels as LV
from _gpu_common import need_gpu, report

pytestmark = pytest.mark.gpu


def _desc(krl, lev, n_mol_t):
    return krl.levels_desc(lev.E_K, lev.g, lev.A, lev.k_coll, lev.mass_amu, n_mol_t)


def test_solve_matches_numpy_on_given_rates():
    krl = need_gpu()
    import torch
    p, n_mol, spec = W.cloud(n=8, seed=5)
    lev = LV.rotor(spec.n_lev, spec.B_K, spec.A1, spec.k_ul, spec.mass_amu)
    ncell = p.ncell
    rng = np.random.default_rng(9)
    trans = lev.transitions()
    gam = rng.lognormal(mean=-16.0, sigma=2.0, size=(len(trans), ncell))
    g = krl.Grid(p)
    try:
        nm_t = torch.from_numpy(n_mol.reshape(-1)).cuda()
        pops = torch.zeros((ncell, lev.n), dtype=torch.float64, device="cuda")
        gam_t = torch.from_numpy(gam).cuda()
        g.levels_solve(_desc(krl, lev, nm_t), gam_t, pops)
        got = pops.cpu().numpy()
    finally:
        g.close()
    ref = LV.solve(lev, p.T_K, p.n_coll.reshape(-1), n_mol.reshape(-1), {tr: gam[i] for i, tr in enumerate(trans)})
    rel = np.abs(got - ref) / np.maximum(ref, 1e-30 * n_mol.reshape(-1)[:, None])
    assert rel.max() < 1e-4, rel.max()
    assert np.allclose(got.sum(axis=1), n_mol.reshape(-1), rtol=1e-12)


def test_collisional_equilibrium_is_boltzmann():
    krl = need_gpu()
    import torch
    p, n_mol, spec = W.cloud(n=8, seed=6)
    lev = LV.rotor(spec.n_lev, spec.B_K, 0.0 + 1e-30, spec.k_ul, spec.mass_amu)
    lev.A[:] = 0.0
    lev.A[1, 0] = 1e-300          # one (negligible) line so the rate layout has a pair
    g = krl.Grid(p)
    try:
        nm_t = torch.from_numpy(n_mol.reshape(-1)).cuda()
        pops = torch.zeros((p.ncell, lev.n), dtype=torch.float64, device="cuda")
        gam = torch.zeros((1, p.ncell), dtype=torch.float64, device="cuda")
        g.levels_solve(_desc(krl, lev, nm_t), gam, pops)
        got = pops.cpu().numpy()
    finally:
        g.close()
    ref = LV.boltzmann(lev, p.T_K, n_mol.reshape(-1))
    assert np.allclose(got, ref, rtol=1e-10)


def test_lambda_iteration_matches_oracle():
    """One device cycle (FP32 walk) against the oracle's (FP64 walk) on the
    same packet streams: the populations agree to the Monte Carlo level."""
    krl = need_gpu()
    import torch
    p, n_mol, spec = W.cloud(n=12, seed=7, packets_per_line=20000)
    lev = LV.rotor(spec.n_lev, spec.B_K, spec.A1, spec.k_ul, spec.mass_amu)
    N, seed = 20000, 3
    g = krl.Grid(p)
    try:
        nm_t = torch.from_numpy(n_mol.reshape(-1)).cuda()
        pops = torch.zeros((p.ncell, lev.n), dtype=torch.float64, device="cuda")
        ch = g.levels_iterate(_desc(krl, lev, nm_t), 2, N, seed, pops, init_lte=True)
        got = pops.cpu().numpy()
    finally:
        g.close()
    ref, rch = LV.lambda_iterate(oracle, p, n_mol, lev, 2, N, seed)
    nm = n_mol.reshape(-1)[:, None]
    frac_diff = np.abs(got - ref) / nm
    assert np.allclose(got.sum(axis=1), nm[:, 0], rtol=1e-10)
    assert np.median(frac_diff) < 2e-3 and frac_diff.max() < 0.05, (np.median(frac_diff), frac_diff.max())
    assert abs(ch[0] - rch[0]) < 0.1 * rch[0] + 1e-3
    # the iteration moves the populations away from LTE toward subthermal excitation
    lte = LV.boltzmann(lev, p.T_K, n_mol.reshape(-1))
    assert np.mean(got[:, 0] > lte[:, 0]) > 0.9


def test_lambda_iteration_settles_at_the_sampling_floor():
    """Sec. 2.1.3 runs the Lambda iteration to convergence without a stated
    criterion. After the first cycle the largest population change over the
    cells, max |dn| / n_mol, stops falling: what is left is the Monte Carlo
    noise of the radiative rates, so 4x the packets per line roughly halves
    that floor (N^-1/2), and the floor shows no trend over the cycles."""
    krl = need_gpu()
    import torch
    p, n_mol, spec = W.cloud(n=16, seed=11, packets_per_line=200_000)
    lev = LV.rotor(spec.n_lev, spec.B_K, spec.A1, spec.k_ul, spec.mass_amu)
    g = krl.Grid(p)
    try:
        nm_t = torch.from_numpy(n_mol.reshape(-1)).cuda()
        pops = torch.zeros((p.ncell, lev.n), dtype=torch.float64, device="cuda")
        ch1 = np.asarray(g.levels_iterate(_desc(krl, lev, nm_t), 8, 200_000, 5, pops, init_lte=True))
        ch4 = np.asarray(g.levels_iterate(_desc(krl, lev, nm_t), 5, 800_000, 6, pops, init_lte=True))
    finally:
        g.close()
    floor1, floor4 = np.median(ch1[1:]), np.median(ch4[1:])
    report("lambda_floor_16cube", floor_2e5=floor1, floor_8e5=floor4, ratio=floor1 / floor4,
           first_change=float(ch1[0]), changes=[float(c) for c in ch1])
    assert ch1[0] > 1.5 * floor1                        # the first cycle leaves LTE
    assert 1.3 < floor1 / floor4 < 3.0, (floor1, floor4)
    # no drift: the later cycles' floor matches the earlier cycles'
    assert abs(np.median(ch1[1:4]) - np.median(ch1[4:])) < 0.35 * floor1, ch1
