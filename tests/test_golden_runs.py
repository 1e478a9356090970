"""The stored FP64 oracle runs (tests/golden/oracle_runs, written by
tests/golden/make_oracle_runs.py) that the statistical GPU gates compare
against: every case is present, made with the current walk and tables,
self-consistent, and -- being large oracle runs -- it is checked once more
against what the paper and the physics fix at that size."""
import importlib.util
import math
import os

import numpy as np
import pytest

import _oracle_stats as S
from _gpu_common import x_peak

HERE = os.path.dirname(os.path.abspath(__file__))


def _cases():
    spec = importlib.util.spec_from_file_location("make_oracle_runs", os.path.join(HERE, "golden", "make_oracle_runs.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.CASES


CASES = _cases()


@pytest.mark.parametrize("name", sorted(CASES))
def test_stored_run_is_current_and_consistent(name):
    run = S.load(name)
    fn, kw, first, n, seed, batches = CASES[name]
    assert (run["workload"]["fn"], run["workload"]["kwargs"], run["first"], run["n"], run["seed"]) == \
        (fn, kw, first, n, seed)
    assert S.is_current(run), f"{name}: oracle walk or tables changed since the run was stored"
    spec = np.asarray(run["spec_c"], dtype=np.int64)
    st = np.asarray(run["stats"], dtype=np.int64)
    assert st[0] == n == spec.sum() == st[1]                 # every packet escapes (no destruction)
    assert sum(run["nscat_hist"]) == n
    assert run["nscat_sum"] == st[4]
    if "shells_per_batch" in run:
        sh = np.asarray(run["shells_per_batch"], dtype=np.int64)
        assert sh.shape == (batches, S.N_SHELLS + 1)
        assert sh.sum() == st[4]
        assert sh[:, S.N_SHELLS].sum() == 0                   # no gas outside the sphere


def test_slab_peak_and_symmetry_at_1e6_packets():
    """Static slab, a tau0 = 100: the peaks sit near the Neufeld value
    +-1.0664 (a tau0)^{1/3} = +-4.95 (loose at this a tau0: 10 %), and the
    spectrum is symmetric about line centre (chi^2 of mirrored halves)."""
    from _gpu_common import chi2_two_sample
    run = S.load("slab64_tau1e4_n1e6_seed0")
    c = np.asarray(run["spec_c"][1:-1], dtype=np.float64)
    pred = 1.0664 * (1e-2 * 1e4) ** (1.0 / 3.0)
    assert abs(x_peak(c, -30.0, 30.0, pred) / pred - 1.0) < 0.10
    half = c.size // 2
    assert chi2_two_sample(c[:half][::-1], c[half:])[2] > 1e-3


def test_sphere_runs_against_the_physics():
    """64^3 sphere, a tau0 = 470: the static spectrum peaks near the
    sphere's +-0.931 (a tau0)^{1/3} (15 %) and is symmetric; the mean number
    of scatterings per packet is of order tau0; outflow escapes red (x < 0)
    and infall blue, as mirror images of each other (velocity reversal)."""
    from _gpu_common import chi2_two_sample
    st = S.load("sphere64_tau1e6_static_n2e4_seed0")
    c = np.asarray(st["spec_c"][1:-1], dtype=np.float64)
    pred = 0.931 * (4.7e-4 * 1e6) ** (1.0 / 3.0)
    assert abs(x_peak(c, -60.0, 60.0, pred) / pred - 1.0) < 0.15
    assert chi2_two_sample(c[:200][::-1], c[200:])[2] > 1e-3
    assert 5e5 < st["nscat_sum"] / st["n"] < 3e6
    out = np.asarray(S.load("sphere64_tau1e6_out200_n2e5_seed0")["spec_c"], dtype=np.float64)
    inn = np.asarray(S.load("sphere64_tau1e6_in200_n2e5_seed0")["spec_c"], dtype=np.float64)
    assert out[1:201].sum() / out.sum() > 0.9 and inn[201:-1].sum() / inn.sum() > 0.9
    assert chi2_two_sample(out, inn[::-1])[2] > 1e-3


def test_static_sphere_at_2e5_packets():
    """The 2e5-packet static headline run (third seed): its peak sits at the
    sphere's 0.931 (a tau0)^{1/3} within 5 % (the 2e4-packet runs allow 15 %),
    its spectrum is symmetric, and it agrees with the independent 2e4-packet
    run of seed 0 (two-sample chi^2)."""
    from _gpu_common import chi2_two_sample
    big = S.load("sphere64_tau1e6_static_n2e5_seed2")
    c = np.asarray(big["spec_c"][1:-1], dtype=np.float64)
    pred = 0.931 * (4.7e-4 * 1e6) ** (1.0 / 3.0)
    assert abs(x_peak(c, -60.0, 60.0, pred) / pred - 1.0) < 0.05
    assert chi2_two_sample(c[:200][::-1], c[200:])[2] > 1e-3
    small = S.load("sphere64_tau1e6_static_n2e4_seed0")
    assert chi2_two_sample(np.asarray(small["spec_c"]), np.asarray(big["spec_c"]))[2] > 1e-3
    assert abs(big["nscat_sum"] / big["n"] / (small["nscat_sum"] / small["n"]) - 1.0) < 0.03


def test_two_seed_floors_match_their_expectation():
    """The measured two-seed L1 distance of each pair of stored runs sits at
    its expected value 2 sqrt(B_eff / (pi N)) (within 25 %): the stored
    runs are independent samples of one distribution."""
    from _gpu_common import rel_l1
    for a, b in [("sphere64_tau1e6_static_n2e4_seed0", "sphere64_tau1e6_static_n2e4_seed1"),
                 ("slab64_tau1e4_n1e6_seed0", "slab64_tau1e4_n1e6_seed1"),
                 ("sphere64_tau1e6_out200_n2e5_seed0", "sphere64_tau1e6_out200_n2e5_seed1"),
                 ("sphere64_tau1e6_in200_n2e5_seed0", "sphere64_tau1e6_in200_n2e5_seed1"),
                 ("sphere32_tau1e5_out200_n6e5_seed0", "sphere32_tau1e5_out200_n6e5_seed1"),
                 ("sphere32_tau1e5_in200_n6e5_seed0", "sphere32_tau1e5_in200_n6e5_seed1")]:
        ra, rb = S.load(a), S.load(b)
        ca, cb = np.asarray(ra["spec_c"]), np.asarray(rb["spec_c"])
        got = rel_l1(cb, ca)
        exp = S.l1_floor(ca + cb, ra["n"])
        assert abs(got / exp - 1.0) < 0.25, (a, got, exp)
        assert math.isfinite(got)


def test_two_seed_shell_z_is_moderate():
    """The shell z-scores of one stored oracle run against another seed's
    (independent samples of one distribution) stay within the gate the GPU
    comparisons use (|z| < 4.5), with the sparse outer shells merged."""
    for a, b in [("sphere64_tau1e6_static_n2e4_seed0", "sphere64_tau1e6_static_n2e4_seed1"),
                 ("sphere64_tau1e6_out200_n2e5_seed0", "sphere64_tau1e6_out200_n2e5_seed1"),
                 ("sphere64_tau1e6_in200_n2e5_seed0", "sphere64_tau1e6_in200_n2e5_seed1"),
                 ("sphere32_tau1e5_out200_n6e5_seed0", "sphere32_tau1e5_out200_n6e5_seed1"),
                 ("sphere32_tau1e5_in200_n6e5_seed0", "sphere32_tau1e5_in200_n6e5_seed1")]:
        ra, rb = S.load(a), S.load(b)
        z = S.shell_z(np.asarray(rb["shells_per_batch"], dtype=np.float64).sum(axis=0), rb["n"], ra)
        assert np.abs(z).max() < 4.5, (a, z)
