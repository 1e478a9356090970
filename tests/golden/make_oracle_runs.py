"""Writes the stored FP64 oracle runs that the statistical GPU parity gates
compare against (tests/golden/oracle_runs/<case>.json).

Every number in those files comes from the oracle (``oracle.run``) on the
seeded workloads of ``workloads``; nothing is read from the CUDA path. A
file records the workload call, the packet-id range, the seed, the sha256 of
the oracle sources it was made with (a CPU test checks that they are still
current), and reductions of the run: the escaped-spectrum counts, the
counters, a log10 histogram of the scatterings per packet, their sum and
sum of squares, and, for the spheres, the scatterings per radial shell in
each of `batches` consecutive packet blocks (their spread gives the standard
error of the shell means).

These runs are long on a CPU (the 64^3, tau0 = 1e6 sphere needs about
1.3e6 scatterings per packet), which is why they are stored instead of
recomputed by each GPU test run.

    python tests/golden/make_oracle_runs.py [case ...] [--threads N]
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
import workloads as W  # noqa: E402
import _oracle_stats as S  # noqa: E402

# name -> (workload function, kwargs, first id, packets, seed, batches)
CASES = {
    # the static slab of the Neufeld test at the size where the two-sample
    # L1 noise floor of its 200-bin spectrum is below 1 %
    "slab64_tau1e4_n1e6_seed0": ("slab", {}, 0, 1_000_000, 0, 1),
    "slab64_tau1e4_n1e6_seed1": ("slab", {}, 0, 1_000_000, 1, 1),
    # the 64^3, tau0 = 1e6 sphere (static; outflow and infall at 200 km/s)
    "sphere64_tau1e6_static_n2e4_seed0": ("sphere", {}, 0, 20_000, 0, 20),
    "sphere64_tau1e6_static_n2e4_seed1": ("sphere", {}, 0, 20_000, 1, 20),
    # the static sphere at 2e5 packets (two-sample L1 floor ~2.3 %)
    "sphere64_tau1e6_static_n2e5_seed2": ("sphere", {}, 0, 200_000, 2, 20),
    "sphere64_tau1e6_out200_n2e5_seed0": ("sphere", {"vmax_kms": 200.0}, 0, 200_000, 0, 20),
    "sphere64_tau1e6_in200_n2e5_seed0": ("sphere", {"vmax_kms": -200.0}, 0, 200_000, 0, 20),
    # second seeds of the moving headline spheres, for their measured two-seed floors
    "sphere64_tau1e6_out200_n2e5_seed1": ("sphere", {"vmax_kms": 200.0}, 0, 200_000, 1, 20),
    "sphere64_tau1e6_in200_n2e5_seed1": ("sphere", {"vmax_kms": -200.0}, 0, 200_000, 1, 20),
    # the 32^3, tau0 = 1e5 moving spheres, at the size where their spectra's
    # two-sample floor is below 1 %; two seeds each for the measured floor
    "sphere32_tau1e5_out200_n6e5_seed0": ("sphere", {"vmax_kms": 200.0, "tau0": 1e5, "n": 32}, 0, 600_000, 0, 20),
    "sphere32_tau1e5_out200_n6e5_seed1": ("sphere", {"vmax_kms": 200.0, "tau0": 1e5, "n": 32}, 0, 600_000, 1, 20),
    "sphere32_tau1e5_in200_n6e5_seed0": ("sphere", {"vmax_kms": -200.0, "tau0": 1e5, "n": 32}, 0, 600_000, 0, 20),
    "sphere32_tau1e5_in200_n6e5_seed1": ("sphere", {"vmax_kms": -200.0, "tau0": 1e5, "n": 32}, 0, 600_000, 1, 20),
}


def problem_of(fn: str, kwargs: dict):
    return getattr(W, fn)(**kwargs)


def make(name: str, threads: int) -> dict:
    fn, kw, first, n, seed, batches = CASES[name]
    p = problem_of(fn, kw)
    spec = np.zeros(p.spectrum[2] + 2, np.int64)
    stats = np.zeros(8, np.int64)
    hist = np.zeros(S.NSCAT_LOG_BINS + 1, np.int64)
    s1 = 0
    s2 = 0.0
    shells = []
    t0 = time.time()
    per = n // batches
    for b in range(batches):
        lo = first + b * per
        m = per if b < batches - 1 else n - b * per
        r = oracle.run(p, n=m, first=lo, seed=seed, records=True, nthreads=threads)
        spec += r["spec_c"].astype(np.int64)
        stats += r["stats"].astype(np.int64)
        ns = r["records"]["nscat"].astype(np.int64)
        hist += S.nscat_hist(ns)
        s1 += int(ns.sum())
        s2 += float((ns.astype(np.float64) ** 2).sum())
        if r["scat"] is not None:
            shells.append(S.shell_profile(r["scat"], p.shape).astype(np.int64).tolist())
        print(f"{name}: block {b + 1}/{batches} done, {time.time() - t0:.0f} s", flush=True)
    out = {
        "case": name, "workload": {"fn": fn, "kwargs": kw}, "first": first, "n": n, "seed": seed,
        "batches": batches, "oracle_sha256": S.oracle_digest(),
        "host": {"machine": platform.machine(), "threads": threads}, "seconds": round(time.time() - t0, 1),
        "spec_c": spec.tolist(), "stats": stats.tolist(),
        "nscat_hist": hist.tolist(), "nscat_sum": s1, "nscat_sumsq": s2,
    }
    if shells:
        out["shells_per_batch"] = shells
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("cases", nargs="*")
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    a = ap.parse_args()
    oracle.build()
    os.makedirs(S.GOLDEN_RUNS, exist_ok=True)
    for name in a.cases or list(CASES):
        d = make(name, a.threads)
        with open(os.path.join(S.GOLDEN_RUNS, name + ".json"), "w") as f:
            json.dump(d, f, separators=(",", ":"))
            f.write("\n")
        print(f"wrote {name} ({d['seconds']} s)", flush=True)


if __name__ == "__main__":
    main()
