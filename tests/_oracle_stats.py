"""Reductions of a transport run used by the statistical parity gates (test
infrastructure; imported by the tests and by tests/golden/make_oracle_runs.py).

None of this is the method's arithmetic: it only bins what a run produced
(per-packet scattering counts, the per-cell scattering map) so that an FP32
GPU run and a stored FP64 oracle run can be compared on equal terms.
"""
from __future__ import annotations

import hashlib
import json
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN_RUNS = os.path.join(HERE, "golden", "oracle_runs")
ORACLE_DIR = os.path.join(os.path.dirname(HERE), "oracle")
# oracle sources recorded with a stored run; the walk and the tables decide
# its numbers, so those two must be unchanged for the run to stay valid
ORACLE_SOURCES = ("transport.c", "tables.py", "__init__.py")
CHECKED_SOURCES = ("transport.c", "tables.py")

# log10(nscat) histogram: [0, 9) in steps of 0.05, plus one bin for nscat = 0
NSCAT_LOG_LO, NSCAT_LOG_HI, NSCAT_LOG_BINS = 0.0, 9.0, 180
N_SHELLS = 8


def oracle_digest() -> dict:
    """sha256 of each oracle source file."""
    out = {}
    for name in ORACLE_SOURCES:
        with open(os.path.join(ORACLE_DIR, name), "rb") as f:
            out[name] = hashlib.sha256(f.read()).hexdigest()
    return out


def nscat_hist(nscat) -> np.ndarray:
    """Counts of packets per log10(nscat) bin; element 0 counts nscat == 0."""
    v = np.asarray(nscat, dtype=np.float64)
    zero = int((v == 0).sum())
    lv = np.log10(v[v > 0])
    h, _ = np.histogram(np.clip(lv, NSCAT_LOG_LO, NSCAT_LOG_HI - 1e-9), bins=NSCAT_LOG_BINS,
                        range=(NSCAT_LOG_LO, NSCAT_LOG_HI))
    return np.concatenate([[zero], h]).astype(np.int64)


def shell_index(shape) -> np.ndarray:
    """Shell of every cell of a cube of side n: floor(r / (n/16)) of its
    centre's distance r from the cube's centre, capped at N_SHELLS (the cells
    outside the inscribed sphere, which hold no gas in the sphere workloads)."""
    nz, ny, nx = shape
    R = nx / 2.0
    z, y, x = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5, indexing="ij")
    r = np.sqrt((x - R) ** 2 + (y - R) ** 2 + (z - R) ** 2)
    k = np.floor(r / (R / N_SHELLS)).astype(np.int64)
    k[r >= R] = N_SHELLS
    return np.minimum(k, N_SHELLS).reshape(-1)


def shell_profile(scatmap, shape) -> np.ndarray:
    """Scatterings per shell (N_SHELLS + 1 entries)."""
    return np.bincount(shell_index(shape), weights=np.asarray(scatmap, dtype=np.float64).reshape(-1),
                       minlength=N_SHELLS + 1)


def beff(counts) -> float:
    """Effective number of bins (sum_i sqrt(p_i))^2 of a histogram: the
    expected relative L1 distance between two independent samples of N
    packets from it is about 2 sqrt(beff / (pi N))."""
    c = np.asarray(counts, dtype=np.float64)
    p = c / c.sum()
    return float(np.sqrt(p).sum() ** 2)


def l1_floor(counts, n: int) -> float:
    return 2.0 * math.sqrt(beff(counts) / (math.pi * n))


def load(name: str) -> dict:
    with open(os.path.join(GOLDEN_RUNS, name + ".json")) as f:
        return json.load(f)


def is_current(run: dict) -> bool:
    """True if the stored run was made with the present walk and tables."""
    now = oracle_digest()
    return all(run["oracle_sha256"].get(k) == now[k] for k in CHECKED_SOURCES)


def merged_shells(counts, weights) -> np.ndarray:
    """Shell counts with the sparse outer shells merged: working inwards
    from the outermost shell, a shell joins the next inner one until the
    group holds at least 1 % of all scatterings (by `weights`, the oracle's
    totals). Per-block means of shells that see a scattering only now and
    then are far from Gaussian, so they are not tested on their own."""
    c = np.asarray(counts, dtype=np.float64)
    w = np.asarray(weights, dtype=np.float64)
    tot = w.sum()
    out, acc_c, acc_w = [], 0.0, 0.0
    for k in range(w.size - 1, -1, -1):
        acc_c += c[..., k] if c.ndim > 1 else c[k]
        acc_w += w[k]
        if acc_w >= 0.01 * tot or k == 0:
            out.append(acc_c)
            acc_c, acc_w = 0.0, 0.0
    if acc_w:            # (only if the innermost shell closed a group early)
        out[-1] = out[-1] + acc_c
    return np.stack(out[::-1], axis=-1)


def shell_z(gpu_shells, n_gpu: int, run: dict) -> np.ndarray:
    """z-scores of the GPU's scatterings per packet in each shell (sparse
    outer shells merged, see merged_shells) against a stored oracle run. The
    oracle's standard error of the mean comes from the spread of its
    per-block means (blocks of n / batches packets, which are independent);
    the GPU's is taken equal (same distribution under the hypothesis that
    the two walks agree). Groups with no scatterings on either side get
    z = 0."""
    raw = np.asarray(run["shells_per_batch"], dtype=np.float64)
    weights = raw.sum(axis=0)
    blocks = merged_shells(raw, weights)
    gpu_shells = merged_shells(np.asarray(gpu_shells, dtype=np.float64), weights)
    B = blocks.shape[0]
    per = run["n"] // B
    means = blocks / per
    m_o = blocks.sum(axis=0) / run["n"]
    se = means.std(axis=0, ddof=1) / math.sqrt(B)
    m_g = np.asarray(gpu_shells, dtype=np.float64) / n_gpu
    z = np.zeros_like(m_o)
    nz = se > 0
    z[nz] = (m_g[nz] - m_o[nz]) / (math.sqrt(2.0) * se[nz])
    return z


def mean_nscat_z(nscat_gpu, run: dict) -> float:
    """z-score of the GPU's mean scatterings per packet against the stored
    run's (variances from both samples)."""
    g = np.asarray(nscat_gpu, dtype=np.float64)
    n = run["n"]
    m_o = run["nscat_sum"] / n
    v_o = run["nscat_sumsq"] / n - m_o * m_o
    se = math.sqrt(v_o / n + g.var() / g.size)
    return (g.mean() - m_o) / se
