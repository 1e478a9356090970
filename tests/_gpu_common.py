"""Helpers shared by the GPU parity tests (import only from tests)."""
import numpy as np
import pytest


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_09340_gb300 import build as b
    b.build()
    import paper_2608_09340_gb300 as krl
    krl.load_library()
    return krl


def gpu_run(krl, problem, precision, n=None, first=0, seed=None, records=True, tallies=True, **tune):
    import torch
    g = krl.Grid(problem)
    try:
        st, rc, rec = g.run(n=n, first=first, seed=seed, precision=precision, records=records, **tune)
        torch.cuda.synchronize()
        out = {"stats": st, "rc": rc, "info": g.info}
        if records:
            out["records"] = krl.records_to_numpy(rec)
        if tallies:
            for name in ("spec_w", "spec_n", "scatmap", "exc", "J", "emiss", "stats", "absw"):
                t = g.tally(name)
                out["stats_tally" if name == "stats" else name] = None if t is None else t.cpu().numpy()
        return out
    finally:
        g.close()


def agreement(gpu_rec, ref_rec, strict=True):
    """Per-packet agreement. strict (FP64 lockstep): status, scatterings,
    face crossings and emission cell all equal. Otherwise (FP32 walk): status
    and scatterings; FP32 rounding may move a scattering point across a
    periodic face, which adds a crossing without changing the walk."""
    ok = (gpu_rec["status"] == ref_rec["status"]) & (gpu_rec["nscat"] == ref_rec["nscat"])
    if strict:
        ok &= (gpu_rec["ncross"] == ref_rec["ncross"]) & (gpu_rec["cell0"] == ref_rec["cell0"])
    return ok


def rel_l1(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a - b).sum() / max(np.abs(b).sum(), 1e-300)


def chi2_two_sample(c1, c2, min_count=10):
    """Two-sample chi^2 on histograms of equal total (bins merged until each
    holds >= min_count counts in both); returns (stat, dof, p)."""
    from scipy.stats import chi2
    c1 = np.asarray(c1, dtype=np.float64)
    c2 = np.asarray(c2, dtype=np.float64)
    m1, m2 = [], []
    a = b = 0.0
    for x, y in zip(c1, c2):
        a += x
        b += y
        if a >= min_count and b >= min_count:
            m1.append(a)
            m2.append(b)
            a = b = 0.0
    if m1:
        m1[-1] += a
        m2[-1] += b
    m1, m2 = np.array(m1), np.array(m2)
    n1, n2 = m1.sum(), m2.sum()
    k1, k2 = np.sqrt(n2 / n1), np.sqrt(n1 / n2)
    stat = np.sum((k1 * m1 - k2 * m2) ** 2 / (m1 + m2))
    dof = len(m1) - 1
    return stat, dof, chi2.sf(stat, dof) if dof > 0 else 1.0


def x_peak(spec, lo, hi, guess):
    """Peak of an escaped spectrum folded to |x|: the histogram (bins of
    [lo, hi), symmetric about 0) smoothed with a Gaussian of width 0.1 guess,
    then a parabola through the largest smoothed bin and its neighbours."""
    c = np.asarray(spec, dtype=np.float64)
    n = c.size
    edges = np.linspace(lo, hi, n + 1)
    xc = 0.5 * (edges[1:] + edges[:-1])
    dx = edges[1] - edges[0]
    pos = xc > 0
    folded = c[pos] + c[~pos][::-1]
    xs = xc[pos]
    sig = 0.1 * guess / dx
    k = np.arange(-int(4 * sig) - 1, int(4 * sig) + 2)
    ker = np.exp(-0.5 * (k / sig) ** 2)
    sm = np.convolve(folded, ker / ker.sum(), mode="same")
    i = int(np.argmax(sm[1:-1])) + 1
    y0, y1, y2 = sm[i - 1], sm[i], sm[i + 1]
    den = y0 - 2 * y1 + y2
    off = 0.5 * (y0 - y2) / den if den != 0 else 0.0
    return xs[i] + off * dx
