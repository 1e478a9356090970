"""The seeded synthetic inputs follow the recipes their docstrings state:
depths, velocity laws, density laws, random-field normalisation and
spectra, the many-model draw, and reproducibility from the seed."""
import math

import numpy as np

import workloads as W


def test_slab_and_sphere_depths_and_flow():
    s = W.slab(tau0=1e4, nz=64)
    assert s.shape == (64, 1, 1) and np.allclose(s.opacity, 1e4 / 32)
    assert s.periodic == (True, True, False) and s.source.plane == 32
    p = W.sphere(vmax_kms=200.0, tau0=1e6, n=16)
    R = 8.0
    x, y, z = np.meshgrid(np.arange(16) + 0.5, np.arange(16) + 0.5, np.arange(16) + 0.5, indexing="ij")
    r = np.sqrt((x - R) ** 2 + (y - R) ** 2 + (z - R) ** 2)          # symmetric: axis order irrelevant
    assert np.allclose(p.opacity[r < R], 1e6 / R) and np.all(p.opacity[r >= R] == 0)
    speed = np.sqrt((p.vel_cms.astype(np.float64) ** 2).sum(axis=0))
    assert np.allclose(speed, 200e5 * r / R, rtol=1e-6)
    assert p.source.pos == (R, R, R)


def test_envelope_laws():
    p = W.envelope(n=32)
    AU, G, Msun = 1.495978707e13, 6.67430e-8, 1.98892e33
    cell = 2000.0 * AU / 32
    c = np.arange(32) + 0.5 - 16
    Z, Y, X = np.meshgrid(c * cell, c * cell, c * cell, indexing="ij")
    r = np.sqrt(X * X + Y * Y + Z * Z)
    out = r >= 100 * AU
    nH2 = p.n_coll.astype(np.float64)
    assert np.all(nH2[~out] == 0)
    assert np.allclose(nH2[out], 1e6 * (r[out] / (100 * AU)) ** -1.5, rtol=1e-6)
    assert np.allclose(p.source.rate, 1e-4 * nH2, rtol=1e-6)
    assert np.allclose(p.opacity, 0.09 * 1e-4 * nH2, rtol=1e-6)
    V = p.vel_cms.astype(np.float64)
    v_r = (V[0] * X + V[1] * Y + V[2] * Z) / np.where(out, r, 1.0)
    GM = G * Msun
    assert np.allclose(v_r[out], -np.sqrt(2 * GM / r[out]), rtol=1e-5)           # free-fall infall
    Rc = np.sqrt(X * X + Y * Y)
    v_phi = (-V[0] * Y + V[1] * X) / np.where(Rc > 0, Rc, 1.0)
    m = out & (Rc > 0)
    assert np.allclose(v_phi[m], np.sqrt(GM / r[m]) * Rc[m] / r[m], rtol=1e-5)   # Keplerian about z
    v0, dv, n_ch = p.channels
    assert n_ch == 16 and math.isclose(v0, -5e5) and math.isclose(v0 + n_ch * dv, 5e5)
    assert [round(math.degrees(t)) for t, _ in p.cameras] == [0, 45, 90]


def test_cloud_normalisation_and_spectra():
    p, n_mol, spec = W.cloud(n=32, seed=3)
    dens = p.n_coll.astype(np.float64)
    assert math.isclose(dens.mean(), 1e3, rel_tol=1e-6)
    assert np.allclose(n_mol, 1e-4 * dens, rtol=1e-6)
    lnrho = np.log(dens / dens.mean())
    assert math.isclose((lnrho - lnrho.mean()).std(), 1.5, rel_tol=1e-4)
    for comp in p.vel_cms.astype(np.float64):
        assert math.isclose(comp.std(), 1e5, rel_tol=1e-5) and abs(comp.mean()) < 1e-6 * 1e5
    # the velocity field's shell-averaged power falls as k^-4 (fit over the inertial range)
    f = np.fft.rfftn(p.vel_cms[0].astype(np.float64))
    kz = np.fft.fftfreq(32)[:, None, None]
    ky = np.fft.fftfreq(32)[None, :, None]
    kx = np.fft.rfftfreq(32)[None, None, :]
    k = np.sqrt(kx * kx + ky * ky + kz * kz)
    bins = np.arange(2, 12) / 32
    pw = [np.mean(np.abs(f[(k >= lo) & (k < hi)]) ** 2) for lo, hi in zip(bins[:-1], bins[1:])]
    slope = np.polyfit(np.log(0.5 * (bins[:-1] + bins[1:])), np.log(pw), 1)[0]
    assert abs(slope + 4.0) < 0.4, slope
    p2, n2, _ = W.cloud(n=32, seed=3)
    assert np.array_equal(n_mol, n2) and np.array_equal(p.vel_cms, p2.vel_cms)
    E, g, A, kc = spec.arrays()
    assert np.allclose(E, 2.77 * np.arange(5) * np.arange(1, 6)) and np.allclose(g, 2 * np.arange(5) + 1)
    assert np.isclose(A[4, 3], 1e-7 * 64) and A[3, 1] == 0 and np.all(kc[np.tril_indices(5, -1)] == 1e-11)


def test_model_set_draw():
    ms = W.model_set(n_models=64, total_packets=10_000_000, seed=4)
    assert len(ms) == 64
    sides = {p.shape[0] for p in ms}
    assert sides <= {32, 48, 64, 96, 128}
    taus = np.array([p.opacity.max() * p.shape[0] / 2 for p in ms])
    assert taus.min() >= 1e3 * (1 - 1e-5) and taus.max() <= 1e7 * (1 + 1e-5)
    npk = np.array([p.n_packets for p in ms])
    assert npk.sum() <= 10_000_000 and np.allclose(npk / npk.sum(), taus / taus.sum(), rtol=0.02, atol=1e-6)
    again = W.model_set(n_models=64, total_packets=10_000_000, seed=4)
    assert [p.name for p in again] == [p.name for p in ms]
