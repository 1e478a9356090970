"""Seeded synthetic workloads for the Monte Carlo line-transfer pass.

This module only builds inputs: grids of per-cell fields in physical units,
line constants, source and tally specifications. It holds none of the
method's arithmetic (no Doppler widths, cross sections, profiles or
redistribution); both the CUDA path and the FP64 oracle derive those
themselves from what is given here.

Every field is float32, C-order [nz][ny][nx], because the method keeps its
per-cell fields in single precision (Sec. 2.3).

Workloads (shapes follow the paper's validation and application setups):

* ``slab``      - plane-parallel static slab, 64 cells along z, periodic in x/y
                  (Sec. 3.1, the Neufeld test, line-centre convention).
* ``sphere``    - uniform sphere on a 64^3 grid with a Hubble-like radial flow
                  (static, outflow or infall) and a central point source.
* ``thin_slab`` - optically thin moving slab lit by an in-plane beam and seen
                  face-on (Sec. 3.3, Eq. thin-slab).
* ``dusty_slab`` - the slab with uniform continuum absorption (Sec. 3.2).
* ``box``       - uniform cube with a volume source and thermal emission
                  profile (Sec. 3.5.2, Table 1 setup).
* ``envelope``  - rotating, infalling envelope with an inner cavity and
                  volume source, several cameras and velocity channels.
* ``model_set`` - a set of independent spheres of uneven size and depth for
                  the batched launch.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

# Mass of a hydrogen atom in atomic mass units (the resonance-line workloads).
HYDROGEN_AMU = 1.00794
# Lyman-alpha rest frequency [Hz]; only enters when opacity is given as n_l.
LYA_NU0_HZ = 2.466e15
LYA_A_UL = 6.265e8

SOURCE_POINT = "point"
SOURCE_PLANE = "plane"
SOURCE_BEAM = "beam"
SOURCE_VOLUME = "volume"

PROFILE_LINE_CENTRE = "line_centre"
PROFILE_GAUSSIAN = "gaussian"


@dataclasses.dataclass
class Line:
    nu0_hz: float
    mass_amu: float
    A_ul: float
    g_u: float = 3.0
    g_l: float = 1.0
    k_ul: float = 0.0          # collisional de-excitation coefficient [cm^3 s^-1]
    a_fixed: float = 0.0       # > 0: damping parameter given directly
    ph_mode: int = 2           # profile mode: 2 = 1-D slice, 1 = 2-D table, 3 = core-wing blend


@dataclasses.dataclass
class Source:
    kind: str = SOURCE_POINT
    pos: tuple = (0.0, 0.0, 0.0)   # point position in cell units (x, y, z)
    axis: int = 2                  # plane normal / beam travel axis (0=x, 1=y, 2=z)
    plane: float = 0.0             # plane source: coordinate in cell units along `axis`
    band_axis: int = -1            # beam: transverse axis whose entry range is limited
    band: tuple = (0.0, 0.0)       # beam: [lo, hi) along band_axis in cell units
    profile: str = PROFILE_LINE_CENTRE
    luminosity: float = 1.0        # photons per second carried by the whole run
    rate: Optional[np.ndarray] = None  # volume source: per-cell emission rate


@dataclasses.dataclass
class Problem:
    name: str
    shape: tuple                   # (nz, ny, nx)
    cell_cm: float
    periodic: tuple                # (x, y, z) periodic flags
    opacity_kind: str              # "tau": line-centre optical depth per cell width
                                   # "n_l": lower-level density [cm^-3]
    opacity: np.ndarray            # float32 [nz, ny, nx]
    T_K: float
    line: Line
    source: Source
    vel_cms: Optional[np.ndarray] = None    # float32 [3, nz, ny, nx] (vx, vy, vz) [cm/s]
    n_coll: Optional[np.ndarray] = None     # float32 [nz, ny, nx] collider density [cm^-3]
    tau_abs: Optional[np.ndarray] = None    # float32 [nz, ny, nx] continuum (dust) absorption
                                            # optical depth per cell width
    spectrum: tuple = (-30.0, 30.0, 200)    # escaped spectrum bins in x: (lo, hi, n)
    channels: Optional[tuple] = None        # (v_min [cm/s], dv [cm/s], n_ch)
    cameras: tuple = ()                     # ((theta, phi), ...) in radians
    tallies: tuple = ()                     # subset of {"scatmap", "exc", "J", "emiss"}
    n_packets: int = 10_000
    seed: int = 0

    @property
    def ncell(self) -> int:
        nz, ny, nx = self.shape
        return nx * ny * nz


def _cell_centres(shape):
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5,
                          np.arange(nx) + 0.5, indexing="ij")
    return x, y, z


def slab(tau0: float = 1e4, a: float = 1e-2, nz: int = 64, n_packets: int = 10_000,
         seed: int = 0, T_K: float = 1e4, bins: tuple = (-30.0, 30.0, 200),
         tallies: tuple = ()) -> Problem:
    """Static slab, half-thickness line-centre depth tau0 over nz/2 cells,
    1x1 periodic transverse cell, line-centre photons from the midplane."""
    tau_cell = tau0 / (nz / 2)
    op = np.full((nz, 1, 1), tau_cell, dtype=np.float32)
    return Problem(
        name=f"slab_tau{tau0:g}_a{a:g}", shape=(nz, 1, 1), cell_cm=1.0e13,
        periodic=(True, True, False), opacity_kind="tau", opacity=op, T_K=T_K,
        line=Line(LYA_NU0_HZ, HYDROGEN_AMU, LYA_A_UL, 6.0, 2.0, 0.0, a),
        source=Source(SOURCE_PLANE, axis=2, plane=nz / 2, profile=PROFILE_LINE_CENTRE),
        spectrum=bins, tallies=tallies, n_packets=n_packets, seed=seed)


def sphere(vmax_kms: float = 0.0, tau0: float = 1e6, a: float = 4.7e-4, n: int = 64,
           n_packets: int = 1_000_000, seed: int = 0, T_K: float = 1e4,
           bins: tuple = (-60.0, 60.0, 400), tallies: tuple = ("scatmap",)) -> Problem:
    """Uniform sphere of radius n/2 cells (cell centres inside), centre-to-edge
    line-centre depth tau0, radial velocity v = vmax * r / R, central point
    source at line centre."""
    R = n / 2
    x, y, z = _cell_centres((n, n, n))
    dx, dy, dz = x - R, y - R, z - R
    r = np.sqrt(dx * dx + dy * dy + dz * dz)
    inside = r < R
    op = np.where(inside, tau0 / R, 0.0).astype(np.float32)
    vel = None
    if vmax_kms != 0.0:
        s = vmax_kms * 1e5 / R
        vel = np.stack([s * dx, s * dy, s * dz]).astype(np.float32)
    return Problem(
        name=f"sphere{n}_tau{tau0:g}_v{vmax_kms:g}", shape=(n, n, n), cell_cm=1.0e15,
        periodic=(False, False, False), opacity_kind="tau", opacity=op, T_K=T_K,
        line=Line(LYA_NU0_HZ, HYDROGEN_AMU, LYA_A_UL, 6.0, 2.0, 0.0, a),
        source=Source(SOURCE_POINT, pos=(R, R, R), profile=PROFILE_LINE_CENTRE),
        vel_cms=vel, spectrum=bins, tallies=tallies, n_packets=n_packets, seed=seed)


def dusty_slab(tau_a: float, tau0: float = 1e5, a: float = 0.015, nz: int = 64, n_packets: int = 200_000,
               seed: int = 0, bins: tuple = (-60.0, 60.0, 240), tallies: tuple = ()) -> Problem:
    """Static slab with uniform continuum (dust) absorption (Sec. 3.2): T =
    10 K (a = 0.015 for the resonance line), line-centre depth tau0 and
    absorption depth tau_a from the midplane to a face, a central plane of
    line-centre photons, transverse axes periodic."""
    p = slab(tau0=tau0, a=a, nz=nz, n_packets=n_packets, seed=seed, T_K=10.0, bins=bins, tallies=tallies)
    p.name = f"dusty_slab_tau{tau0:g}_a{a:g}_taua{tau_a:g}"
    p.tau_abs = np.full(p.shape, tau_a / (nz / 2), dtype=np.float32)
    return p


def box(tau0: float = 1e3, a: float = 4.73e-3, n: int = 32, T_K: float = 100.0,
        n_packets: int = 100_000, seed: int = 0, bins: tuple = (-20.0, 20.0, 200),
        tallies: tuple = ()) -> Problem:
    """Uniform cube, centre-to-face line-centre depth tau0, uniform volume
    source with a thermal (Gaussian) emission profile (Sec. 3.5.2)."""
    op = np.full((n, n, n), tau0 / (n / 2), dtype=np.float32)
    rate = np.ones((n, n, n), dtype=np.float32)
    return Problem(
        name=f"box{n}_tau{tau0:g}", shape=(n, n, n), cell_cm=1.0e15,
        periodic=(False, False, False), opacity_kind="tau", opacity=op, T_K=T_K,
        line=Line(LYA_NU0_HZ, HYDROGEN_AMU, LYA_A_UL, 6.0, 2.0, 0.0, a),
        source=Source(SOURCE_VOLUME, profile=PROFILE_GAUSSIAN, rate=rate),
        spectrum=bins, tallies=tallies, n_packets=n_packets, seed=seed)


def thin_slab(tau0: float = 0.01, a: float = 0.01, nt: int = 4, b_kms: float = 1.0,
              n_ch: int = 32, n_packets: int = 200_000, seed: int = 0) -> Problem:
    """Optically thin moving slab (Sec. 3.3, Eq. thin-slab).

    Grid (nz, ny, nx) = (3, nt, nt), periodic in y, open in x and z. The
    slab is the middle z layer (one cell thick, line-centre depth tau0 along
    its normal z) and moves at v_z = b toward a face-on camera looking down
    +z. A plane-parallel beam of line-centre photons enters the x = 0 face
    inside the slab layer and travels along +x, i.e. in the slab plane, so
    the scattering angle toward the camera is 90 degrees (g = 0).
    T_K = 60.6137 K is the temperature at which a hydrogen atom's thermal
    Doppler width is 1 km/s; channels span +-5 b_kms."""
    T_K = 60.6137
    op = np.zeros((3, nt, nt), dtype=np.float32)
    op[1] = tau0
    vel = np.zeros((3, 3, nt, nt), dtype=np.float32)
    vel[2, 1] = b_kms * 1e5
    half = 5.0 * b_kms * 1e5
    dv = 2.0 * half / n_ch
    return Problem(
        name=f"thin_slab_tau{tau0:g}", shape=(3, nt, nt), cell_cm=1.0e14,
        periodic=(False, True, False), opacity_kind="tau", opacity=op, T_K=T_K,
        line=Line(LYA_NU0_HZ, HYDROGEN_AMU, LYA_A_UL, 6.0, 2.0, 0.0, a),
        source=Source(SOURCE_BEAM, axis=0, band_axis=2, band=(1.0, 2.0),
                      profile=PROFILE_LINE_CENTRE),
        vel_cms=vel, spectrum=(-10.0, 10.0, 100), channels=(-half, dv, n_ch),
        cameras=((0.0, 0.0),), tallies=("emiss",), n_packets=n_packets, seed=seed)


def envelope(n: int = 64, n_ch: int = 16, n_packets: int = 100_000, seed: int = 0,
             box_au: float = 2000.0, r_in_au: float = 100.0, n_in: float = 1e6,
             abundance: float = 1e-4, T_K: float = 30.0, M_sun: float = 1.0,
             v_half_kms: float = 5.0, k_ul: float = 1e-11,
             cameras_deg: tuple = (0.0, 45.0, 90.0)) -> Problem:
    """Rotating, infalling envelope: n_H2 = n_in (r / r_in)^-1.5 outside an
    inner cavity r_in, emitter abundance 1e-4, free-fall infall plus
    Keplerian rotation about z around a point mass, a rotor J=1-0 line at
    115.27 GHz (A = 1e-7 s^-1, g_u = 3, g_l = 1, 28 amu), volume source
    proportional to the emitter density, channels spanning +-v_half.
    The lower level holds a fixed fraction 0.09 of the emitters (about the
    J=0 share of a B/k = 2.77 K rotor at 30 K), stated here as an input."""
    AU = 1.495978707e13
    G = 6.67430e-8
    Msun = 1.98892e33
    cell = box_au * AU / n
    x, y, z = _cell_centres((n, n, n))
    c = n / 2
    dx, dy, dz = (x - c) * cell, (y - c) * cell, (z - c) * cell
    r = np.sqrt(dx * dx + dy * dy + dz * dz)
    r_in = r_in_au * AU
    nH2 = np.where(r >= r_in, n_in * (np.maximum(r, r_in) / r_in) ** -1.5, 0.0)
    n_mol = abundance * nH2
    GM = G * M_sun * Msun
    rs = np.maximum(r, 0.5 * cell)
    v_ff = np.sqrt(2.0 * GM / rs)
    v_k = np.sqrt(GM / rs)
    Rcyl = np.sqrt(dx * dx + dy * dy)
    # radial infall
    vx = -v_ff * dx / rs
    vy = -v_ff * dy / rs
    vz = -v_ff * dz / rs
    # rotation about +z: phi-hat = (-y, x, 0) / Rcyl, scaled by Rcyl / r
    with np.errstate(invalid="ignore", divide="ignore"):
        vx += np.where(Rcyl > 0, -v_k * dy / rs, 0.0)
        vy += np.where(Rcyl > 0, v_k * dx / rs, 0.0)
    inside = r >= r_in
    vel = np.stack([np.where(inside, vx, 0.0), np.where(inside, vy, 0.0),
                    np.where(inside, vz, 0.0)]).astype(np.float32)
    dv = 2.0 * v_half_kms * 1e5 / n_ch
    return Problem(
        name=f"envelope{n}", shape=(n, n, n), cell_cm=cell, periodic=(False, False, False),
        opacity_kind="n_l", opacity=(0.09 * n_mol).astype(np.float32), T_K=T_K,
        line=Line(115.27e9, 28.0, 1e-7, 3.0, 1.0, k_ul, 0.0),
        source=Source(SOURCE_VOLUME, profile=PROFILE_GAUSSIAN,
                      rate=n_mol.astype(np.float32)),
        vel_cms=vel, n_coll=nH2.astype(np.float32),
        spectrum=(-40.0, 40.0, 160), channels=(-v_half_kms * 1e5, dv, n_ch),
        cameras=tuple((math.radians(t), 0.0) for t in cameras_deg),
        tallies=("exc", "J", "emiss"), n_packets=n_packets, seed=seed)


def gaussian_field(shape, slope: float, rng) -> np.ndarray:
    """Periodic Gaussian random field with 3-D power spectrum P(k) ~ k^slope,
    zero mean and unit variance (white noise shaped in Fourier space)."""
    nz, ny, nx = shape
    kz = np.fft.fftfreq(nz)[:, None, None]
    ky = np.fft.fftfreq(ny)[None, :, None]
    kx = np.fft.rfftfreq(nx)[None, None, :]
    k = np.sqrt(kx * kx + ky * ky + kz * kz)
    amp = np.zeros_like(k)
    amp[k > 0] = k[k > 0] ** (slope / 2.0)
    f = np.fft.irfftn(np.fft.rfftn(rng.normal(size=shape)) * amp, s=shape, axes=(0, 1, 2))
    return (f - f.mean()) / f.std()


@dataclasses.dataclass
class LevelSpec:
    """Levels of a linear rotor for the statistical-equilibrium workloads."""
    n_lev: int = 5
    B_K: float = 2.77            # E_J = B J (J + 1)
    A1: float = 1e-7             # A_{J -> J-1} = A1 J^3
    k_ul: float = 1e-11          # collisional de-excitation, every pair u > l
    mass_amu: float = 28.0

    def arrays(self):
        """The level data as arrays: energies E_J / k_B = B J (J + 1) [K],
        degeneracies 2J + 1, A[u][l] (A1 u^3 for l = u - 1, else 0) and the
        collision coefficients k[u][l] (k_ul for every u > l)."""
        J = np.arange(self.n_lev, dtype=np.float64)
        A = np.zeros((self.n_lev, self.n_lev))
        k = np.zeros((self.n_lev, self.n_lev))
        for u in range(1, self.n_lev):
            A[u, u - 1] = self.A1 * u ** 3
            k[u, :u] = self.k_ul
        return self.B_K * J * (J + 1.0), 2.0 * J + 1.0, A, k


def cloud(n: int = 128, seed: int = 3, mean_n: float = 1e3, sigma_lnrho: float = 1.5, T_K: float = 20.0,
          sigma_v_kms: float = 1.0, abundance: float = 1e-4, box_pc: float = 0.04,
          packets_per_line: int = 10_000_000):
    """Non-LTE molecular cloud: log-normal density (ln rho a Gaussian random
    field with P(k) ~ k^-11/3, sigma_lnrho = 1.5, mean n = 1e3 cm^-3 exactly),
    each velocity component a Gaussian random field with P(k) ~ k^-4 and a
    1-D dispersion of exactly 1 km/s, T = 20 K, emitter abundance 1e-4, a
    5-level rotor. Returns (Problem, n_mol [nz,ny,nx], LevelSpec); the
    Problem's opacity and source are placeholders that the level iteration
    replaces line by line."""
    rng = np.random.default_rng(seed)
    shape = (n, n, n)
    lnrho = sigma_lnrho * gaussian_field(shape, -11.0 / 3.0, rng)
    rho = np.exp(lnrho)
    dens = mean_n * rho / rho.mean()
    vel = np.stack([sigma_v_kms * 1e5 * gaussian_field(shape, -4.0, rng) for _ in range(3)])
    n_mol = (abundance * dens).astype(np.float32)
    pc = 3.0856775814913673e18
    spec = LevelSpec()
    p = Problem(
        name=f"cloud{n}", shape=shape, cell_cm=box_pc * pc / n, periodic=(False, False, False),
        opacity_kind="n_l", opacity=n_mol.copy(), T_K=T_K,
        line=Line(115.27e9, spec.mass_amu, spec.A1, 3.0, 1.0, spec.k_ul, 0.0),
        source=Source(SOURCE_VOLUME, profile=PROFILE_GAUSSIAN, rate=n_mol.copy()),
        vel_cms=vel.astype(np.float32), n_coll=dens.astype(np.float32),
        spectrum=(-20.0, 20.0, 80), tallies=("exc",), n_packets=packets_per_line, seed=seed)
    return p, n_mol, spec


def model_set(n_models: int = 64, total_packets: int = 10_000_000, seed: int = 4,
              sides=(32, 48, 64, 96, 128), tau_range=(1e3, 1e7), a_range=(1e-4, 1e-2),
              vmax_kms=300.0, T_K: float = 1e4):
    """Independent uniform spheres of uneven size: side drawn from `sides`,
    tau0 log-uniform, a log-uniform, v_max uniform in [-vmax, vmax];
    packets split in proportion to tau0. Returns a list of Problems."""
    rng = np.random.default_rng(seed)
    side = rng.choice(np.asarray(sides), size=n_models)
    tau = np.exp(rng.uniform(math.log(tau_range[0]), math.log(tau_range[1]), n_models))
    a = np.exp(rng.uniform(math.log(a_range[0]), math.log(a_range[1]), n_models))
    vm = rng.uniform(-vmax_kms, vmax_kms, n_models)
    share = tau / tau.sum()
    npk = np.maximum(1, np.floor(share * total_packets)).astype(np.int64)
    out = []
    for i in range(n_models):
        p = sphere(vmax_kms=float(vm[i]), tau0=float(tau[i]), a=float(a[i]), n=int(side[i]),
                   n_packets=int(npk[i]), seed=seed, T_K=T_K, tallies=())
        p.name = f"model{i}_" + p.name
        out.append(p)
    return out
