"""FP64 CPU oracle of the Monte Carlo line-transfer pass.

TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg may import this package; the product path never does and
shares no code with it.

* ``oracle.tables``     - line physics and sampling tables (numpy/scipy, FP64).
* ``oracle/transport.c`` - the packet walk (plain C, FP64, pthreads), built
  into ``oracle/_liborc.so`` by :func:`build`.
* ``oracle.run``        - derive the per-cell inputs from a workload Problem
  and run packets through the C walk.
* ``oracle.raytrace``   - FP64 formal solution for channel maps.
* ``oracle.levels``     - FP64 statistical-equilibrium solves and the Lambda
  iteration's excitation rates.
* ``oracle.exact``      - O-exact: the static-slab walk with no tables (the
  Voigt function evaluated directly, exact velocity draws), to measure the
  tabulated method's table error.
"""
from __future__ import annotations

import ctypes as C
import functools
import math
import os
import subprocess

import numpy as np

from . import tables as T

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "transport.c")
_LIB = os.path.join(_HERE, "_liborc.so")

TALLY_BITS = {"scatmap": 1, "exc": 2, "J": 4, "emiss": 8}
SRC_KIND = {"point": 0, "plane": 1, "beam": 2, "volume": 3}
PROFILE = {"line_centre": 0, "gaussian": 1}
ESCAPED, DESTROYED, STUCK, ABSORBED = 1, 2, 3, 4
# A packet whose weight falls below this (after continuum absorption) ends
# as absorbed (reading: the paper does not say how weights are cut off).
WEIGHT_CUT = 1e-12


def build(force: bool = False) -> str:
    """Compile the C walk with gcc (no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", "-pthread", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Problem(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("periodic", C.c_int * 3),
        ("tau0", C.POINTER(C.c_double)), ("vel", C.POINTER(C.c_double)),
        ("eps", C.POINTER(C.c_double)), ("a", C.c_double),
        ("voigt_lnH", C.POINTER(C.c_double)), ("voigt_H0", C.c_double),
        ("us_x", C.POINTER(C.c_double)), ("us_lncdf", C.POINTER(C.c_double)),
        ("rtab", C.POINTER(C.c_double)),
        ("src_kind", C.c_int), ("src_pos", C.c_double * 3), ("src_axis", C.c_int),
        ("src_plane", C.c_double), ("band_axis", C.c_int),
        ("band_lo", C.c_double), ("band_hi", C.c_double),
        ("src_profile", C.c_int), ("src_cdf", C.POINTER(C.c_double)),
        ("spec_lo", C.c_double), ("spec_hi", C.c_double), ("spec_n", C.c_int),
        ("n_ch", C.c_int), ("ch_x0", C.c_double), ("ch_dx", C.c_double),
        ("n_cam", C.c_int), ("cam_dir", C.POINTER(C.c_double)),
        ("tally_flags", C.c_uint), ("max_iters", C.c_uint64),
        ("ph_mode", C.c_int), ("voigt2d", C.POINTER(C.c_double)), ("u0", C.c_double),
        ("tau_abs", C.POINTER(C.c_double)), ("wcut", C.c_double),
    ]


RECORD_DTYPE = np.dtype([("x", "<f8"), ("nscat", "<u4"), ("ncross", "<u4"),
                         ("status", "<u4"), ("cell0", "<u4")])


class _Tallies(C.Structure):
    _fields_ = [
        ("spec_w", C.POINTER(C.c_double)), ("spec_c", C.POINTER(C.c_uint64)),
        ("scat", C.POINTER(C.c_uint64)), ("exc", C.POINTER(C.c_double)),
        ("J", C.POINTER(C.c_double)), ("emiss", C.POINTER(C.c_double)),
        ("absw", C.POINTER(C.c_double)),
        ("stats", C.c_uint64 * 8), ("rec", C.c_void_p),
    ]


@functools.lru_cache(maxsize=1)
def _lib():
    lib = C.CDLL(build())
    lib.orc_run.restype = C.c_int
    lib.orc_run.argtypes = [C.POINTER(_Problem), C.c_uint64, C.c_uint64, C.c_uint32,
                            C.c_uint32, C.c_int, C.POINTER(_Tallies)]
    lib.orc_trace.restype = C.c_int
    lib.orc_trace.argtypes = [C.POINTER(_Problem), C.POINTER(C.c_double), C.POINTER(C.c_double),
                              C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_double)]
    lib.orc_philox.restype = None
    lib.orc_philox.argtypes = [C.POINTER(C.c_uint32), C.c_uint32, C.c_uint32,
                               C.POINTER(C.c_uint32), C.c_int]
    for name in ("orc_us_sample", "orc_voigt"):
        f = getattr(lib, name)
        f.restype = C.c_double
        f.argtypes = [C.POINTER(_Problem), C.c_double] + ([C.c_double] if name == "orc_us_sample" else [])
    lib.orc_rkernel.restype = C.c_double
    lib.orc_rkernel.argtypes = [C.POINTER(_Problem), C.c_double, C.c_double, C.c_double]
    return lib


@functools.lru_cache(maxsize=1)
def voigt2d_f64():
    """The ph_mode 1 table (float32 values) as a contiguous FP64 array."""
    return np.ascontiguousarray(T.voigt2d_table(), dtype=np.float64)


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


@functools.lru_cache(maxsize=8)
def line_tables(a: float, with_r: bool = True):
    """All float32 tables for damping parameter a, as FP64 arrays."""
    lnH, H0 = T.voigt_table(a)
    xs, lnc = T.usampler_table(a)
    rt = T.rtable(a) if with_r else None
    f64 = lambda v: None if v is None else np.ascontiguousarray(v, dtype=np.float64)
    return {"voigt_lnH": f64(lnH), "voigt_H0": float(H0), "us_x": f64(xs),
            "us_lncdf": f64(lnc), "rtab": f64(rt)}


def derive(problem):
    """Per-cell inputs of the walk from a workload Problem (FP64 arithmetic,
    fields rounded to float32 as the method stores them):
    b (Sec. 2.1), a, line-centre optical depth per cell width (Eq. sigma0
    when the opacity is given as n_l), bulk velocity in units of b,
    destruction probability (Eq. eps), emission CDF over cells."""
    ln = problem.line
    b = T.doppler_b(problem.T_K, ln.mass_amu)
    a = ln.a_fixed if ln.a_fixed > 0 else T.damping_a(ln.A_ul, ln.nu0_hz, b)
    op = np.asarray(problem.opacity, dtype=np.float64).reshape(-1)
    if problem.opacity_kind == "tau":
        tau0 = op.astype(np.float32).astype(np.float64)
    else:
        s0 = T.sigma0(ln.g_u, ln.g_l, ln.A_ul, ln.nu0_hz, b)
        tau0 = (op * s0 * problem.cell_cm).astype(np.float32).astype(np.float64)
    vel = None
    if problem.vel_cms is not None:
        v = np.asarray(problem.vel_cms, dtype=np.float64).reshape(3, -1).T / b
        vel = np.ascontiguousarray(v.astype(np.float32).astype(np.float64))
    eps = None
    if ln.k_ul > 0 and problem.n_coll is not None:
        e = T.epsilon(ln.k_ul, np.asarray(problem.n_coll, dtype=np.float64).reshape(-1), ln.A_ul)
        eps = e.astype(np.float32).astype(np.float64)
    tau_abs = None
    if getattr(problem, "tau_abs", None) is not None:
        tau_abs = np.asarray(problem.tau_abs, dtype=np.float32).astype(np.float64).reshape(-1)
    cdf = None
    if problem.source.kind == "volume":
        r = np.asarray(problem.source.rate, dtype=np.float32).astype(np.float64).reshape(-1)
        cs = np.cumsum(r)
        cdf = cs / cs[-1]
    cams = None
    if problem.cameras:
        cams = np.array([[math.sin(t) * math.cos(p), math.sin(t) * math.sin(p), math.cos(t)]
                         for t, p in problem.cameras], dtype=np.float64)
    return {"b": b, "a": a, "tau0": tau0, "vel": vel, "eps": eps, "cdf": cdf, "cam": cams, "tau_abs": tau_abs}


def run(problem, n: int | None = None, first: int = 0, seed: int | None = None,
        nthreads: int | None = None, records: bool = False, max_iters: int = (1 << 32) - 1,
        tables: dict | None = None):
    """Run packets [first, first+n) of `problem` through the FP64 walk.

    max_iters: per-packet event budget; the default is the library's
    (2^32 - 1, the largest the CUDA walk accepts), so both stop a packet at
    the same event.

    Returns a dict: spec_w, spec_c (under, bins, over), scat, exc, J, emiss
    (raw sums with unit packet weight, lengths in cell widths), absw (weight
    absorbed by the continuum per cell, when the problem has tau_abs), stats
    (emitted, escaped, destroyed, stuck, scatterings, crossings, absorbed),
    records, and the derived b, a."""
    n = problem.n_packets if n is None else int(n)
    seed = problem.seed if seed is None else int(seed)
    d = derive(problem)
    need_r = "emiss" in problem.tallies
    tb = tables if tables is not None else line_tables(float(d["a"]), need_r)
    nz, ny, nx = problem.shape
    ncell = nx * ny * nz
    flags = 0
    for t in problem.tallies:
        flags |= TALLY_BITS[t]
    src = problem.source
    P = _Problem()
    P.nx, P.ny, P.nz = nx, ny, nz
    P.periodic = (C.c_int * 3)(*[int(bool(v)) for v in problem.periodic])
    keep = [d["tau0"], d["vel"], d["eps"], d["cdf"], d["cam"], tb["voigt_lnH"], tb["us_x"],
            tb["us_lncdf"], tb["rtab"]]
    P.tau0, P.vel, P.eps = _dp(d["tau0"]), _dp(d["vel"]), _dp(d["eps"])
    P.a = d["a"]
    P.voigt_lnH, P.voigt_H0 = _dp(tb["voigt_lnH"]), tb["voigt_H0"]
    P.us_x, P.us_lncdf, P.rtab = _dp(tb["us_x"]), _dp(tb["us_lncdf"]), _dp(tb["rtab"])
    P.src_kind = SRC_KIND[src.kind]
    P.src_pos = (C.c_double * 3)(*src.pos)
    P.src_axis, P.src_plane = src.axis, src.plane
    P.band_axis, P.band_lo, P.band_hi = src.band_axis, src.band[0], src.band[1]
    P.src_profile = PROFILE[src.profile]
    P.src_cdf = _dp(d["cdf"])
    P.spec_lo, P.spec_hi, P.spec_n = problem.spectrum[0], problem.spectrum[1], problem.spectrum[2]
    nch = 0
    if problem.channels is not None:
        vmin, dv, nch = problem.channels
        P.ch_x0, P.ch_dx = vmin / d["b"], dv / d["b"]
    P.n_ch = nch
    P.n_cam = len(problem.cameras)
    P.cam_dir = _dp(d["cam"])
    P.tally_flags = flags
    P.max_iters = max_iters
    ph = int(getattr(problem.line, "ph_mode", 2) or 2)
    P.ph_mode = ph
    if ph == 1:
        T.voigt2d_weights(float(d["a"]))          # range check
        v2 = voigt2d_f64()
        keep.append(v2)
        P.voigt2d = _dp(v2)
    elif ph == 3:
        P.u0 = T.blend_u0(float(d["a"]))
    if d["tau_abs"] is not None:
        keep.append(d["tau_abs"])
        P.tau_abs = _dp(d["tau_abs"])
    P.wcut = WEIGHT_CUT
    ncam = max(1, len(problem.cameras))
    out = {
        "spec_w": np.zeros(problem.spectrum[2] + 2), "spec_c": np.zeros(problem.spectrum[2] + 2, np.uint64),
        "scat": np.zeros(ncell, np.uint64) if flags & 1 else None,
        "exc": np.zeros(ncell) if flags & 2 else None,
        "J": np.zeros(ncell * max(nch, 1)) if flags & 4 else None,
        "emiss": np.zeros(ncam * ncell * max(nch, 1)) if flags & 8 else None,
        "records": np.zeros(n, RECORD_DTYPE) if records else None,
        "absw": np.zeros(ncell) if d["tau_abs"] is not None else None,
    }
    Tl = _Tallies()
    Tl.spec_w = _dp(out["spec_w"])
    Tl.spec_c = out["spec_c"].ctypes.data_as(C.POINTER(C.c_uint64))
    Tl.scat = out["scat"].ctypes.data_as(C.POINTER(C.c_uint64)) if out["scat"] is not None else None
    Tl.exc, Tl.J, Tl.emiss = _dp(out["exc"]), _dp(out["J"]), _dp(out["emiss"])
    Tl.absw = _dp(out["absw"])
    Tl.rec = out["records"].ctypes.data if records else None
    nthreads = nthreads or os.cpu_count() or 1
    rc = _lib().orc_run(C.byref(P), first, n, seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF,
                        nthreads, C.byref(Tl))
    del keep
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    out["stats"] = np.array(list(Tl.stats), dtype=np.uint64)
    if out["J"] is not None:
        out["J"] = out["J"].reshape(ncell, nch)
    if out["emiss"] is not None:
        out["emiss"] = out["emiss"].reshape(ncam, ncell, nch)
    out["b"], out["a"] = d["b"], d["a"]
    out["nthreads"] = nthreads
    return out


def _problem_for_lookups(a: float, tb: dict):
    P = _Problem()
    P.a = a
    P.voigt_lnH, P.voigt_H0 = _dp(tb["voigt_lnH"]), tb["voigt_H0"]
    P.us_x, P.us_lncdf, P.rtab = _dp(tb["us_x"]), _dp(tb["us_lncdf"]), _dp(tb["rtab"])
    return P


def c_lookups(a: float, ph_mode: int = 2):
    """The C walk's own sampler, profile and kernel lookups, for the tests."""
    tb = line_tables(a, True)
    P = _problem_for_lookups(a, tb)
    P.ph_mode = ph_mode
    v2 = None
    if ph_mode == 1:
        v2 = voigt2d_f64()
        P.voigt2d = _dp(v2)
    elif ph_mode == 3:
        P.u0 = T.blend_u0(a)
    lib = _lib()

    class L:
        keep = (tb, P, v2)

        @staticmethod
        def us_sample(x, xi):
            return lib.orc_us_sample(C.byref(P), x, xi)

        @staticmethod
        def voigt(x):
            return lib.orc_voigt(C.byref(P), x)

        @staticmethod
        def rkernel(D, x, g):
            return lib.orc_rkernel(C.byref(P), D, x, g)
    return L


def philox(ctr: np.ndarray, seed: int) -> np.ndarray:
    """Raw Philox4x32-10 words for counters ctr[n, 4] (uint32) under key=seed."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32)
    out = np.zeros_like(ctr)
    _lib().orc_philox(ctr.ctypes.data_as(C.POINTER(C.c_uint32)), seed & 0xFFFFFFFF,
                      (seed >> 32) & 0xFFFFFFFF, out.ctypes.data_as(C.POINTER(C.c_uint32)),
                      ctr.shape[0])
    return out


def trace(shape, periodic, X, n, max_seg: int = 100000):
    """Cell walk of one ray through an opacity-free grid (geometry only)."""
    nz, ny, nx = shape
    P = _Problem()
    P.nx, P.ny, P.nz = nx, ny, nz
    P.periodic = (C.c_int * 3)(*[int(bool(v)) for v in periodic])
    Xa = np.ascontiguousarray(X, dtype=np.float64)
    na = np.ascontiguousarray(n, dtype=np.float64)
    cells = np.zeros(max_seg, np.int64)
    lens = np.zeros(max_seg)
    k = _lib().orc_trace(C.byref(P), _dp(Xa), _dp(na), max_seg,
                         cells.ctypes.data_as(C.POINTER(C.c_int64)), _dp(lens))
    return cells[:k], lens[:k]
