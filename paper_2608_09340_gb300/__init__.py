"""GB300 Monte Carlo line-transfer library: Python binding of libkrl.so.

Argument marshalling only. Every step of the walk runs in the CUDA kernels of
libkrl.so (built for sm_103a by :func:`paper_2608_09340_gb300.build.build`);
this module fails loudly when that library is missing. PyTorch provides
device memory and the current stream.

The C functions keep their names (``krl_grid_create``, ``krl_line_set``,
``krl_run_packets``, ``krl_tallies_get``, ...); :class:`Grid` wraps them for
the workloads in ``workloads``.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkrl.so")

KRL_OK, KRL_ERR_ARG, KRL_ERR_CUDA, KRL_ERR_OOM, KRL_ERR_BUDGET, KRL_ERR_STATE, KRL_ERR_NUMERIC = 0, -1, -2, -3, -4, -5, -6
STATUS_NAMES = {0: "KRL_OK", -1: "KRL_ERR_ARG", -2: "KRL_ERR_CUDA", -3: "KRL_ERR_OOM", -4: "KRL_ERR_BUDGET",
                -5: "KRL_ERR_STATE", -6: "KRL_ERR_NUMERIC"}
KRL_PERIODIC = (1, 2, 4)
KRL_OPACITY = {"tau": 0, "n_l": 1}
KRL_SRC = {"point": 0, "plane": 1, "beam": 2, "volume": 3}
KRL_PROFILE = {"line_centre": 0, "gaussian": 1}
KRL_TALLY = {"scatmap": 1, "exc": 2, "J": 4, "emiss": 8}
KRL_PREC_FP32, KRL_PREC_FP64 = 0, 1
KRL_MAX_CAMERAS = 8
OUT = {"spec_w": 0, "spec_n": 1, "scatmap": 2, "exc": 3, "J": 4, "emiss": 5, "stats": 6, "absw": 7,
       "voigt": 16, "us_x": 17, "us_lncdf": 18, "rtab": 19, "cells": 20, "eps": 21, "src_cdf": 22, "H0": 23,
       "voigt2d": 24}
OUT_DTYPE = {0: "float64", 1: "int64", 2: "int64", 3: "float64", 4: "float64", 5: "float32", 6: "int64", 7: "float64",
             16: "float32", 17: "float32", 18: "float32", 19: "float32", 20: "float32", 21: "float32",
             22: "float64", 23: "float32", 24: "float32"}


class KrlError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class krl_grid_desc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("cell_cm", C.c_double),
                ("boundary_flags", C.c_uint32), ("opacity_kind", C.c_int), ("opacity", C.c_void_p),
                ("T_K", C.c_double), ("vx", C.c_void_p), ("vy", C.c_void_p), ("vz", C.c_void_p),
                ("n_coll", C.c_void_p), ("tau_abs", C.c_void_p)]


class krl_line_desc(C.Structure):
    _fields_ = [("nu0_hz", C.c_double), ("mass_amu", C.c_double), ("A_ul", C.c_double),
                ("g_u", C.c_double), ("g_l", C.c_double), ("k_ul", C.c_double), ("a_fixed", C.c_double),
                ("src_kind", C.c_int), ("src_pos", C.c_double * 3), ("src_axis", C.c_int),
                ("src_plane", C.c_double), ("band_axis", C.c_int), ("band_lo", C.c_double),
                ("band_hi", C.c_double), ("src_profile", C.c_int), ("src_rate", C.c_void_p),
                ("luminosity", C.c_double), ("spec_xmin", C.c_double), ("spec_xmax", C.c_double),
                ("spec_nbins", C.c_int), ("ch_vmin_cms", C.c_double), ("ch_dv_cms", C.c_double),
                ("n_ch", C.c_int), ("n_cam", C.c_int), ("cam_theta", C.c_double * KRL_MAX_CAMERAS),
                ("cam_phi", C.c_double * KRL_MAX_CAMERAS), ("tally_flags", C.c_uint32),
                ("ph_mode", C.c_int)]


class krl_line_info(C.Structure):
    _fields_ = [("b_cms", C.c_double), ("nu_D_hz", C.c_double), ("a", C.c_double),
                ("sigma0_cm2", C.c_double), ("H0", C.c_double), ("ncell", C.c_int)]


class krl_raytrace_desc(C.Structure):
    _fields_ = [("camera", C.c_int), ("theta", C.c_double), ("phi", C.c_double), ("npix_x", C.c_int),
                ("npix_y", C.c_int), ("fov_cells", C.c_double), ("emiss", C.c_void_p), ("jline", C.c_void_p),
                ("no_scratch", C.c_int)]


KRL_MAX_LEVELS = 8


class krl_levels_desc(C.Structure):
    _fields_ = [("n_lev", C.c_int), ("E_K", C.c_double * KRL_MAX_LEVELS), ("g", C.c_double * KRL_MAX_LEVELS),
                ("A", (C.c_double * KRL_MAX_LEVELS) * KRL_MAX_LEVELS),
                ("k_coll", (C.c_double * KRL_MAX_LEVELS) * KRL_MAX_LEVELS),
                ("mass_amu", C.c_double), ("n_mol", C.c_void_p)]


def levels_desc(E_K, g, A, k_coll, mass_amu, n_mol_tensor) -> krl_levels_desc:
    """krl_levels_desc from arrays (A[u][l], k_coll[u][l] for u > l)."""
    d = krl_levels_desc()
    n = len(E_K)
    d.n_lev = n
    for i in range(n):
        d.E_K[i], d.g[i] = float(E_K[i]), float(g[i])
        for j in range(n):
            d.A[i][j], d.k_coll[i][j] = float(A[i][j]), float(k_coll[i][j])
    d.mass_amu = float(mass_amu)
    d.n_mol = n_mol_tensor.data_ptr()
    return d


KRL_TABLES_SHARED, KRL_TABLES_CONSTANT = 0, 1


class krl_tune(C.Structure):
    _fields_ = [("precision", C.c_int), ("block", C.c_int), ("ctas_per_sm", C.c_int),
                ("refill_min", C.c_int), ("max_iters", C.c_uint64), ("emiss_records", C.c_int64),
                ("table_space", C.c_int)]


class krl_run_stats(C.Structure):
    _fields_ = [("emitted", C.c_uint64), ("escaped", C.c_uint64), ("destroyed", C.c_uint64),
                ("stuck", C.c_uint64), ("scatterings", C.c_uint64), ("crossings", C.c_uint64),
                ("absorbed", C.c_uint64)]


RECORD_DTYPE = np.dtype([("x", "<f4"), ("nscat", "<u4"), ("ncross", "<u4"), ("status", "<u2"),
                         ("pad", "<u2"), ("cell0", "<u4"), ("scat_cells", "<u4")])
assert RECORD_DTYPE.itemsize == 24

EXPORTS = ["krl_last_error", "krl_version", "krl_grid_create", "krl_grid_destroy", "krl_line_set",
           "krl_line_info_get", "krl_run_packets", "krl_tallies_get", "krl_tally_bytes", "krl_tallies_reset",
           "krl_emission_cdf_noalloc", "krl_raytrace_channels", "krl_batch_create", "krl_batch_run",
           "krl_batch_destroy", "krl_levels_solve", "krl_levels_iterate"]

_lib_handle = None


def load_library(path: str | None = None):
    """Load libkrl.so (raises if it has not been built: there is no fallback)."""
    global _lib_handle
    if _lib_handle is not None and path is None:
        return _lib_handle
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"libkrl.so not found at {p}; build it with paper_2608_09340_gb300.build.build()")
    lib = C.CDLL(p)
    vp = C.c_void_p
    lib.krl_last_error.restype = C.c_char_p
    lib.krl_last_error.argtypes = []
    lib.krl_version.restype = C.c_int
    lib.krl_grid_create.argtypes = [C.POINTER(vp), C.POINTER(krl_grid_desc), vp]
    lib.krl_grid_destroy.argtypes = [vp]
    lib.krl_line_set.argtypes = [vp, C.POINTER(krl_line_desc), vp]
    lib.krl_line_info_get.argtypes = [vp, C.POINTER(krl_line_info)]
    lib.krl_run_packets.argtypes = [vp, C.c_uint64, C.c_uint64, C.c_uint64, C.POINTER(krl_tune), vp,
                                    C.POINTER(krl_run_stats), vp]
    lib.krl_tallies_get.argtypes = [vp, C.c_int, vp, C.c_size_t, vp]
    lib.krl_tally_bytes.restype = C.c_size_t
    lib.krl_tally_bytes.argtypes = [vp, C.c_int]
    lib.krl_tallies_reset.argtypes = [vp, vp]
    lib.krl_emission_cdf_noalloc.argtypes = [vp, C.c_int, vp, vp]
    lib.krl_raytrace_channels.argtypes = [vp, C.POINTER(krl_raytrace_desc), vp, vp]
    lib.krl_batch_create.argtypes = [C.POINTER(vp), C.POINTER(vp), C.c_int, vp]
    lib.krl_levels_solve.argtypes = [vp, C.POINTER(krl_levels_desc), vp, vp, C.POINTER(C.c_double), vp]
    lib.krl_levels_iterate.argtypes = [vp, C.POINTER(krl_levels_desc), C.c_int, C.c_uint64, C.c_uint64, C.c_int, vp,
                                       C.POINTER(C.c_double), vp]
    lib.krl_batch_destroy.argtypes = [vp]
    lib.krl_batch_run.argtypes = [vp, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64), C.c_uint64,
                                  C.POINTER(krl_tune), C.POINTER(vp), C.POINTER(krl_run_stats), vp]
    for name in ("krl_grid_create", "krl_grid_destroy", "krl_line_set", "krl_line_info_get",
                 "krl_run_packets", "krl_tallies_get", "krl_tallies_reset", "krl_emission_cdf_noalloc",
                 "krl_raytrace_channels", "krl_batch_create", "krl_batch_destroy", "krl_batch_run",
                 "krl_levels_solve", "krl_levels_iterate"):
        getattr(lib, name).restype = C.c_int
    if path is None:
        _lib_handle = lib
    return lib


def _check(st: int, lib=None):
    if st != KRL_OK:
        lib = lib or load_library()
        raise KrlError(st, lib.krl_last_error().decode(errors="replace"))


def _stream_handle(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


# ------------------------------------------------------------------ C-named wrappers

def krl_grid_create(desc: krl_grid_desc, stream=None):
    lib = load_library()
    h = C.c_void_p()
    _check(lib.krl_grid_create(C.byref(h), C.byref(desc), _stream_handle(stream)))
    return h


def krl_grid_destroy(handle):
    _check(load_library().krl_grid_destroy(handle))


def krl_line_set(handle, desc: krl_line_desc, stream=None):
    _check(load_library().krl_line_set(handle, C.byref(desc), _stream_handle(stream)))


def krl_line_info_get(handle) -> krl_line_info:
    info = krl_line_info()
    _check(load_library().krl_line_info_get(handle, C.byref(info)))
    return info


def krl_run_packets(handle, n: int, first_id: int, seed: int, tune: krl_tune | None = None,
                    records=None, want_stats: bool = False, stream=None):
    lib = load_library()
    st = krl_run_stats() if want_stats else None
    rc = lib.krl_run_packets(handle, int(n), int(first_id), int(seed) & ((1 << 64) - 1),
                             C.byref(tune) if tune is not None else None, _ptr(records),
                             C.byref(st) if st is not None else None, _stream_handle(stream))
    if rc == KRL_ERR_BUDGET and st is not None:
        return st, rc
    _check(rc)
    return st, rc


def krl_tally_bytes(handle, kind: int) -> int:
    return int(load_library().krl_tally_bytes(handle, int(kind)))


def krl_tallies_get(handle, kind: int, dst, stream=None):
    nbytes = dst.numel() * dst.element_size()
    _check(load_library().krl_tallies_get(handle, int(kind), _ptr(dst), nbytes, _stream_handle(stream)))


def krl_tallies_reset(handle, stream=None):
    _check(load_library().krl_tallies_reset(handle, _stream_handle(stream)))


def krl_raytrace_channels(handle, desc: krl_raytrace_desc, maps, stream=None):
    _check(load_library().krl_raytrace_channels(handle, C.byref(desc), _ptr(maps), _stream_handle(stream)))


def krl_emission_cdf_noalloc(rate, cdf, stream=None):
    """Emission CDF of a float32 rate tensor into a float64 cdf tensor (both on
    the device), with no device allocation: for callers that cannot call
    cudaMalloc (see include/krl.h). Overlapping calls race; the first call on
    a device should come before any stream capture."""
    _check(load_library().krl_emission_cdf_noalloc(_ptr(rate), int(rate.numel()), _ptr(cdf),
                                                   _stream_handle(stream)))


# ------------------------------------------------------------------ workload marshalling

class Grid:
    """A krl_grid with its line, built from a ``workloads.Problem``."""

    def __init__(self, problem, device="cuda", stream=None):
        import torch
        self.problem = problem
        self.device = torch.device(device)
        self._keep = []
        nz, ny, nx = problem.shape

        def dev(a):
            if a is None:
                return None
            if isinstance(a, torch.Tensor):     # e.g. pinned host memory: async copy
                t = a.to(device=self.device, dtype=torch.float32, non_blocking=True).contiguous()
            else:
                t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(self.device)
            self._keep.append(t)
            return t

        op = dev(problem.opacity)
        vel = [None, None, None]
        if problem.vel_cms is not None:
            vel = [dev(problem.vel_cms[k]) for k in range(3)]
        nco = dev(problem.n_coll)
        tab = dev(getattr(problem, "tau_abs", None))
        d = krl_grid_desc()
        d.nx, d.ny, d.nz = nx, ny, nz
        d.cell_cm = problem.cell_cm
        d.boundary_flags = sum(b for b, p in zip(KRL_PERIODIC, problem.periodic) if p)
        d.opacity_kind = KRL_OPACITY[problem.opacity_kind]
        d.opacity = op.data_ptr()
        d.T_K = problem.T_K
        d.vx, d.vy, d.vz = [v.data_ptr() if v is not None else None for v in vel]
        d.n_coll = nco.data_ptr() if nco is not None else None
        d.tau_abs = tab.data_ptr() if tab is not None else None
        self.handle = krl_grid_create(d, stream)
        try:
            ln, src = problem.line, problem.source
            L = krl_line_desc()
            L.nu0_hz, L.mass_amu, L.A_ul = ln.nu0_hz, ln.mass_amu, ln.A_ul
            L.g_u, L.g_l, L.k_ul, L.a_fixed = ln.g_u, ln.g_l, ln.k_ul, ln.a_fixed
            L.ph_mode = int(getattr(ln, "ph_mode", 2))
            L.src_kind = KRL_SRC[src.kind]
            L.src_pos = (C.c_double * 3)(*src.pos)
            L.src_axis, L.src_plane = src.axis, src.plane
            L.band_axis, L.band_lo, L.band_hi = src.band_axis, src.band[0], src.band[1]
            L.src_profile = KRL_PROFILE[src.profile]
            rate = dev(src.rate) if src.kind == "volume" else None
            L.src_rate = rate.data_ptr() if rate is not None else None
            L.luminosity = src.luminosity
            L.spec_xmin, L.spec_xmax, L.spec_nbins = problem.spectrum
            if problem.channels is not None:
                L.ch_vmin_cms, L.ch_dv_cms, L.n_ch = problem.channels
            L.n_cam = len(problem.cameras)
            for i, (t, p) in enumerate(problem.cameras):
                L.cam_theta[i], L.cam_phi[i] = t, p
            L.tally_flags = sum(KRL_TALLY[t] for t in problem.tallies)
            krl_line_set(self.handle, L, stream)
            self.info = krl_line_info_get(self.handle)
        except Exception:
            krl_grid_destroy(self.handle)
            self.handle = None
            raise

    def close(self):
        if getattr(self, "handle", None) is not None:
            krl_grid_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, n: int | None = None, first: int = 0, seed: int | None = None, precision: int = KRL_PREC_FP32,
            records: bool = False, block: int = 0, ctas_per_sm: int = 0, refill_min: int = 0,
            max_iters: int = 0, want_stats: bool = True, stream=None, emiss_records: int = 0,
            table_space: int = KRL_TABLES_SHARED):
        """Run packets [first, first+n); returns (stats, status code, records
        tensor or None). emiss_records, table_space: krl_tune's fields."""
        import torch
        n = self.problem.n_packets if n is None else int(n)
        seed = self.problem.seed if seed is None else int(seed)
        tune = krl_tune(precision, block, ctas_per_sm, refill_min, max_iters, emiss_records, table_space)
        rec = None
        if records:
            rec = torch.empty(n * RECORD_DTYPE.itemsize, dtype=torch.uint8, device=self.device)
        st, rc = krl_run_packets(self.handle, n, first, seed, tune, rec, want_stats, stream)
        return st, rc, rec

    def tally(self, name: str, stream=None):
        import torch
        kind = OUT[name]
        nbytes = krl_tally_bytes(self.handle, kind)
        if nbytes == 0:
            return None
        dt = getattr(torch, OUT_DTYPE[kind])
        out = torch.empty(nbytes // torch.tensor([], dtype=dt).element_size(), dtype=dt, device=self.device)
        krl_tallies_get(self.handle, kind, out, stream)
        return out

    def reset(self, stream=None):
        krl_tallies_reset(self.handle, stream)

    def levels_solve(self, desc: krl_levels_desc, gamma, pops, stream=None):
        ch = C.c_double(0.0)
        _check(load_library().krl_levels_solve(self.handle, C.byref(desc), _ptr(gamma), _ptr(pops), C.byref(ch),
                                               _stream_handle(stream)))
        return ch.value

    def levels_iterate(self, desc: krl_levels_desc, n_iter: int, packets_per_line: int, seed: int, pops,
                       init_lte: bool = True, stream=None):
        """Lambda iteration; returns the per-cycle population change."""
        ch = (C.c_double * max(1, n_iter))()
        _check(load_library().krl_levels_iterate(self.handle, C.byref(desc), int(n_iter), int(packets_per_line),
                                                 int(seed), int(bool(init_lte)), _ptr(pops), ch,
                                                 _stream_handle(stream)))
        return list(ch)[:n_iter]

    def raytrace(self, camera: int, npix_x: int, npix_y: int, fov_cells: float, emiss=None, jline=None,
                 theta: float = 0.0, phi: float = 0.0, no_scratch: bool = False, stream=None):
        """Channel maps [n_ch, npix_y, npix_x] (float32 tensor) for one camera."""
        import torch
        nch = self.problem.channels[2]
        maps = torch.empty((nch, npix_y, npix_x), dtype=torch.float32, device=self.device)
        d = krl_raytrace_desc(camera, theta, phi, npix_x, npix_y, fov_cells,
                              emiss.data_ptr() if emiss is not None else None,
                              jline.data_ptr() if jline is not None else None, int(bool(no_scratch)))
        krl_raytrace_channels(self.handle, d, maps, stream)
        return maps


class Batch:
    """krl_batch over several Grids: all models in one persistent launch."""

    def __init__(self, grids, stream=None):
        lib = load_library()
        self.grids = list(grids)
        arr = (C.c_void_p * len(self.grids))(*[g.handle.value for g in self.grids])
        h = C.c_void_p()
        _check(lib.krl_batch_create(C.byref(h), arr, len(self.grids), _stream_handle(stream)))
        self.handle = h

    def run(self, packets, first_ids=None, seed: int = 0, precision: int = KRL_PREC_FP32, block: int = 0,
            ctas_per_sm: int = 0, refill_min: int = 0, max_iters: int = 0, want_stats: bool = False, stream=None,
            records=None):
        """records: None, or one device tensor (or None) per model that
        receives that model's packet records (RECORD_DTYPE, one per packet)."""
        n = len(self.grids)
        pk = (C.c_uint64 * n)(*[int(v) for v in packets])
        fi = (C.c_uint64 * n)(*[int(v) for v in first_ids]) if first_ids is not None else None
        tune = krl_tune(precision, block, ctas_per_sm, refill_min, max_iters)
        st = (krl_run_stats * n)() if want_stats else None
        rp = None
        if records is not None:
            for r, k in zip(records, packets):
                if r is not None and r.numel() * r.element_size() < int(k) * RECORD_DTYPE.itemsize:
                    raise ValueError("record buffer smaller than the model's packet count")
            rp = (C.c_void_p * n)(*[None if r is None else r.data_ptr() for r in records])
        rc = load_library().krl_batch_run(self.handle, pk, fi, int(seed) & ((1 << 64) - 1), C.byref(tune),
                                          rp, st, _stream_handle(stream))
        if not (rc == KRL_ERR_BUDGET and st is not None):
            _check(rc)
        return (list(st) if st is not None else None), rc

    def close(self):
        if getattr(self, "handle", None) is not None:
            _check(load_library().krl_batch_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def records_to_numpy(rec_tensor) -> np.ndarray:
    return rec_tensor.cpu().numpy().view(RECORD_DTYPE)
