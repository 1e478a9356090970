"""Throughput of the Monte Carlo line-transfer pass on the 64^3, tau0 = 1e6
uniform sphere (T = 1e4 K, a = 4.7e-4, central point source at line centre,
FP32 walk, 400-bin escaped spectrum and per-cell scattering map).

One step = one krl_run_packets launch over a whole 1e6-packet job (the next
1e6 packet ids; every part of the pass runs: emission, cell walk, scattering,
tallies, escape, regeneration, counter reduction). Inputs are resident on
the device; L2 is flushed (a 256 MiB write) before every timed step. Steps
rotate over --streams streams (default 2) so that one job's tail (its last,
longest packets) overlaps the next job's start (--serial: one stream); the
K steps are bracketed by CUDA events, and every launch also by its own pair
on its stream.

Prints one JSON line (rank 0). `--impl reference` times the FP64 CPU oracle
on the host cores on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

JOB_PACKETS = 1_000_000
PACKETS_PER_STEP = JOB_PACKETS
E2E_MAX_STEPS = 3
METRIC = "scatterings/s & packets/s (64³ τ0=1e6 sphere)"
UNIT = "scatterings/s"
# Lane operations per event. The roofline counts the arithmetic operations
# (integer, FP32, conversion and bit-manipulation instruction classes) that
# the walk executes per scattering and per face crossing, from the ncu
# instruction mix of the committed profile (two workloads with different
# crossing fractions, solved for the two event kinds), used only when that
# profile was taken on the current kernel source. Beside it: the per-unit
# work estimate of the pass (a scattering = 2 Philox4x32-10 blocks, ~120
# integer ops, + ~8 special-function ops + ~14 sampler steps + ~100 FP32 ops
# = 242; a crossing = one Voigt lookup + ~30 FP32 ops = 32), and the issue
# ceiling from all executed thread instructions per event.
OPS_PER_SCAT = 242
OPS_PER_CROSS = 32
FP32_LANES_PER_SM = 128
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "transport_sphere64_tau1e4.txt")
KERNEL_SRC = [os.path.join(ROOT, "paper_2608_09340_gb300", "csrc", f)
              for f in ("transport_impl.cuh", "transport.cu", "krl_internal.cuh")]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="krl", choices=["krl", "reference"])
    ap.add_argument("--packets", type=int, default=None,
                    help=f"packets per step (default {PACKETS_PER_STEP}; 2^21 for --profile-case)")
    ap.add_argument("--tau0", type=float, default=None,
                    help="centre-to-edge line-centre depth (default 1e6, the benchmark; 3e4 for --profile-case)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-raytrace", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--batch-full-range", action="store_true",
                    help="also time the many-model set over its full tau0 range [1e3, 1e7] (2e5 packets; "
                         "several minutes), batched against one launch per model")
    ap.add_argument("--no-next", action="store_true", help="skip the levels / profile-mode / dusty-slab legs")
    ap.add_argument("--streams", type=int, default=2,
                    help="streams the steps rotate over (1: no overlap of one step's tail with the next)")
    ap.add_argument("--serial", dest="streams", action="store_const", const=1,
                    help="same as --streams 1")
    ap.add_argument("--no-serial-leg", action="store_true",
                    help="skip the one-stream job timed after the main leg")
    # small fixed cases of one kernel for profiler captures (no bench line)
    ap.add_argument("--profile-case", choices=["transport", "raytrace", "emissivity"], default=None,
                    help="run one small case of a kernel (a warm-up launch, then --launches timed "
                         "launches) and print its CUDA-event time per launch instead of the bench line")
    ap.add_argument("--vmax", type=float, default=0.0, help="profile case: sphere v_max [km/s]")
    ap.add_argument("--grid", type=int, default=128, help="profile case: envelope grid side")
    ap.add_argument("--pixels", type=int, default=512, help="profile case: image side in pixels")
    ap.add_argument("--channels", type=int, default=64, help="profile case: velocity channels")
    ap.add_argument("--launches", type=int, default=1, help="profile case: timed launches")
    ap.add_argument("--table-space", choices=["shared", "constant"], default="shared",
                    help="profile case transport: where the walk reads the slice and the sampler")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


PROFILE_KEYS = ("dram_bytes_per_launch_scaled", "thread_instructions_per_event", "thread_instructions_per_scattering",
                "thread_instructions_per_crossing", "arith_ops_per_scattering", "arith_ops_per_crossing")


def profile_values():
    """The numeric figures of the committed ncu summary (PROFILE_KEYS present
    in it), if it was taken on the current kernel source; else {}."""
    try:
        txt = open(PROFILE_SUMMARY).read()
        src_hash = hashlib.sha256(b"".join(open(f, "rb").read() for f in KERNEL_SRC)).hexdigest()[:16]
        vals = dict(l.split(":", 1) for l in txt.splitlines() if ":" in l and not l.startswith(" "))
        if vals.get("kernel_source_sha256_16", "").strip() != src_hash:
            return {}
        return {k: float(vals[k].strip()) for k in PROFILE_KEYS if k in vals}
    except Exception:
        return {}


def profile_figures():
    """(DRAM bytes per launch, thread instructions per event) recorded by the
    committed ncu summary, if it was taken on the current kernel source
    (else None for both)."""
    v = profile_values()
    return v.get("dram_bytes_per_launch_scaled"), v.get("thread_instructions_per_event")


def traffic_from_profile():
    return profile_figures()[0]


RT_GRID = 256
RT_CHANNELS = 64
RT_PIXELS = 1024
RT_CAMERAS = 3
RT_PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "raytrace_envelope128_64ch.txt")
RT_KERNEL_SRC = [os.path.join(ROOT, "paper_2608_09340_gb300", "csrc", f) for f in ("raytrace.cu", "krl_internal.cuh")]
# Arithmetic of one channel-segment of the formal solution (Eq. imaging-
# formal): dtau = alpha dl, e = exp(-dtau), f = (1 - e)/dtau (2), the
# increment T j dl f (3), I += it, tau += dtau, T = exp(-tau): 10 ops.
RT_OPS_PER_CHANNEL_SEGMENT = 10


def ray_cells(shape, theta, phi, npix_x, npix_y, fov):
    """Number of cells each orthographic, pixel-centred ray of a camera at
    (theta, phi) crosses in a box of shape (nz, ny, nx) (the image centred on
    the box, fov cells wide): 1 + the face crossings between its entry and
    exit points. Returns the total over all pixels (a count of the
    segments the trace marches, for throughput figures)."""
    import numpy as np
    nz, ny, nx = shape
    n = np.array([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)])
    u = np.array([np.cos(theta) * np.cos(phi), np.cos(theta) * np.sin(phi), -np.sin(theta)])
    v = np.array([-np.sin(phi), np.cos(phi), 0.0])
    pix = fov / npix_x
    ix = (np.arange(npix_x) + 0.5) * pix - 0.5 * pix * npix_x
    iy = (np.arange(npix_y) + 0.5) * pix - 0.5 * pix * npix_y
    uc, vc = np.meshgrid(ix, iy)
    hi = np.array([nx, ny, nz], dtype=np.float64)
    P = hi / 2.0 + uc[..., None] * u + vc[..., None] * v
    t0 = np.full(uc.shape, -np.inf)
    t1 = np.full(uc.shape, np.inf)
    inside = np.ones(uc.shape, dtype=bool)
    for d in range(3):
        if n[d] != 0.0:
            a, b = (0.0 - P[..., d]) / n[d], (hi[d] - P[..., d]) / n[d]
            t0 = np.maximum(t0, np.minimum(a, b))
            t1 = np.minimum(t1, np.maximum(a, b))
        else:
            inside &= (P[..., d] >= 0.0) & (P[..., d] < hi[d])
    hit = inside & (t1 > t0)
    eps = 1e-9
    cells = np.ones(uc.shape)
    for d in range(3):
        x0 = np.clip(P[..., d] + (t0 + eps) * n[d], 0.0, hi[d] - 1e-9)
        x1 = np.clip(P[..., d] + (t1 - eps) * n[d], 0.0, hi[d] - 1e-9)
        cells += np.abs(np.floor(x1) - np.floor(x0))
    return float(cells[hit].sum())


def rt_profile_values():
    """Thread instructions per channel-segment of the trace from the committed
    ray-trace profile, if it was taken on the current source; else {}."""
    try:
        txt = open(RT_PROFILE_SUMMARY).read()
        src_hash = hashlib.sha256(b"".join(open(f, "rb").read() for f in RT_KERNEL_SRC)).hexdigest()[:16]
        vals = dict(l.split(":", 1) for l in txt.splitlines() if ":" in l and not l.startswith(" "))
        if vals.get("kernel_source_sha256_16", "").split()[0].strip() != src_hash:
            return {}
        return {k: float(vals[k].strip()) for k in ("thread_instructions_per_channel_segment",) if k in vals}
    except Exception:
        return {}


def bench_raytrace(args, dev):
    """Channel maps of the envelope imaging workload: a 256^3 rotating, infalling
    envelope with 64 velocity channels over +-5 km/s, imaged at 1024^2 pixels
    from 3 inclinations (0, 45, 90 deg). The emissivity cube (3 x 256^3 x 64
    FP32) is filled first by the configuration's Monte Carlo pass of 1e8
    packets (100 runs of 1e6, each with its own segment buffer, accumulating
    into the cube); one pass = the three cameras' ray traces, timed with
    CUDA events."""
    import torch
    import paper_2608_09340_gb300 as krl
    import workloads as W
    fill_runs, per_run = 100, 1_000_000
    p = W.envelope(n=RT_GRID, n_ch=RT_CHANNELS, n_packets=per_run)
    g = krl.Grid(p, device=dev)
    try:
        # the Monte Carlo fill of the emissivity cube (rich walk: excitation, J,
        # camera-directed emissivity through the R_IIA table, destruction)
        g.run(n=100_000, first=1 << 40, want_stats=False)           # warm-up
        g.reset()
        torch.cuda.synchronize(dev)
        f0 = time.perf_counter()
        for r in range(fill_runs):
            g.run(n=per_run, first=r * per_run, want_stats=False)
        torch.cuda.synchronize(dev)
        fill_s = time.perf_counter() - f0
        fst_t = g.tally("stats").cpu().numpy()

        class _St:
            scatterings, crossings = int(fst_t[4]), int(fst_t[5])
        fst = _St()
        for _ in range(max(1, args.warmup)):
            for m in range(RT_CAMERAS):
                g.raytrace(m, RT_PIXELS, RT_PIXELS, fov_cells=float(RT_GRID))
        torch.cuda.synchronize(dev)
        stream = torch.cuda.current_stream(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = max(1, args.steps)
        e0.record(stream)
        for _ in range(reps):
            for m in range(RT_CAMERAS):
                g.raytrace(m, RT_PIXELS, RT_PIXELS, fov_cells=float(RT_GRID))
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / reps
    finally:
        g.close()
    rays = RT_CAMERAS * RT_PIXELS * RT_PIXELS
    cube = RT_CAMERAS * RT_GRID ** 3 * RT_CHANNELS * 4
    segs = sum(ray_cells(p.shape, th, ph, RT_PIXELS, RT_PIXELS, float(RT_GRID)) for th, ph in p.cameras)
    chseg_per_s = segs * RT_CHANNELS / ms * 1e3
    props = torch.cuda.get_device_properties(dev)
    peaks, peak_kind = measured_peaks()
    peak_ops = props.multi_processor_count * FP32_LANES_PER_SM * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    rtp = rt_profile_values()
    rt_roof = {"bound": "alu", "ops_per_channel_segment": RT_OPS_PER_CHANNEL_SEGMENT,
               "achieved": RT_OPS_PER_CHANNEL_SEGMENT * chseg_per_s / 1e12, "peak": peak_ops / 1e12,
               "unit": "Tops/s", "frac": RT_OPS_PER_CHANNEL_SEGMENT * chseg_per_s / peak_ops,
               "issue_ceiling_frac": (rtp["thread_instructions_per_channel_segment"] * chseg_per_s / peak_ops
                                      if rtp else None),
               "thread_instructions_per_channel_segment": rtp.get("thread_instructions_per_channel_segment"),
               "peak_source": f"{peak_kind} max SM clock"}
    return {"workload": f"envelope {RT_GRID}^3, {RT_CHANNELS} ch, {RT_PIXELS}^2 px, {RT_CAMERAS} inclinations",
            "rays_per_s": rays / ms * 1e3, "channel_rays_per_s": rays * RT_CHANNELS / ms * 1e3,
            "segments_per_pass": segs, "channel_segments_per_s": chseg_per_s, "roofline": rt_roof,
            "ms_per_pass": ms, "passes": reps,
            "gpu_launches_per_pass": 2 * RT_CAMERAS,      # per camera: profile cube, then the trace
            "emissivity_bytes": cube,
            "mc_fill": {"packets": fill_runs * per_run, "s": fill_s, "packets_per_s": fill_runs * per_run / fill_s,
                        "scatterings_per_s": fst.scatterings / fill_s,
                        "segments_per_s": (fst.scatterings + fst.crossings) / fill_s,
                        "note": "rich walk (excitation, J, destruction) recording each segment, then "
                                "the two-stage deposit: per segment up to ~20 channels x 3 cameras of "
                                "R_IIA-weighted emissivity (FP32 atomics); 100 runs of 1e6 packets, host-timed"},
            "min_hbm_gbs": cube / ms / 1e6,               # the emissivity cube read once per pass
            "l2": "inputs larger than L2 (emissivity 12.9 GB per pass)"}


BATCH_MODELS = 64
BATCH_PACKETS = 300_000
BATCH_TAU = (1e3, 1e5)


def bench_batch(args, dev, tau_range=None, total_packets=None, with_graph=True, tuned=None):
    """The many-model set at the scaled size (64 uniform spheres, sides in
    {32, 48, 64, 96, 128}, tau0 log-uniform in [1e3, 1e5], a log-uniform in
    [1e-4, 1e-2], v_max uniform in [-300, 300] km/s, 3e5 packets split in
    proportion to tau0): one persistent batched launch (launch parameters
    from the autotuner), the same launch replayed from a CUDA graph, and one
    launch per model on one stream, each over the same packets. tau_range
    and total_packets override the scaled set's, and tuned skips the
    autotuner (the full-range leg reuses the scaled set's choice)."""
    tau_range = tau_range or BATCH_TAU
    total_packets = total_packets or BATCH_PACKETS
    import torch
    import paper_2608_09340_gb300 as krl
    from paper_2608_09340_gb300 import autotune
    import workloads as W
    ms = W.model_set(n_models=BATCH_MODELS, total_packets=total_packets, tau_range=tau_range)
    grids = [krl.Grid(p, device=dev) for p in ms]
    pk = [p.n_packets for p in ms]
    stream = torch.cuda.current_stream(dev)

    def timed(fn):
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / 1e3

    def total_scat():
        return sum(int(g.tally("stats")[4]) for g in grids)

    try:
        b = krl.Batch(grids)
        # pilots of the full size (disjoint ids): a smaller pilot's time is set
        # by its own few longest packets and ranked close candidates by chance
        tune_table = None
        if tuned is not None:
            best = tuned
        else:
            best, timings = autotune.tune_batch(b, pk, fraction=1.0, repeats=1)
            tune_table = [[round(ms / 1e3, 4), cand] for ms, cand in timings]
        b.run(pk, seed=7, **best)                                  # warm-up
        for g in grids:
            g.reset()
        t_batch = timed(lambda: b.run(pk, seed=7, **best))
        scat = total_scat()
        t_graph = None
        if with_graph:
            for g in grids:
                g.reset()
            s = torch.cuda.Stream(device=dev)
            graph = torch.cuda.CUDAGraph()
            torch.cuda.synchronize(dev)
            with torch.cuda.graph(graph, stream=s):
                b.run(pk, seed=7, stream=s, **best)
            t_graph = timed(lambda: graph.replay())
            assert total_scat() == scat
        for g in grids:
            g.reset()
        t_single = timed(lambda: [g.run(n=n, seed=7, want_stats=False) for g, n in zip(grids, pk)])
        assert total_scat() == scat
        b.close()
    finally:
        for g in grids:
            g.close()
    return {"workload": f"{BATCH_MODELS} spheres, tau0 log-U{list(tau_range)}, {total_packets} packets",
            "scatterings": scat, "tuned": best, "tuning_s_per_candidate": tune_table,
            "batched_scat_per_s": scat / t_batch, "graph_scat_per_s": scat / t_graph if t_graph else None,
            "per_model_scat_per_s": scat / t_single, "speedup_vs_per_model": t_single / t_batch,
            "s_batched": t_batch, "s_graph": t_graph, "s_per_model": t_single}


def bench_next_rows(args, dev):
    """Timings of the rows beyond the core pass, each on its own workload:
    statistical equilibrium, the Lambda iteration on the molecular cloud (128^3, 5-level rotor,
    4 lines; 1e7 packets per line and cycle, 20 cycles, the change per cycle recorded);
    the line-profile modes, the Sec. 3.1 slab (a = 0.149, tau_m = 32000, 1e6 packets) in each
    line-profile mode (mode 1: 2-D table and sampler in global memory; mode
    2: the slice in shared memory; mode 3: the core-wing blend); continuum absorption, the
    Sec. 3.2 dusty slab at (a tau0)^{1/3} tau_a = 1 (2e5 packets)."""
    import dataclasses
    import math
    import numpy as np
    import torch
    import paper_2608_09340_gb300 as krl
    import workloads as W
    out = {}

    def timed(fn):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        r = fn()
        torch.cuda.synchronize(dev)
        return time.perf_counter() - t0, r

    # statistical equilibrium (Lambda iteration)
    p, n_mol, spec = W.cloud(n=128, packets_per_line=1_000_000)
    E, gdeg, A, k = spec.arrays()
    g = krl.Grid(p, device=dev)
    try:
        nm = torch.from_numpy(n_mol.reshape(-1)).to(dev)
        pops = torch.zeros((p.ncell, spec.n_lev), dtype=torch.float64, device=dev)
        desc = krl.levels_desc(E, gdeg, A, k, spec.mass_amu, nm)
        g.levels_iterate(desc, 1, 100_000, 1, pops, init_lte=True)          # warm-up
        n_iter, ppl = 20, 10_000_000          # the configuration's 20 cycles of 1e7 packets per line
        dt, ch = timed(lambda: g.levels_iterate(desc, n_iter, ppl, 2, pops, init_lte=True))
        n_lines = int((A > 0).sum())
        # The largest change over the 2.1e6 cells settles, after the first
        # cycle, at the Monte Carlo noise of the least-sampled cells; 4x the
        # packets per line should halve that plateau (N^-1/2) if it is noise
        _, ch4 = timed(lambda: g.levels_iterate(desc, 5, 4 * ppl, 3, pops, init_lte=True))
        plateau = float(np.median(ch[1:]))
        plateau4 = float(np.median(ch4[1:]))
        out["levels"] = {"workload": "cloud 128^3, 5-level rotor, 4 lines", "cycles": n_iter,
                         "packets_per_line": ppl, "s_per_cycle": dt / n_iter,
                         "packets_per_s": n_iter * n_lines * ppl / dt,
                         "max_change": [float(c) for c in ch],
                         "plateau": plateau, "plateau_4x_packets": plateau4,
                         "plateau_ratio": plateau / plateau4 if plateau4 > 0 else None}
    finally:
        g.close()

    # line-profile modes
    tau_m = 32000.0
    base = W.slab(tau0=tau_m / math.sqrt(math.pi), a=0.149, nz=128, n_packets=1_000_000, bins=(-40.0, 40.0, 800))
    modes = {}
    for m in (1, 2, 3):
        q = dataclasses.replace(base, line=dataclasses.replace(base.line, ph_mode=m))
        g = krl.Grid(q, device=dev)
        try:
            g.run(n=100_000, first=1 << 40, want_stats=False)                # warm-up
            g.reset()
            dt, st = timed(lambda: g.run(n=1_000_000, first=0)[0])
            modes[f"ph_mode_{m}"] = {"scat_per_s": st.scatterings / dt, "s": dt}
        finally:
            g.close()
    modes["mode1_over_mode2"] = modes["ph_mode_1"]["scat_per_s"] / modes["ph_mode_2"]["scat_per_s"]
    out["profile_modes"] = {"workload": "slab 128 cells, a = 0.149, tau_m = 32000, 1e6 packets", **modes}

    # Table placement (Sec. 2.3.1 recommends the constant bank): profile mode 2
    # with the slice and the sampler read from shared memory (the production
    # walk) and from the constant bank, on the same slab and on the 64^3
    # sphere at tau0 = 1e4 (2^19 packets: enough that the launch is not set
    # by its longest packets, as a short tau0 = 1e6 run would be)
    place = {}
    for wl, q, npk in (("slab", base, 200_000), ("sphere64_tau1e4", W.sphere(tau0=1e4), 1 << 19)):
        g = krl.Grid(q, device=dev)
        try:
            row = {}
            for nm, ts in (("shared", krl.KRL_TABLES_SHARED), ("constant", krl.KRL_TABLES_CONSTANT)):
                g.run(n=min(npk, 100_000) // 10, first=1 << 40, want_stats=False, table_space=ts)
                g.reset()
                dt, st = timed(lambda: g.run(n=npk, first=0, table_space=ts)[0])
                row[nm] = {"scat_per_s": st.scatterings / dt, "s": dt}
            row["constant_over_shared"] = row["constant"]["scat_per_s"] / row["shared"]["scat_per_s"]
            place[wl] = row
        finally:
            g.close()
    out["table_placement"] = {"workloads": "slab as above (2e5 packets); 64^3 tau0 = 1e4 sphere, 2^19 packets",
                              **place}

    # The paper's own timing setup (Sec. 3.5.2, Table 1: uniform 32^3 box,
    # line-centre tau0 = 1e3 from centre to face, T = 100 K, volume source with
    # the thermal profile), for N = 1e3 .. 1e7: the transport launch alone, and
    # the total including grid creation and the line's table builds. The
    # paper's figures are its code on one RTX 3090 (the MCRT column) and its
    # totals with ~0.3 s of fixed overheads; context, not a target.
    paper_mcrt_s = {1_000: 0.030, 10_000: 0.034, 100_000: 0.086, 1_000_000: 0.435, 10_000_000: 3.901}
    paper_total_s = {1_000: 0.42, 10_000: 0.31, 100_000: 0.38, 1_000_000: 0.84, 10_000_000: 5.44}
    rows = []
    wq = W.box(n_packets=1000)
    g = krl.Grid(wq, device=dev)
    g.run(n=1000, first=1 << 40, want_stats=False)                  # warm-up (module load, first launch)
    g.close()
    for npk in sorted(paper_mcrt_s):
        bq = W.box(n_packets=npk)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        g = krl.Grid(bq, device=dev)
        try:
            torch.cuda.synchronize(dev)
            t1 = time.perf_counter()
            st, _, _ = g.run(n=npk, first=0)
            torch.cuda.synchronize(dev)
            t2 = time.perf_counter()
        finally:
            g.close()
        rows.append({"packets": npk, "mcrt_s": t2 - t1, "total_s": t2 - t0,
                     "scatterings_per_s": st.scatterings / (t2 - t1),
                     "paper_rtx3090_mcrt_s": paper_mcrt_s[npk], "paper_rtx3090_total_s": paper_total_s[npk]})
    out["paper_table1_box"] = {"workload": "box 32^3, tau0 = 1e3, T = 100 K, a = 4.73e-3, volume source, "
                                           "thermal profile (the paper's timing setup)", "rows": rows}

    # continuum absorption
    a, tau0 = 0.015, 1e5
    q = W.dusty_slab(1.0 / (a * tau0) ** (1.0 / 3.0), tau0=tau0, a=a, n_packets=200_000)
    g = krl.Grid(q, device=dev)
    try:
        g.run(n=20_000, first=1 << 40, want_stats=False)
        g.reset()
        dt, st = timed(lambda: g.run(n=200_000, first=0)[0])
        f_esc = float(g.tally("spec_w").sum().item()) / 200_000
        out["dusty_slab"] = {"workload": "slab a = 0.015, tau0 = 1e5, (a tau0)^1/3 tau_a = 1, 2e5 packets",
                             "scat_per_s": st.scatterings / dt, "f_esc": f_esc, "absorbed": int(st.absorbed)}
    finally:
        g.close()
    return out


# ------------------------------------------------------------------ profiler cases
#
# Each case sets up its inputs, runs one warm-up launch and then --launches
# timed launches of the kernel of interest (so that a capture can skip the
# warm-up with `-s 1`), and prints the CUDA-event time per launch. The
# defaults keep a few GB at most on the device:
#
#   python bench.py --profile-case transport [--tau0 T] [--vmax V] [--packets N] [--launches K]
#   python bench.py --profile-case raytrace [--grid G] [--pixels P] [--channels C]
#   python bench.py --profile-case emissivity [--grid G] [--channels C] [--packets N]

def _timed_launches(fn, k):
    import torch
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(k):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / k


def profile_case(args):
    import torch
    import paper_2608_09340_gb300 as krl
    import workloads as W
    torch.cuda.set_device(0)
    k = [0]
    if args.profile_case == "transport":
        p = W.sphere(vmax_kms=args.vmax, tau0=args.tau0)
        ts = krl.KRL_TABLES_CONSTANT if args.table_space == "constant" else krl.KRL_TABLES_SHARED
        g = krl.Grid(p)
        try:
            g.run(n=args.packets, first=0, want_stats=False, table_space=ts)
            g.reset()

            def one():
                k[0] += 1
                g.run(n=args.packets, first=k[0] * args.packets, want_stats=False, table_space=ts)
            ms = _timed_launches(one, args.launches)
            st = g.tally("stats").cpu().numpy()
        finally:
            g.close()
        scat, cross = int(st[4]), int(st[5])
        out = {"case": "transport", "tau0": args.tau0, "vmax_kms": args.vmax, "packets": args.packets,
               "table_space": args.table_space,
               "ms_per_launch": ms, "scatterings_per_launch": scat / args.launches,
               "crossings_per_launch": cross / args.launches, "scat_per_s": scat / args.launches / ms * 1e3}
    elif args.profile_case == "emissivity":
        # the rich walk filling the envelope's emissivity cube (3 cameras)
        p = W.envelope(n=args.grid, n_ch=args.channels, n_packets=args.packets)
        g = krl.Grid(p)
        try:
            g.run(n=args.packets // 10, first=1 << 40, want_stats=False)
            g.reset()

            def one():
                k[0] += 1
                g.run(n=args.packets, first=k[0] * args.packets, want_stats=False)
            ms = _timed_launches(one, args.launches)
            st = g.tally("stats").cpu().numpy()
        finally:
            g.close()
        scat, cross = int(st[4]), int(st[5])
        out = {"case": "emissivity", "grid": args.grid, "channels": args.channels, "packets": args.packets,
               "ms_per_launch": ms, "segments_per_s": (scat + cross) / args.launches / ms * 1e3,
               "packets_per_s": args.packets / ms * 1e3}
    else:
        p = W.envelope(n=args.grid, n_ch=args.channels, n_packets=200_000)
        g = krl.Grid(p)
        try:
            g.run(want_stats=False)
            g.raytrace(0, args.pixels, args.pixels, fov_cells=float(args.grid))
            ms = _timed_launches(lambda: g.raytrace(1, args.pixels, args.pixels, fov_cells=float(args.grid)),
                                 args.launches)
        finally:
            g.close()
        rays = args.pixels * args.pixels
        out = {"case": "raytrace", "grid": args.grid, "pixels": args.pixels, "channels": args.channels,
               "ms_per_launch": ms, "rays_per_s": rays / ms * 1e3}
    print(json.dumps(out), flush=True)


def run_reference(args, rank):
    """The FP64 oracle as it stands, on the host cores, a bounded sample per step."""
    if rank != 0:
        return
    import numpy as np
    import oracle
    import workloads as W
    p = W.sphere(vmax_kms=0.0)
    cores = os.cpu_count() or 1
    per_step = max(cores, 16)
    oracle.build()
    oracle.line_tables(float(p.line.a_fixed), False)
    for s in range(args.warmup):
        oracle.run(p, n=cores, first=s * per_step, nthreads=cores)
    tot_scat = tot_pk = 0
    t0 = time.perf_counter()
    for s in range(args.steps):
        r = oracle.run(p, n=per_step, first=(args.warmup + s) * per_step, nthreads=cores)
        tot_scat += int(r["stats"][4])
        tot_pk += per_step
    dt = time.perf_counter() - t0
    val = tot_scat / dt
    sample = f"{per_step} packets per step of the 64^3 tau0=1e6 static sphere (ids advance per step), FP64"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "packets_per_s": tot_pk / dt,
        "config": {"workload": "sphere64_tau1e6_static", "packets_per_step": per_step},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def cpu_baseline(p):
    """Oracle on a bounded sample (about 10 s of host work) at N = 1, rank 0."""
    import oracle
    cores = os.cpu_count() or 1
    n = 40 * cores                  # about 12 s at the oracle's ~50 packets/s on 16 cores
    oracle.line_tables(float(p.line.a_fixed), False)
    t0 = time.perf_counter()
    r = oracle.run(p, n=n, first=JOB_PACKETS - n, nthreads=cores)
    dt = time.perf_counter() - t0
    # one core, on 4 packets of the same sample (~1 s)
    t1 = time.perf_counter()
    r1 = oracle.run(p, n=4, first=JOB_PACKETS - n, nthreads=1)
    dt1 = time.perf_counter() - t1
    return {"value": float(r["stats"][4]) / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "single_core_value": float(r1["stats"][4]) / dt1,
            "sample": f"{n} packets (ids {JOB_PACKETS - n}..{JOB_PACKETS - 1}) of the same static sphere, "
                      f"{int(r['stats'][4])} scatterings in {dt:.1f} s, FP64; single core: the first 4 of them"}


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.profile_case:
        args.packets = 1 << 21 if args.packets is None else args.packets
        args.tau0 = 3e4 if args.tau0 is None else args.tau0
        profile_case(args)
        return
    args.packets = PACKETS_PER_STEP if args.packets is None else args.packets
    args.tau0 = 1e6 if args.tau0 is None else args.tau0
    if args.impl == "reference":
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group("gloo")
        run_reference(args, rank)
        return
    import numpy as np
    import torch
    import paper_2608_09340_gb300 as krl
    from paper_2608_09340_gb300 import shard
    import workloads as W

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    krl.load_library()
    dev = torch.device("cuda", local)
    p = W.sphere(vmax_kms=0.0, tau0=args.tau0)
    B = args.packets
    g = krl.Grid(p, device=dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    # Steps are issued round robin on several streams: a step's launch starts on
    # the SMs that the previous step's tail (its last, longest packets) has
    # already released, as a production job streams its batches. Each stream
    # flushes L2 (its own 256 MiB write) before each of its steps.
    nstr = max(1, args.streams)
    streams = [torch.cuda.Stream(device=dev) for _ in range(nstr)]
    flushes = [flush] + [torch.empty(256 << 20, dtype=torch.uint8, device=dev) for _ in range(nstr - 1)]
    step_id = 0
    for _ in range(args.warmup):
        lo, n = shard.step_range(step_id, rank, world, B)
        g.run(n=n, first=lo, want_stats=False)
        step_id += 1
    g.reset()
    barrier()
    clocks = Clocks(local)
    clocks.start()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t_wall = time.perf_counter()
    t_start.record(stream)
    for st_ in streams:
        st_.wait_stream(stream)
    for k in range(args.steps):
        sk = streams[k % nstr]
        with torch.cuda.stream(sk):
            flushes[k % nstr].zero_()
            lo, n = shard.step_range(step_id, rank, world, B)
            ev[k][0].record(sk)
            g.run(n=n, first=lo, want_stats=False, stream=sk)
            ev[k][1].record(sk)
        step_id += 1
    for st_ in streams:
        stream.wait_stream(st_)
    exchange_bytes = 0
    if world > 1:
        # the job's one exchange: every rank ends with the whole job's tallies
        tallies = [g.tally("spec_n"), g.tally("spec_w"), g.tally("scatmap")]
        shard.reduce_tallies(tallies)
        exchange_bytes = sum(t.numel() * t.element_size() for t in tallies)
    t_end.record(stream)
    barrier()
    wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    kern_s = t_start.elapsed_time(t_end) / 1e3
    launch_ms = [a.elapsed_time(b) for a, b in ev]
    stats = g.tally("stats").cpu().numpy()
    scat, cross, emitted = int(stats[4]), int(stats[5]), int(stats[0])
    t_max = shard.max_over_ranks(kern_s)
    tot = torch.tensor([scat, cross, emitted], dtype=torch.float64, device=dev)
    shard.sum_over_ranks(tot)
    scat_all, cross_all, pk_all = [float(v) for v in tot.cpu()]
    value = scat_all / t_max

    # roofline (ALU-bound walk): algorithmic lane-ops per launch / mean launch time
    peaks, peak_kind = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    props = torch.cuda.get_device_properties(dev)
    peak_ops = props.multi_processor_count * FP32_LANES_PER_SM * sm_max * 1e6
    pv = profile_values()
    traffic, inst_per_event = pv.get("dram_bytes_per_launch_scaled"), pv.get("thread_instructions_per_event")
    # per GPU: this rank's events over its own timed region
    est_frac = (OPS_PER_SCAT * scat + OPS_PER_CROSS * cross) / kern_s / peak_ops
    if "arith_ops_per_scattering" in pv:
        ops_s, ops_c, ops_src = pv["arith_ops_per_scattering"], pv["arith_ops_per_crossing"], "ncu instruction mix"
    else:
        ops_s, ops_c, ops_src = OPS_PER_SCAT, OPS_PER_CROSS, "per-unit estimate (profile not on this source)"
    achieved = (ops_s * scat + ops_c * cross) / kern_s
    # issue ceiling: every SM sub-partition issuing one warp instruction per
    # cycle at full SIMT width, over the measured thread instructions per
    # scattering and per crossing
    issue_frac = None
    if "thread_instructions_per_scattering" in pv:
        issue_frac = (pv["thread_instructions_per_scattering"] * scat +
                      pv["thread_instructions_per_crossing"] * cross) / kern_s / peak_ops
    elif inst_per_event:
        issue_frac = inst_per_event * (scat + cross) / kern_s / peak_ops
    roof = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12, "unit": "Tops/s",
            "frac": achieved / peak_ops, "traffic": traffic, "issue_ceiling_frac": issue_frac,
            "frac_at_estimated_ops": est_frac, "estimated_ops_per_scattering": OPS_PER_SCAT,
            "estimated_ops_per_crossing": OPS_PER_CROSS,
            "thread_instructions_per_event": inst_per_event,
            "launch_ms_mean": sum(launch_ms) / len(launch_ms),
            "peak_source": f"{props.multi_processor_count} SMs x {FP32_LANES_PER_SM} FP32 lanes x "
                           f"{sm_max:.0f} MHz ({peak_kind} max SM clock)",
            "ops_per_scattering": ops_s, "ops_per_crossing": ops_c, "ops_source": ops_src}

    # One more job alone on one stream (no overlap of its tail with another
    # job): the rate a single job gets, beside the streamed rate above.
    serial = None
    if not args.no_serial_leg and world == 1 and nstr > 1:
        lo, n = shard.step_range(step_id, rank, world, B)
        step_id += 1
        flush.zero_()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        s0.record(stream)
        g.run(n=n, first=lo, want_stats=False, stream=stream)
        s1.record(stream)
        torch.cuda.synchronize(dev)
        st_after = g.tally("stats").cpu().numpy()
        sec = s0.elapsed_time(s1) / 1e3
        js = int(st_after[4]) - scat
        serial = {"scatterings_per_s": js / sec, "s": sec, "packets": n, "scatterings": js,
                  "alu_frac": (ops_s * js + ops_c * (int(st_after[5]) - cross)) / sec / peak_ops}

    # End to end through the public API with host buffers, jobs streamed the
    # way a user runs several: each job's grid is created from pinned host
    # fields on one of two alternating streams, its run and its result reads
    # (spectrum, scattering map, counters into pinned host buffers) are
    # enqueued on that stream, so one job's setup and tail overlap the next
    # job's walk. Grids are destroyed after the timed region (freeing device
    # memory synchronises the device).
    e2e = None
    if not args.no_e2e:
        op_host = torch.from_numpy(np.ascontiguousarray(p.opacity, dtype=np.float32)).pin_memory()
        e2e_steps = min(args.steps, E2E_MAX_STEPS)
        spec_h = [torch.empty(p.spectrum[2] + 2, dtype=torch.float64).pin_memory() for _ in range(e2e_steps)]
        scat_h = [torch.empty(p.ncell, dtype=torch.int64).pin_memory() for _ in range(e2e_steps)]
        stat_h = [torch.empty(8, dtype=torch.int64).pin_memory() for _ in range(e2e_steps)]
        e_streams = [torch.cuda.Stream(device=dev) for _ in range(2)]
        grids = []
        barrier()
        t0 = time.perf_counter()
        for k in range(e2e_steps):
            sk = e_streams[k % 2]
            with torch.cuda.stream(sk):
                q = W.sphere(vmax_kms=0.0, tau0=args.tau0)
                q.opacity = op_host          # pinned host buffer: copied by the binding's marshalling
                gg = krl.Grid(q, device=dev)
                grids.append(gg)
                lo, n = shard.step_range(step_id, rank, world, B)
                gg.run(n=n, first=lo, want_stats=False, stream=sk)
                spec_h[k].copy_(gg.tally("spec_w"), non_blocking=True)
                scat_h[k].copy_(gg.tally("scatmap"), non_blocking=True)
                stat_h[k].copy_(gg.tally("stats"), non_blocking=True)
            step_id += 1
        torch.cuda.synchronize(dev)
        e_dt = shard.max_over_ranks(time.perf_counter() - t0)
        for gg in grids:
            gg.close()
        e_scat = sum(int(h[4]) for h in stat_h)
        et = torch.tensor([float(e_scat)], dtype=torch.float64, device=dev)
        shard.sum_over_ranks(et)
        e2e = {"value": float(et.item()) / e_dt, "unit": UNIT,
               "h2d_bytes_per_step": int(op_host.numel() * 4),
               "d2h_bytes_per_step": int(spec_h[0].numel() * 8 + scat_h[0].numel() * 8 + 8 * 8),
               "steps": e2e_steps,
               "path": "per job: Grid from pinned host fields (grid creation, line tables), run, tally reads "
                       "into pinned host memory; jobs on two alternating streams"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(p)
    g.close()
    rt = None
    if rank == 0 and not args.no_raytrace:
        rt = bench_raytrace(args, dev)
    bt = None
    if rank == 0 and not args.no_batch:
        bt = bench_batch(args, dev)
        if args.batch_full_range:
            bt["full_range"] = bench_batch(args, dev, tau_range=(1e3, 1e7), total_packets=200_000, with_graph=False,
                                           tuned=bt["tuned"])
    nx = None
    if rank == 0 and not args.no_next:
        nx = bench_next_rows(args, dev)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "fp32", "data": "synthetic",
            "packets_per_s": pk_all / t_max,
            "config": {"workload": "sphere64_tau1e6_static" if args.tau0 == 1e6 else f"sphere64_tau{args.tau0:g}_static",
                       "grid": "64^3", "tau0": args.tau0, "a": 4.7e-4,
                       "T_K": 1e4, "source": "central point, line centre", "packets_per_step": B,
                       "job_packets": JOB_PACKETS, "scatterings_per_packet": scat_all / max(pk_all, 1),
                       "l2": "flushed before every timed step (256 MiB write)",
                       "steps_issue": f"{nstr} streams, round robin" if nstr > 1 else "one stream",
                       "parallelism": f"packet-id shards x{world}",
                       "exchange": f"tally all-reduce, {exchange_bytes} bytes per rank" if world > 1 else "none"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk, "raytrace": rt, "batch": bt,
            "next_rows": nx, "crossings_per_s": cross_all / t_max, "one_stream_job": serial,
            "gpu_launches": 2 * args.steps, "wall_s_timed": wall,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
