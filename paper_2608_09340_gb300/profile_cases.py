"""Small, fixed cases of the device kernels for profiler captures.

    python -m paper_2608_09340_gb300.profile_cases transport [--tau0 T] [--packets N] [--launches K]
    python -m paper_2608_09340_gb300.profile_cases raytrace [--grid G] [--pixels P] [--channels C]
    python -m paper_2608_09340_gb300.profile_cases emissivity [--grid G] [--channels C] [--packets N]

Each case sets up its inputs, runs one warm-up launch and then K timed
launches of the kernel of interest (so a capture can skip the warm-up with
`-s 1`), and prints the CUDA-event time per launch. Sizes default to cases
that keep a few GB at most on the device.
"""
from __future__ import annotations

import argparse
import json
import os
import sys


def _timed(fn, k):
    import torch
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(k):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / k


def transport(args):
    import paper_2608_09340_gb300 as krl
    import workloads as W
    p = W.sphere(vmax_kms=args.vmax, tau0=args.tau0)
    g = krl.Grid(p)
    try:
        g.run(n=args.packets, first=0, want_stats=False)
        g.reset()
        k = [0]

        def one():
            k[0] += 1
            g.run(n=args.packets, first=k[0] * args.packets, want_stats=False)
        ms = _timed(one, args.launches)
        st = g.tally("stats").cpu().numpy()
    finally:
        g.close()
    scat, cross = int(st[4]), int(st[5])
    print(json.dumps({"case": "transport", "tau0": args.tau0, "vmax_kms": args.vmax, "packets": args.packets,
                      "ms_per_launch": ms, "scatterings_per_launch": scat / args.launches,
                      "crossings_per_launch": cross / args.launches,
                      "scat_per_s": scat / args.launches / ms * 1e3}))


def emissivity(args):
    """The rich walk filling the envelope's emissivity cube (3 cameras)."""
    import paper_2608_09340_gb300 as krl
    import workloads as W
    p = W.envelope(n=args.grid, n_ch=args.channels, n_packets=args.packets)
    g = krl.Grid(p)
    try:
        g.run(n=args.packets // 10, first=1 << 40, want_stats=False)
        g.reset()
        k = [0]

        def one():
            k[0] += 1
            g.run(n=args.packets, first=k[0] * args.packets, want_stats=False)
        ms = _timed(one, args.launches)
        st = g.tally("stats").cpu().numpy()
    finally:
        g.close()
    scat, cross = int(st[4]), int(st[5])
    print(json.dumps({"case": "emissivity", "grid": args.grid, "channels": args.channels, "packets": args.packets,
                      "ms_per_launch": ms, "segments_per_s": (scat + cross) / args.launches / ms * 1e3,
                      "packets_per_s": args.packets / ms * 1e3}))


def raytrace(args):
    import paper_2608_09340_gb300 as krl
    import workloads as W
    p = W.envelope(n=args.grid, n_ch=args.channels, n_packets=200_000)
    g = krl.Grid(p)
    try:
        g.run(want_stats=False)
        g.raytrace(0, args.pixels, args.pixels, fov_cells=float(args.grid))
        ms = _timed(lambda: g.raytrace(1, args.pixels, args.pixels, fov_cells=float(args.grid)), args.launches)
    finally:
        g.close()
    rays = args.pixels * args.pixels
    print(json.dumps({"case": "raytrace", "grid": args.grid, "pixels": args.pixels, "channels": args.channels,
                      "ms_per_launch": ms, "rays_per_s": rays / ms * 1e3}))


def main(argv=None):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["transport", "raytrace", "emissivity"])
    ap.add_argument("--tau0", type=float, default=3e4)
    ap.add_argument("--vmax", type=float, default=0.0)
    ap.add_argument("--packets", type=int, default=1 << 21)
    ap.add_argument("--grid", type=int, default=128)
    ap.add_argument("--pixels", type=int, default=512)
    ap.add_argument("--channels", type=int, default=64)
    ap.add_argument("--launches", type=int, default=1)
    args = ap.parse_args(argv)
    import torch
    torch.cuda.set_device(0)
    {"transport": transport, "raytrace": raytrace, "emissivity": emissivity}[args.case](args)


if __name__ == "__main__":
    main()
