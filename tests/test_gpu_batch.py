"""Many models in one persistent launch (krl_batch_run, the server-worker
scheduling of Sec. 2.3.2 over models): against the oracle model by model
(FP64 lockstep, and one FP32 model against a stored oracle run), exactly the
tallies of one krl_run_packets launch per model (one of them with continuum
absorption), also when the batched launch is captured into a CUDA graph and
replayed."""
import numpy as np
import pytest

import workloads as W
import _oracle_stats as S
from _gpu_common import check_lockstep, chi2_two_sample, grid_tallies, need_gpu, rel_l1, report

pytestmark = pytest.mark.gpu


def _models():
    ms = [W.sphere(vmax_kms=120.0, tau0=3e4, n=24, n_packets=3000, tallies=("scatmap",)),
          W.sphere(vmax_kms=0.0, tau0=2e3, n=16, n_packets=700, tallies=("scatmap",)),
          W.slab(tau0=5e3, a=1e-2, n_packets=1500),
          W.sphere(vmax_kms=-250.0, tau0=1e5, n=32, n_packets=2500, a=1e-3, tallies=("scatmap",)),
          W.box(tau0=50.0, n=8, n_packets=4000, tallies=("scatmap", "exc")),
          W.dusty_slab(0.1, tau0=3e3, n_packets=1500, bins=(-30.0, 30.0, 60))]
    for i, p in enumerate(ms):
        p.seed = 11
    return ms


def _tallies(g):
    out = {k: g.tally(k) for k in ("spec_n", "spec_w", "scatmap", "stats", "exc", "absw")}
    return {k: (None if v is None else v.cpu().numpy()) for k, v in out.items()}


def test_batch_equals_one_launch_per_model():
    krl = need_gpu()
    import torch
    ms = _models()
    single = []
    for p in ms:
        g = krl.Grid(p)
        g.run(first=100, seed=11, want_stats=False)
        torch.cuda.synchronize()
        single.append(_tallies(g))
        g.close()
    grids = [krl.Grid(p) for p in ms]
    try:
        b = krl.Batch(grids)
        st, rc = b.run([p.n_packets for p in ms], first_ids=[100] * len(ms), seed=11, want_stats=True)
        torch.cuda.synchronize()
        for m, (g, ref) in enumerate(zip(grids, single)):
            got = _tallies(g)
            assert np.array_equal(got["spec_n"], ref["spec_n"]), m
            assert np.array_equal(got["stats"], ref["stats"]), m
            if ref["scatmap"] is not None:
                assert np.array_equal(got["scatmap"], ref["scatmap"]), m
            if ref["exc"] is not None:
                assert np.allclose(got["exc"], ref["exc"], rtol=1e-5), m
            if ref["absw"] is not None:         # the dusty slab's absorbed weight
                # (summed in FP32 per cell visit; the visits are cut at the tail
                # compactions, which differ between launches: as exc, 1e-5)
                assert np.allclose(got["absw"], ref["absw"], rtol=1e-5, atol=1e-12), m
            assert np.allclose(got["spec_w"], ref["spec_w"], rtol=1e-9, atol=1e-12), m
            assert st[m].emitted == ms[m].n_packets and st[m].scatterings == ref["stats"][4]
        b.close()
    finally:
        for g in grids:
            g.close()


def test_batch_fp64_against_the_oracle():
    """The batched kernel in FP64 (the same walk in double): every model's
    packet records agree with the oracle's for >= 99.9 % of the packets, and
    its tallies and counters element by element (packets that diverge are
    rerun alone on both sides and taken out)."""
    krl = need_gpu()
    import torch
    ms = _models()
    grids = [krl.Grid(p) for p in ms]
    try:
        b = krl.Batch(grids)
        recs = [torch.empty(p.n_packets * krl.RECORD_DTYPE.itemsize, dtype=torch.uint8, device="cuda") for p in ms]
        st, rc = b.run([p.n_packets for p in ms], first_ids=[100] * len(ms), seed=11, precision=krl.KRL_PREC_FP64,
                       records=recs, want_stats=True)
        torch.cuda.synchronize()
        for m, (p, g) in enumerate(zip(ms, grids)):
            gpu = grid_tallies(g)
            gpu["records"] = krl.records_to_numpy(recs[m])
            assert st[m].emitted == p.n_packets
            ok, _ = check_lockstep(krl, p, gpu, p.n_packets, first=100, seed=11, label=f"batched model {m}")
            report("batch_fp64_lockstep", model=m, name=p.name, packets=p.n_packets, identical=float(ok.mean()))
        b.close()
    finally:
        for g in grids:
            g.close()


def test_batch_fp32_model_against_the_oracle():
    """One model of an FP32 batch -- the 32^3, tau0 = 1e5 outflow sphere at
    6e5 packets, batched with three other models -- against the stored FP64
    oracle run on the same ids and seed: relative L1 < 2 % and chi^2 p > 0.01
    of the escaped spectrum, and the scattering map's radial profile."""
    krl = need_gpu()
    import torch
    run = S.load("sphere32_tau1e5_out200_n6e5_seed0")
    assert S.is_current(run)
    seed = run["seed"]
    target = W.sphere(**run["workload"]["kwargs"], seed=seed)
    others = [W.sphere(vmax_kms=-150.0, tau0=3e4, n=24, n_packets=200_000, seed=seed),
              W.slab(tau0=1e4, n_packets=100_000, seed=seed),
              W.sphere(vmax_kms=0.0, tau0=1e4, n=48, n_packets=50_000, a=1e-3, seed=seed)]
    ms = [others[0], target] + others[1:]
    grids = [krl.Grid(p) for p in ms]
    try:
        b = krl.Batch(grids)
        pk = [p.n_packets for p in ms]
        pk[1] = run["n"]
        b.run(pk, first_ids=[run["first"]] * len(ms), seed=seed)
        torch.cuda.synchronize()
        t = grid_tallies(grids[1])
        b.close()
    finally:
        for g in grids:
            g.close()
    g_ = t["spec_n"].astype(np.int64)
    r = np.asarray(run["spec_c"], dtype=np.int64)
    l1, pv = rel_l1(g_, r), chi2_two_sample(g_, r)[2]
    gs = S.shell_profile(t["scatmap"], target.shape)
    rs = np.asarray(run["shells_per_batch"], dtype=np.float64).sum(axis=0)
    z = S.shell_z(gs, run["n"], run)
    report("batch_fp32_vs_oracle", case=run["case"], spectrum_l1=l1, spectrum_chi2_p=pv,
           shell_l1=rel_l1(gs, rs), shell_max_abs_z=float(np.abs(z).max()))
    assert int(g_.sum()) == run["n"]
    assert l1 < 0.02 and pv > 0.01, (l1, pv)
    assert rel_l1(gs, rs) < 0.02 and np.abs(z).max() < 4.5, z


def test_batch_in_a_cuda_graph():
    krl = need_gpu()
    import torch
    ms = _models()[:3]
    grids = [krl.Grid(p) for p in ms]
    try:
        b = krl.Batch(grids)
        pk = [p.n_packets for p in ms]
        b.run(pk, seed=3)
        torch.cuda.synchronize()
        once = [_tallies(g) for g in grids]
        for g in grids:
            g.reset()
        torch.cuda.synchronize()
        s = torch.cuda.Stream()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=s):
            b.run(pk, seed=3, stream=s)
        for g in grids:            # capture ran nothing
            assert int(g.tally("stats").cpu()[0]) == 0
        graph.replay()
        graph.replay()
        torch.cuda.synchronize()
        for g, ref in zip(grids, once):
            got = _tallies(g)
            assert np.array_equal(got["spec_n"], 2 * ref["spec_n"])
            assert np.array_equal(got["stats"], 2 * ref["stats"])
        b.close()
    finally:
        for g in grids:
            g.close()


def test_batch_detects_a_changed_line():
    krl = need_gpu()
    ms = _models()[:2]
    grids = [krl.Grid(p) for p in ms]
    try:
        b = krl.Batch(grids)
        import ctypes as C
        from paper_2608_09340_gb300 import krl_line_desc, krl_line_set
        b.run([10, 10], seed=1)
        # give grid 0 a new line through the C ABI
        L = krl_line_desc()
        L.nu0_hz, L.mass_amu, L.A_ul, L.g_u, L.g_l, L.a_fixed = 2.466e15, 1.00794, 6.265e8, 6.0, 2.0, 2e-3
        L.src_kind, L.spec_xmin, L.spec_xmax, L.spec_nbins = 0, -30.0, 30.0, 50
        L.src_pos = (C.c_double * 3)(12.0, 12.0, 12.0)
        krl_line_set(grids[0].handle, L)
        with pytest.raises(krl.KrlError) as e:
            b.run([10, 10], seed=1)
        assert e.value.status == krl.KRL_ERR_STATE
        b.close()
    finally:
        for g in grids:
            g.close()
