"""GPU walk (FP64 instantiation, the same kernel as production with double
arithmetic) against the FP64 oracle on the same Philox streams: packet by
packet and tally by tally, element by element."""
import dataclasses

import numpy as np
import pytest

import oracle
import workloads as W
from _gpu_common import check_lockstep, gpu_run, need_gpu

pytestmark = pytest.mark.gpu


def _cases():
    c = {}
    c["slab_tau1e4"] = W.slab(tau0=1e4, a=1e-2, n_packets=1000)
    c["sphere_outflow"] = W.sphere(vmax_kms=200.0, tau0=1e4, n=16, n_packets=1000)
    c["sphere_infall"] = W.sphere(vmax_kms=-200.0, tau0=1e4, n=16, n_packets=1000)
    rag = W.sphere(tau0=300.0, n=7, n_packets=777)                # odd grid, ragged packet count
    rag.source = dataclasses.replace(rag.source, pos=(3.5, 3.5, 3.5))
    c["sphere_ragged"] = rag
    c["thin_slab"] = W.thin_slab(n_packets=20000)
    c["box_volume"] = W.box(tau0=100.0, n=8, n_packets=3000, tallies=("scatmap", "exc"))
    c["envelope"] = W.envelope(n=16, n_ch=16, n_packets=2000)
    return c


CASES = _cases()


@pytest.mark.parametrize("name", list(CASES))
def test_lockstep(name):
    krl = need_gpu()
    p = CASES[name]
    gpu = gpu_run(krl, p, krl.KRL_PREC_FP64)
    rs = gpu["stats"]                       # this run's counters (krl_run_stats)
    gpu["stats"] = gpu.pop("stats_tally")   # the grid's accumulated counters
    assert rs.emitted == p.n_packets == rs.escaped + rs.destroyed + rs.stuck + rs.absorbed
    assert [rs.emitted, rs.escaped, rs.destroyed, rs.stuck, rs.scatterings, rs.crossings] == \
        [int(v) for v in gpu["stats"][:6]]
    check_lockstep(krl, p, gpu, p.n_packets, label=name)


def test_edge_cases():
    krl = need_gpu()
    p = W.slab(tau0=1e3, n_packets=64)
    # n = 0 is a no-op
    g = krl.Grid(p)
    try:
        st, rc, _ = g.run(n=0)
        assert st.emitted == 0 and rc == 0
        # one packet, far id, 64-bit id range
        st, rc, rec = g.run(n=1, first=(1 << 40) + 5, records=True, precision=krl.KRL_PREC_FP64)
        r = krl.records_to_numpy(rec)
        ref = oracle.run(p, n=1, first=(1 << 40) + 5, records=True)["records"]
        assert r["nscat"][0] == ref["nscat"][0] and r["status"][0] == ref["status"][0]
        # iteration budget: every packet stops after exactly max_iters iterations
        st, rc, rec = g.run(n=32, records=True, max_iters=50)
        assert rc == krl.KRL_ERR_BUDGET and st.stuck == 32
        r = krl.records_to_numpy(rec)
        assert np.all(r["status"] == 3) and np.all(r["nscat"] + r["ncross"] == 50)
    finally:
        g.close()
    # a source outside the domain leaves at once
    q = W.sphere(n=4, tau0=10.0, n_packets=100, tallies=())
    q.source = dataclasses.replace(q.source, pos=(-3.0, 2.0, 2.0))
    out = gpu_run(krl, q, krl.KRL_PREC_FP32)
    assert out["stats"].escaped == 100 and out["stats"].scatterings == 0
    assert np.all(out["records"]["cell0"] == 0xFFFFFFFF)


def test_bad_inputs_are_rejected():
    krl = need_gpu()
    p = W.slab(tau0=1e3, n_packets=8)
    p.opacity = p.opacity.copy()
    p.opacity[3] = np.nan
    with pytest.raises(krl.KrlError) as e:
        krl.Grid(p)
    assert e.value.status == krl.KRL_ERR_NUMERIC
    p = W.slab(tau0=1e3, n_packets=8)
    p.opacity = -p.opacity
    with pytest.raises(krl.KrlError) as e:
        krl.Grid(p)
    assert e.value.status == krl.KRL_ERR_NUMERIC
    q = W.box(n=4, tau0=1.0)
    q.source = dataclasses.replace(q.source, rate=np.zeros((4, 4, 4), np.float32))
    with pytest.raises(krl.KrlError) as e:
        krl.Grid(q)
    assert e.value.status == krl.KRL_ERR_ARG
    g = krl.Grid(W.slab(tau0=1e3, n_packets=8))
    try:
        with pytest.raises(krl.KrlError):
            g.run(block=48)
        with pytest.raises(krl.KrlError):
            g.run(refill_min=40)
    finally:
        g.close()
