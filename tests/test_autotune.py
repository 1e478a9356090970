"""Host logic of the launch autotuner, without a GPU: every candidate of the
search space is tried once on pilot packets under ids far from any real
run, candidates the walk rejects are skipped, the fastest wins, and the pilot
tallies are reset afterwards."""
import itertools

from paper_2608_09340_gb300 import autotune as AT


class FakeGrid:
    def __init__(self, reject_block=512):
        self.calls = []
        self.resets = 0
        self.reject_block = reject_block

    def run(self, **kw):
        if kw.get("block") == self.reject_block:
            raise RuntimeError("block not supported by this walk")
        self.calls.append(kw)

    def reset(self):
        self.resets += 1


class FakeBatch:
    def __init__(self, n_models):
        self.grids = [FakeGrid() for _ in range(n_models)]
        self.calls = []

    def run(self, packets, first_ids=None, seed=0, **kw):
        self.calls.append((list(packets), list(first_ids), seed, kw))


def _cost(kw):
    # a made-up timing surface with its minimum at block 256, refill 4, all CTAs
    return abs(kw["block"] - 256) / 64 + abs(kw["refill_min"] - 4) * 0.1 + 0.5 * kw["ctas_per_sm"] + 1.0


def test_tune_grid(monkeypatch):
    g = FakeGrid()

    def fake_time(fn):
        fn()
        return _cost(g.calls[-1])

    monkeypatch.setattr(AT, "_time", fake_time)
    best, timings = AT.tune_grid(g, n=1000, fraction=0.05, seed=7)
    assert best == {"block": 256, "refill_min": 4, "ctas_per_sm": 0}
    # 2 x 3 x 2 candidates, the block-512 half rejected by the walk
    assert len(timings) == 6 and len(g.calls) == 6
    assert [t[0] for t in timings] == sorted(t[0] for t in timings)
    assert all(c["n"] == 50 and c["first"] == AT.PILOT_FIRST_ID and c["seed"] == 7 for c in g.calls)
    tried = {(c["block"], c["refill_min"], c["ctas_per_sm"]) for c in g.calls}
    assert tried == set(itertools.product((256,), (1, 4, 16), (0, 1)))
    assert g.resets == 1


def test_tune_batch(monkeypatch):
    b = FakeBatch(3)

    def fake_time(fn):
        fn()
        return _cost(b.calls[-1][3])

    monkeypatch.setattr(AT, "_time", fake_time)
    best, timings = AT.tune_batch(b, [1000, 10, 3], fraction=0.2)
    assert best == {"block": 256, "refill_min": 4, "ctas_per_sm": 0}
    assert len(timings) == 12 and len(b.calls) == 24   # each candidate on two pilot sets
    for i, (packets, first, seed, _) in enumerate(b.calls):
        assert packets == [200, 2, 1]               # at least one pilot packet per model
        assert first == [AT.PILOT_FIRST_ID + (i % 2) * AT.PILOT_SET_STRIDE] * 3
    # the two sets are disjoint id ranges, far above the real runs' ids
    assert AT.PILOT_SET_STRIDE > 1000 and AT.PILOT_FIRST_ID + 2 * AT.PILOT_SET_STRIDE < 1 << 64
    assert [t[0] for t in timings] == sorted(t[0] for t in timings)
    assert timings[0][0] == 2 * _cost(best)
    assert all(g.resets == 1 for g in b.grids)
