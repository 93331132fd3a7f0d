"""Host logic of the continuous-batching server on CPU: the batch engine is
replaced by a fake that advances generation counters, so admission order,
the memory cap, slicing and retirement are checked without a GPU.  The
request stream's recipe (near-square tori, log-uniform sizes) is checked
against its definition."""
import math

import numpy as np
import pytest

from paper_2404_10861_gb300 import serve


class FakeBatch:
    """Stands in for binding.Batch: runs advance one generation per tick."""

    log = None

    def __init__(self, stream=None):
        self.runs = {}
        self.next_id = 0
        self.ticks = 0
        FakeBatch.log = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False

    def add(self, generations, **cfg):
        rid = self.next_id
        self.next_id += 1
        self.runs[rid] = {"gen": 0, "budget": generations, "cfg": cfg, "live": True}
        FakeBatch.log.append(("add", rid, cfg["seed"]))
        return rid

    def info(self, rid):
        r = self.runs[rid]
        return {"generation": r["gen"], "done": r["gen"] >= r["budget"]}

    def run(self, ticks):
        assert ticks >= 1
        self.ticks += ticks
        for r in self.runs.values():
            if r["live"]:
                r["gen"] = min(r["budget"], r["gen"] + ticks)
        FakeBatch.log.append(("run", ticks))

    def sync(self):
        pass

    def sample(self, rid, k):
        seed = self.runs[rid]["cfg"]["seed"]
        words = np.full((k, 4), seed & 0xFFFFFFFF, dtype=np.uint32)
        where = np.zeros((k, 2), dtype=np.uint32)
        return words, where

    def remove(self, rid):
        self.runs[rid]["live"] = False
        FakeBatch.log.append(("remove", rid))

    def stats(self):
        return {"kernel_launches": 0, "tick": self.ticks}


class FakeGrid:
    """Stands in for binding.Grid (a large run advancing on its own grid)."""

    def __init__(self, stream=None, **cfg):
        self.cfg = cfg
        self.gen = 0
        FakeBatch.log.append(("grid", cfg["seed"]))

    def run(self, n):
        assert n >= 1
        self.gen += n
        FakeBatch.log.append(("grid_run", self.cfg["seed"], n))

    def sync(self):
        pass

    def sample(self, k):
        words = np.full((k, 4), self.cfg["seed"] & 0xFFFFFFFF, dtype=np.uint32)
        return words, np.zeros((k, 2), dtype=np.uint32)

    def stats(self):
        return {"kernel_launches": self.gen}

    def close(self):
        FakeBatch.log.append(("grid_close", self.cfg["seed"]))


def footprint(cfg):
    """The fake's device bytes: two 12-byte planes per agent plus records."""
    islands = cfg["rows"] * cfg["cols"]
    return islands * cfg["n"] * 24 + islands * 64


@pytest.fixture
def fake(monkeypatch):
    monkeypatch.setattr(serve.hb, "Batch", FakeBatch)
    monkeypatch.setattr(serve.hb, "Grid", FakeGrid)
    monkeypatch.setattr(serve.hb, "make_config", lambda **cfg: cfg)
    monkeypatch.setattr(serve.hb, "hsga_run_footprint", footprint)
    return FakeBatch


def request(rid, arrival, side, gens):
    cfg = dict(rows=side, cols=side, n=32, tournament=2, policy="tilted", bits=1, W=2,
               interval=1, p_ben=0.0, p_del=0.0, seed=1000 + rid)
    return serve.Request(rid, arrival, cfg, gens, 4)


def replay_memory(log, reqs):
    """Device bytes in use after every admission, from the fake's log."""
    by_seed = {r.config["seed"]: r for r in reqs}
    run_fp, in_use, peak = {}, 0, 0
    for ev in log:
        if ev[0] == "add":
            run_fp[ev[1]] = footprint(by_seed[ev[2]].config)
            in_use += run_fp[ev[1]]
            peak = max(peak, in_use)
        elif ev[0] == "remove":
            in_use -= run_fp[ev[1]]
    return peak, in_use


def test_every_request_completes_with_its_own_result(fake):
    reqs = [request(i, 0.001 * i, 8 + 4 * (i % 3), 50 + 37 * i) for i in range(12)]
    results, stats = serve.serve(reqs, memory_cap=1 << 30, slice_ticks=64)
    assert sorted(r.rid for r in results) == list(range(12))
    for r in results:
        req = reqs[r.rid]
        assert r.words.shape == (4, 4) and (r.words == req.config["seed"]).all()
        assert r.replications == req.agents * req.generations
        assert r.finished >= r.admitted >= r.arrival - 1e-9
    assert stats["admissions_deferred"] == 0
    adds = [ev for ev in fake.log if ev[0] == "add"]
    assert [ev[2] for ev in adds] == [1000 + i for i in range(12)]      # first come, first served
    assert sum(1 for ev in fake.log if ev[0] == "remove") == 12


def test_memory_cap_defers_admission_and_is_never_exceeded(fake):
    reqs = [request(i, 0.0, 16, 100 + 60 * i) for i in range(6)]
    one = footprint(reqs[0].config)
    cap = 2 * one + one // 2                   # room for two runs at a time
    results, stats = serve.serve(reqs, memory_cap=cap, slice_ticks=32)
    assert len(results) == 6
    assert stats["admissions_deferred"] > 0
    assert stats["peak_concurrent_runs"] == 2
    peak, left = replay_memory(fake.log, reqs)
    assert peak <= cap and left == 0
    adds = [ev[2] for ev in fake.log if ev[0] == "add"]
    assert adds == sorted(adds)                # deferral keeps arrival order


def test_slices_stop_at_the_earliest_finishing_run(fake):
    reqs = [request(0, 0.0, 8, 1000), request(1, 0.0, 8, 70)]
    serve.serve(reqs, memory_cap=1 << 30, slice_ticks=256)
    runs = [ev[1] for ev in fake.log if ev[0] == "run"]
    assert runs[0] == 70                       # the short run retires after its own budget
    assert sum(runs) == 1000


def test_request_over_the_cap_is_rejected(fake):
    reqs = [request(0, 0.0, 64, 10)]
    with pytest.raises(ValueError):
        serve.serve(reqs, memory_cap=footprint(reqs[0].config) - 1)


def test_request_stream_follows_its_recipe():
    reqs = serve.poisson_requests(400, rate=200.0, seed=5, gen_scale=10)
    arrivals = np.array([r.arrival for r in reqs])
    assert (np.diff(arrivals) > 0).all()
    gaps = np.diff(np.concatenate([[0.0], arrivals]))
    assert abs(gaps.mean() - 1 / 200.0) < 0.25 / 200.0      # exponential gaps, mean 1/rate
    for r in reqs:
        c = r.config
        islands = c["rows"] * c["cols"]
        assert c["rows"] & (c["rows"] - 1) == 0                      # a power of two
        assert c["rows"] <= math.sqrt(islands) + 1e-9 < 2 * c["rows"] + 1
        assert 1024 <= r.agents and islands * 32 - 32 * c["rows"] <= 4_194_304
        assert 100 <= r.generations <= 10_000
        assert c["policy"] in ("steady", "tilted", "stretched") and c["p_ben"] in (0.0, 1e-3)
        assert r.sample_k == min(10_000, islands)
    assert len({r.config["seed"] for r in reqs}) == len(reqs)
    logs = np.log([r.agents for r in reqs])
    # log-uniform sizes: the median of log(agents) near the middle of the range
    assert abs(np.median(logs) - (math.log(1024) + math.log(4_194_304)) / 2) < 0.6


def test_large_runs_one_at_a_time_and_small_ones_pass_them(fake):
    """Size-aware admission: requests of at least large_agents agents run one
    at a time in arrival order, each on a grid of its own advanced in slices
    beside the batch, and a small request that arrives behind a waiting large
    one is admitted at once."""
    big = 256            # 256 x 256 islands x 32 agents = 2.1M agents: large
    reqs = [request(0, 0.0, big, 300), request(1, 0.0, big, 200), request(2, 0.0, 8, 50),
            request(3, 0.0, big, 100), request(4, 0.0, 16, 80)]
    results, stats = serve.serve(reqs, memory_cap=1 << 34, slice_ticks=64,
                                 large_agents=1 << 20)
    assert sorted(r.rid for r in results) == list(range(5))
    for r in results:
        assert (r.words == reqs[r.rid].config["seed"]).all()
        assert r.replications == reqs[r.rid].agents * reqs[r.rid].generations
    assert stats["peak_concurrent_large_runs"] == 1
    assert stats["kernel_launches"] == 300 + 200 + 100     # the fake grids' generations
    seeds = {r.config["seed"]: r for r in reqs}
    admitted = [seeds[ev[-1] if ev[0] == "add" else ev[1]].rid for ev in fake.log
                if ev[0] in ("add", "grid")]
    assert admitted.index(2) < admitted.index(1) and admitted.index(4) < admitted.index(1)
    assert [a for a in admitted if reqs[a].agents >= 1 << 20] == [0, 1, 3]
    # large runs never enter the batch; each advances in slices of at most 64
    # generations to its budget; never two large grids open at once
    assert all(seeds[ev[2]].agents < 1 << 20 for ev in fake.log if ev[0] == "add")
    live, total = 0, {}
    for ev in fake.log:
        if ev[0] == "grid":
            live += 1
        elif ev[0] == "grid_close":
            live -= 1
        elif ev[0] == "grid_run":
            assert ev[2] <= 64
            total[ev[1]] = total.get(ev[1], 0) + ev[2]
        assert live <= 1
    assert total == {1000: 300, 1001: 200, 1003: 100}
    # inside the batch instead (large_apart=False), still one large run at a time
    serve.serve(reqs, memory_cap=1 << 34, slice_ticks=64, large_agents=1 << 20,
                large_apart=False)
    adds = [seeds[ev[2]].rid for ev in fake.log if ev[0] == "add"]
    assert [a for a in adds if reqs[a].agents >= 1 << 20] == [0, 1, 3]
    assert not any(ev[0] == "grid" for ev in fake.log)
    live_large, rid_to_req = 0, {}
    for ev in fake.log:                     # never two large runs live at once
        if ev[0] == "add":
            rid_to_req[ev[1]] = seeds[ev[2]]
            live_large += rid_to_req[ev[1]].agents >= 1 << 20
        elif ev[0] == "remove":
            live_large -= rid_to_req[ev[1]].agents >= 1 << 20
        assert live_large <= 1
    # without the size rule, admission is first come, first served
    serve.serve(reqs, memory_cap=1 << 34, slice_ticks=64, large_agents=None)
    adds = [seeds[ev[2]].rid for ev in fake.log if ev[0] == "add"]
    assert adds == [0, 1, 2, 3, 4]


def test_large_grids_count_against_the_memory_cap(fake):
    """A large run on its own grid holds its footprint until it retires:
    small requests that would exceed the cap beside it wait, and are
    admitted (in arrival order) once it has finished."""
    big, small = request(0, 0.0, 256, 150), [request(i, 0.0, 16, 40) for i in (1, 2)]
    cap = footprint(big.config) + footprint(small[0].config)     # room for one small beside it
    results, stats = serve.serve([big] + small, memory_cap=cap, slice_ticks=64,
                                 large_agents=1 << 20)
    assert sorted(r.rid for r in results) == [0, 1, 2]
    assert stats["admissions_deferred"] > 0
    order = [ev for ev in fake.log if ev[0] in ("grid", "add", "grid_close", "remove")]
    seeds = [ev[1] if ev[0] in ("grid", "grid_close") else ev[2] if ev[0] == "add" else None
             for ev in order]
    # the second small request is admitted only after the first one retired
    first_small_removed = next(i for i, ev in enumerate(order) if ev[0] == "remove")
    second_small_added = next(i for i, ev in enumerate(order)
                              if ev[0] == "add" and ev[2] == 1002)
    assert second_small_added > first_small_removed
    assert seeds[0] == 1000 and order[0][0] == "grid"           # the large run first
