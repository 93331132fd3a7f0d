"""Batched runs: many independent runs of uneven shape and configuration
advanced together (one launch per tick, ticks replayed from CUDA graphs,
runs admitted between calls) must each equal the oracle's run of the same
configuration, and the same configuration run alone on its own grid, bit
for bit, and a sampled end state must equal the oracle's sampling of that
population."""
import numpy as np
import pytest

from conftest import oracle_config

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_10861_gb300 import _build, binding
    _build.build()
    return binding


def mixed_runs(seed, count):
    """A mix like the batched workload: square and 2:1 tori, 16-64 agents per
    island, every policy, adaptation on or off, uneven budgets (scaled down)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        side = int(rng.choice([2, 3, 4, 8, 16]))
        rows, cols = (side, side) if rng.random() < 0.5 else (side, 2 * side)
        out.append((int(rng.integers(40, 400)),
                    dict(rows=rows, cols=cols, n=int(rng.integers(16, 65)),
                         tournament=int(rng.choice([1, 2, 2, 5])),
                         policy=str(rng.choice(["steady", "tilted", "stretched", "trivial", "none",
                                                "hybrid"])),
                         bits=int(rng.choice([1, 2, 4])), p_ben=float(rng.choice([0.0, 1e-3, 0.05])),
                         p_del=float(rng.choice([0.0, 0.02])), interval=int(rng.choice([1, 1, 2, 0])),
                         coarsen=int(rng.choice([1, 1, 3])),
                         seed=int(rng.integers(1, 2**40)))))
    return out


def alone(hb, gens, kw):
    with hb.Grid(kernel=hb.KERNEL_STREAMED, **kw) as g:
        g.run(gens)
        g.sync()
        return g.population()


def test_batch_runs_equal_oracle_and_runs_alone(hb, orc, oracle_pool):
    runs = mixed_runs(1, 24)
    want = [oracle_pool.submit(orc.run, oracle_config(orc, kw), None, None, 0, gens)
            for gens, kw in runs]
    with hb.Batch() as b:
        ids = [b.add(gens, **kw) for gens, kw in runs[:16]]
        b.run(100)                                         # first wave
        ids += [b.add(gens, **kw) for gens, kw in runs[16:]]   # admitted mid-flight
        b.run(10**6)                                       # until every run is done
        st = b.stats()
        assert st["active_runs"] == 0 and st["live_runs"] == len(runs)
        for rid, (gens, kw) in zip(ids, runs):
            info = b.info(rid)
            assert info["done"] and info["generation"] == gens
            t, s = b.population(rid)
            ot, os_, _ = want[ids.index(rid)].result()
            assert np.array_equal(t, ot), ("oracle", rid, kw)
            assert np.array_equal(s, os_), ("oracle", rid, kw)
            wt, ws = alone(hb, gens, kw)
            assert np.array_equal(t, wt), (rid, kw)
            assert np.array_equal(s, ws), (rid, kw)


def test_batch_sample_and_progress_queries(hb, orc):
    kw = dict(rows=8, cols=16, n=32, tournament=2, policy="tilted", bits=1, p_ben=1e-3, seed=9)
    with hb.Batch() as b:
        r0 = b.add(300, **kw)
        r1 = b.add(120, **dict(kw, seed=10))
        b.run(120)
        assert b.info(r1)["done"] and not b.info(r0)["done"]
        assert b.info(r0)["generation"] == 120
        t, s = b.population(r0)                             # mid-run state
        wt, ws = alone(hb, 120, kw)
        assert np.array_equal(t, wt) and np.array_equal(s, ws)
        b.run(1000)
        t, s = b.population(r0)
        w, where = b.sample(r0, 64)
        c = orc.Config(rows=8, cols=16, n=32, tournament=2, policy=orc.TILTED, bits=1, p_ben=1e-3,
                       seed=9)
        ow, owhere = orc.sample(c, t, s, 300, 64)
        assert np.array_equal(w, ow) and np.array_equal(where, owhere)
        b.remove(r1)
        assert b.stats()["live_runs"] == 1
        with pytest.raises(hb.HsgaError):
            b.population(r1)


def test_footprint_is_host_only(hb):
    cfg = hb.make_config(rows=64, cols=64, n=32)
    assert hb.hsga_run_footprint(cfg) >= 64 * 64 * 32 * 24


def runs_of_32(seed, count):
    """32-agent runs (the paper's island size) of every configuration the
    batch supports, on grids whose island count is and is not a multiple of
    the six-island work item."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        rows, cols = [(2, 3), (3, 4), (4, 6), (5, 7), (6, 6), (1, 13), (8, 9)][i % 7]
        out.append((int(rng.integers(30, 250)),
                    dict(rows=rows, cols=cols, n=32, tournament=int(rng.choice([1, 2, 2, 3, 5])),
                         policy=str(rng.choice(["steady", "tilted", "stretched", "trivial",
                                                "none", "hybrid"])),
                         bits=int(rng.choice([1, 2, 4])), p_ben=float(rng.choice([0.0, 0.05])),
                         p_del=float(rng.choice([0.0, 0.03])),
                         interval=int(rng.choice([1, 1, 2, 0])),
                         coarsen=int(rng.choice([1, 1, 2])), seed=int(rng.integers(1, 2**40)))))
    return out


def test_batch_of_32_agent_runs_equals_oracle(hb, orc, oracle_pool):
    runs = runs_of_32(7, 21)
    want = [oracle_pool.submit(orc.run, oracle_config(orc, kw), None, None, 0, gens)
            for gens, kw in runs]
    with hb.Batch() as b:
        ids = [b.add(gens, **kw) for gens, kw in runs[:12]]
        b.run(17)                                          # an odd tick count: parity moves
        ids += [b.add(gens, **kw) for gens, kw in runs[12:]]
        b.run(10**6)
        b.sync()
        for rid, (gens, kw), fut in zip(ids, runs, want):
            assert b.info(rid)["generation"] == gens
            t, s = b.population(rid)
            ot, os_, _ = fut.result()
            assert np.array_equal(t, ot), (rid, kw)
            assert np.array_equal(s, os_), (rid, kw)
