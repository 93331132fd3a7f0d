"""Pins for the oracle's free-running migration replay.

* Under the schedule that takes every neighbour's same-generation emigrant
  aimed at the island, free-running migration is the synchronous cycle: the
  replay must equal the synchronous run bit-exactly, and every genome's
  counter must equal the generation.
* Under the empty schedule it must equal the synchronous run with migration
  off.
* Under stale schedules, counters never exceed the island's generation and
  only sites written under a genome's own counter hold bits.
* A schedule naming an emigrant that was aimed elsewhere, or a cycle, is
  rejected.
"""
import numpy as np
import pytest

from paper_2404_10861_gb300 import inputs


CFGS = [dict(rows=4, cols=5, n=16, tournament=2, policy=1, bits=1, p_ben=0.01, seed=3),
        dict(rows=3, cols=3, n=32, tournament=5, policy=5, bits=2, p_ben=0.02, p_del=0.01, seed=4),
        dict(rows=1, cols=4, n=8, tournament=1, policy=0, bits=4, seed=5),
        dict(rows=2, cols=2, n=12, tournament=3, policy=2, bits=1, interval=2, seed=6)]


@pytest.mark.parametrize("kw", CFGS)
def test_sync_schedule_reproduces_sync_run(orc, kw):
    c = orc.Config(**kw)
    trait, surf = inputs.small_trait_population(c.agents, seed=1, levels=4)
    G0, n = 50, 30
    want = orc.run(c, trait, surf, G0=G0, generations=n)[:2]
    sched = orc.sync_schedule(c, G0, n)
    t, s, T = orc.run_async(c, trait, surf, np.full(c.agents, G0, np.uint32), G0, n, sched)
    assert np.array_equal(t, want[0]) and np.array_equal(s, want[1])
    assert np.all(T == G0 + n)


def test_empty_schedule_is_migration_off(orc):
    kw = dict(CFGS[0])
    c = orc.Config(**kw)
    c0 = orc.Config(**dict(kw, interval=0))
    trait, surf = inputs.small_trait_population(c.agents, seed=2)
    want = orc.run(c0, trait, surf, G0=7, generations=25)[:2]
    t, s, _ = orc.run_async(c, trait, surf, np.full(c.agents, 7, np.uint32), 7, 25,
                            np.zeros((c.islands, 25, 4), np.uint32))
    assert np.array_equal(t, want[0]) and np.array_equal(s, want[1])


def test_stale_schedule_counters_and_surfaces(orc):
    c = orc.Config(rows=6, cols=6, n=16, tournament=2, policy=orc.TILTED, bits=1, p_ben=0.01,
                   seed=9)
    n = 120
    sync = orc.sync_schedule(c, 0, n)
    rng = np.random.default_rng(0)
    sched = sync.copy()
    # take some emigrants late: the record the neighbour published up to 5
    # generations earlier is replaced by none unless it was aimed here too
    for i, g, d in zip(*np.nonzero(sync)):
        if rng.random() < 0.5:
            sched[i, g, d] = 0
    # and some islands take a neighbour's emigrant a few generations after it
    # was published (later generations of the receiver)
    moved = 0
    for i, g, d in zip(*np.nonzero(sync)):
        lag = int(rng.integers(1, 5))
        if sched[i, g, d] and g + lag < n and not sched[i, g + lag, d]:
            sched[i, g + lag, d] = sched[i, g, d]
            sched[i, g, d] = 0
            moved += 1
    assert moved > 50
    trait, surf = inputs.founders(c.agents)
    t, s, T = orc.run_async(c, trait, surf, np.zeros(c.agents, np.uint32), 0, n, sched)
    assert T.max() <= n and T.min() < n                  # stale immigrants carry older counters
    for Tv in np.unique(T):
        times = orc.lookup(c.policy, 64, 2, int(Tv))
        empty = np.uint64(sum(1 << int(p) for p in np.nonzero(times < 0)[0]))
        assert not np.any(s[T == Tv] & empty)


def test_inconsistent_schedules_rejected(orc):
    c = orc.Config(**CFGS[0])
    trait, surf = inputs.founders(c.agents)
    sync = orc.sync_schedule(c, 0, 10)
    bad = np.zeros_like(sync)
    i, g, d = [int(x) for x in np.argwhere(sync == 0)[0]]
    bad[i, g, d] = g + 1                                 # an emigrant aimed elsewhere
    ok_dirs = sync[i, g, d] == 0
    assert ok_dirs
    with pytest.raises(ValueError):
        orc.run_async(c, trait, surf, np.zeros(c.agents, np.uint32), 0, 10, bad)
    # a causal cycle: two neighbours each wait for the other's next emigrant
    cyc = np.zeros_like(sync)
    nb = orc.neighbour(c, 0, 1)                          # east neighbour of island 0
    cyc[0, 0, 1] = 2
    cyc[nb, 0, 3] = 2
    with pytest.raises(ValueError):
        orc.run_async(c, trait, surf, np.zeros(c.agents, np.uint32), 0, 10, cyc)
