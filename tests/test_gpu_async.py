"""Free-running migration on the GPU.

A free-running run is not reproducible (which neighbour records an island
takes depends on timing), but given the log of its takes it is
deterministic.  The oracle replays the GPU's own log and must reproduce every
trait, surface and per-genome counter bit-exactly -- on single runs of many
shapes, and on every one of 32 replicates, so the distribution of outcomes
(mean trait, phylometrics) over replicates is the oracle's exactly, not just
within a tolerance of it.  The replicates also report how free-running
differs from synchronous migration on the same seeds.
"""
import numpy as np
import pytest
from scipy import stats

from oracle import phylo
from paper_2404_10861_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_10861_gb300 import _build, binding
    _build.build()
    return binding


def ocfg(orc, kw):
    pol = orc.POLICY_NAMES[kw.get("policy", "steady")]
    return orc.Config(rows=kw["rows"], cols=kw["cols"], n=kw["n"],
                      tournament=kw.get("tournament", 2), policy=pol, bits=kw.get("bits", 1),
                      W=kw.get("W", 2), interval=kw.get("interval", 1),
                      p_ben=kw.get("p_ben", 0.0), p_del=kw.get("p_del", 0.0), seed=kw["seed"])


def run_logged(hb, kw, trait, surf, G0, chunks):
    gens = sum(chunks)
    with hb.Grid(mode="async", **kw) as g:
        g.set_population(trait, surf, G0)
        hb.hsga_set_async_log(g.handle, gens)
        for c in chunks:
            g.run(c)
        g.sync()
        t, s = g.population()
        T = g.counters()
        log = hb.hsga_get_async_log(g.handle, kw["rows"] * kw["cols"], gens)
        words, _ = g.sample(min(8, kw["rows"] * kw["cols"]))
    sched = np.where(log > 0, log - np.uint32(G0), 0).astype(np.uint32)
    return t, s, T, sched, words


CASES = [
    dict(rows=8, cols=8, n=32, tournament=2, policy="tilted", bits=1, p_ben=0.01, seed=1),
    dict(rows=16, cols=12, n=24, tournament=5, policy="hybrid", bits=2, p_ben=0.02, p_del=0.01,
         seed=2),
    dict(rows=1, cols=6, n=17, tournament=1, policy="steady", bits=4, seed=3),
    dict(rows=5, cols=5, n=32, tournament=3, policy="stretched", bits=1, interval=3, seed=4),
    dict(rows=64, cols=64, n=32, tournament=2, policy="tilted", bits=2, p_ben=1e-3, seed=5),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_async_run_replays_exactly(hb, orc, case):
    kw = CASES[case]
    c = ocfg(orc, kw)
    trait, surf = inputs.small_trait_population(c.agents, seed=case, levels=4)
    G0 = 100
    chunks = (60, 140) if case != 4 else (200,)
    t, s, T, sched, words = run_logged(hb, kw, trait, surf, G0, chunks)
    gens = sum(chunks)
    ot, os_, oT = orc.run_async(c, trait, surf, np.full(c.agents, G0, np.uint32), G0, gens,
                                sched)
    assert np.array_equal(t, ot) and np.array_equal(s, os_) and np.array_equal(T, oT)
    assert T.min() >= G0                                  # counters only grow
    # sampled records carry the genome's own counter
    assert np.all(np.isin(words[:, 3], T))
    if c.islands > 1 and case != 3:
        assert (sched > 0).sum() > 0                      # islands did take immigrants


def summary(orc, c, t, s, T, G):
    """Mean trait and phylometrics of 48 sampled genomes that share the
    modal counter (genomes carry their own counters in free-running mode)."""
    Tm = np.bincount(T).argmax()
    pool = s[T == Tm]
    rng = np.random.default_rng(0)
    pick = rng.choice(len(pool), size=min(48, len(pool)), replace=False)
    m = phylo.phylometrics(phylo.reconstruct(pool[pick], c.policy, c.bits, c.W, int(Tm)))
    return [float(t.mean()), m["mean_pairwise_distance"], m["sackin"], m["colless"]]


def test_async_replicates_replay_exactly(hb, orc):
    kw = dict(rows=8, cols=8, n=32, tournament=2, policy="tilted", bits=1, p_ben=5e-3)
    gens, reps = 300, 32
    gpu, ora, sync, takes = [], [], [], 0
    for r in range(reps):
        kwr = dict(kw, seed=100 + r)
        c = ocfg(orc, kwr)
        trait, surf = inputs.founders(c.agents)
        t, s, T, sched, _ = run_logged(hb, kwr, trait, surf, 0, (gens,))
        ot, os_, oT = orc.run_async(c, trait, surf, np.zeros(c.agents, np.uint32), 0, gens,
                                    sched)
        assert np.array_equal(t, ot) and np.array_equal(s, os_) and np.array_equal(T, oT), r
        gpu.append(summary(orc, c, t, s, T, gens))
        ora.append(summary(orc, c, ot, os_, oT, gens))
        takes += int((sched > 0).sum())
        with hb.Grid(**kwr) as g:                         # synchronous, same seed
            g.run(gens)
            g.sync()
            st, ss = g.population()
        sync.append(summary(orc, c, st, ss, np.full(c.agents, gens, np.uint32), gens))
    gpu, ora, sync = np.array(gpu), np.array(ora), np.array(sync)
    assert np.array_equal(gpu, ora)                       # identical distributions
    rate = takes / (reps * 64 * gens)
    assert 0 < rate <= 1.0                                # at most one per island-generation
    print(f"free-running takes per island-generation {rate:.3f}; mean trait "
          f"{gpu[:, 0].mean():.2f} vs synchronous {sync[:, 0].mean():.2f}; mean pairwise "
          f"distance {gpu[:, 1].mean():.1f} vs {sync[:, 1].mean():.1f}")


@pytest.mark.parametrize("mode", ["async", "buffered"])
@pytest.mark.parametrize("slice_", [1, 7])
def test_octet_slices_replay_exactly(hb, orc, mode, slice_):
    """Octets advanced several generations per visit (hsga_set_octet_slice)
    on a grid with more octets than resident warps, so warps page octets in
    and out: the logged run still replays exactly (latest-emigrant records
    with the oracle's async replay, per-neighbour buffers with its buffered
    replay)."""
    kw = dict(rows=192, cols=160, n=32, tournament=2, policy="tilted", bits=1, p_ben=0.02,
              seed=31)
    c = ocfg(orc, kw)
    trait, surf = inputs.small_trait_population(c.agents, seed=5, levels=4)
    G0, gens = 50, 30
    with hb.Grid(mode=mode, **kw) as g:
        g.set_population(trait, surf, G0)
        hb.hsga_set_octet_slice(g.handle, slice_)
        hb.hsga_set_async_log(g.handle, gens)
        g.run(13)
        g.run(gens - 13)
        g.sync()
        t, s = g.population()
        T = g.counters()
        log = hb.hsga_get_async_log(g.handle, c.islands, gens)
    T0 = np.full(c.agents, G0, np.uint32)
    if mode == "async":
        sched = np.where(log > 0, log - np.uint32(G0), 0).astype(np.uint32)
        ot, os_, oT = orc.run_async(c, trait, surf, T0, G0, gens, sched)
        assert (sched > 0).sum() > 0
    else:
        ot, os_, oT, _, _ = orc.run_buffered(c, trait, surf, T0, G0, gens, log)
        assert (log >> 1).sum() > 0
    assert np.array_equal(t, ot) and np.array_equal(s, os_) and np.array_equal(T, oT)


def test_octet_slice_is_only_for_free_running_grids(hb):
    with hb.Grid(rows=4, cols=4, n=32) as g:
        with pytest.raises(hb.HsgaError):
            hb.hsga_set_octet_slice(g.handle, 4)
    with hb.Grid(rows=4, cols=4, n=32, mode="async") as g:
        for bad in (0, 65537):
            with pytest.raises(hb.HsgaError):
                hb.hsga_set_octet_slice(g.handle, bad)
