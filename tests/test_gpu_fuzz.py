"""Seeded random configurations against the oracle.

Each case draws a valid configuration -- torus shape (including degenerate
1xC and Rx1 tori), agents per island 1-64, tournament 1-8, policy, differentia
width 1-16, sites per level, surface words, migration interval 0-3, temporal
coarsening, mutation rates, integer or float fitness, kernel, starting
generation and how the run is split into calls -- and requires the library's
population and samples to equal the oracle's.  Free-running cases are
replayed from the GPU's own log.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

POLICIES = ["steady", "tilted", "stretched", "trivial", "none", "hybrid"]


@pytest.fixture(scope="module")
def hb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_10861_gb300 import _build, binding
    _build.build()
    return binding


def draw(rng, mode):
    """A valid configuration for `mode` ("sync", "async" or "buffered")."""
    while True:
        kw = dict(rows=int(rng.choice([1, 2, 3, 5, 8, 13])), cols=int(rng.choice([1, 2, 4, 7, 11])),
                  tournament=int(rng.integers(1, 9)), policy=str(rng.choice(POLICIES)),
                  bits=int(rng.choice([1, 2, 4, 8, 16])), W=int(rng.choice([1, 2, 4])),
                  interval=int(rng.integers(0, 4)), p_ben=float(rng.choice([0, 0.01, 0.2])),
                  p_del=float(rng.choice([0, 0.05, 0.3])), seed=int(rng.integers(1, 2**40)))
        kw["n"] = int(rng.integers(1, 33 if mode != "sync" else 65))
        words, coarsen, fitness, kernel = 1, 1, "trait", 0
        if mode == "sync":
            fitness = str(rng.choice(["trait", "trait", "float"]))
            kernel = int(rng.choice([0, 1, 2, 3]))
            coarsen = int(rng.choice([1, 1, 2, 3]))
            if rng.random() < 0.25:
                words = int(rng.choice([2, 4]))
        if fitness == "float" or words > 1:
            kw["n"] = min(kw["n"], 32)
            kernel = int(rng.choice([0, 1]))
            if words > 1 and kw["policy"] == "none":
                kw["policy"] = "tilted"
        S = 64 * words // kw["bits"]
        if kw["policy"] in ("tilted", "stretched") and S // kw["W"] < 2:
            continue
        if kw["policy"] == "hybrid" and (S // 2) // kw["W"] < 2:
            continue
        if kw["policy"] == "steady" and S < 2:
            continue
        kw.update(words=words, coarsen=coarsen, fitness=fitness, kernel=kernel, mode=mode)
        if fitness == "float":
            kw["sigma"] = float(rng.choice([0.25, 1.0, 3.0]))
        return kw


def ocfg(orc, kw):
    return orc.Config(rows=kw["rows"], cols=kw["cols"], n=kw["n"], tournament=kw["tournament"],
                      policy=orc.POLICY_NAMES[kw["policy"]], bits=kw["bits"], W=kw["W"],
                      interval=kw["interval"], p_ben=kw["p_ben"], p_del=kw["p_del"],
                      seed=kw["seed"], coarsen=kw["coarsen"],
                      fitness=orc.FITNESS_FLOAT if kw["fitness"] == "float" else 0,
                      sigma=kw.get("sigma", 1.0), words=kw["words"])


def start_state(rng, c, kw):
    if kw["fitness"] == "float":
        trait = rng.normal(0, 1, c.agents).astype(np.float32).view(np.uint32)
    else:
        trait = rng.integers(0, 6, c.agents).astype(np.uint32)
    surf = rng.integers(0, 2**64 - 1, c.agents * c.words, dtype=np.uint64, endpoint=True)
    if kw["policy"] == "none":
        surf[:] = 0
    return trait, surf


@pytest.mark.parametrize("case", range(150))
def test_random_sync_config(hb, orc, case):
    rng = np.random.default_rng(1000 + case)
    kw = draw(rng, "sync")
    c = ocfg(orc, kw)
    trait, surf = start_state(rng, c, kw)
    G0 = int(rng.integers(0, 5000))
    chunks = [int(x) for x in rng.integers(1, 40, size=int(rng.integers(1, 4)))]
    gens = sum(chunks)
    want_t, want_s, _ = orc.run(c, trait=trait, surf=surf, G0=G0, generations=gens)
    k = int(rng.integers(1, c.islands + 1))
    want_w, want_where = orc.sample(c, want_t, want_s, G0 + gens, k)
    with hb.Grid(**kw) as g:
        g.set_population(trait, surf, G0)
        for ch in chunks:
            g.run(ch)
        t, s = g.population()
        w, where = g.sample(k)
    assert np.array_equal(t, want_t) and np.array_equal(s, want_s), kw
    assert np.array_equal(w, want_w) and np.array_equal(where, want_where), kw


@pytest.mark.parametrize("mode", ["async", "buffered"])
@pytest.mark.parametrize("case", range(20))
def test_random_free_running_config(hb, orc, mode, case):
    rng = np.random.default_rng(5000 + case + (100 if mode == "buffered" else 0))
    kw = draw(rng, mode)
    c = ocfg(orc, kw)
    trait, surf = start_state(rng, c, kw)
    G0 = int(rng.integers(0, 500))
    gens = int(rng.integers(5, 80))
    with hb.Grid(**kw) as g:
        g.set_population(trait, surf, G0)
        hb.hsga_set_async_log(g.handle, gens)
        g.run(gens)
        g.sync()
        t, s = g.population()
        T = g.counters()
        log = hb.hsga_get_async_log(g.handle, c.islands, gens)
    T0 = np.full(c.agents, G0, np.uint32)
    if mode == "async":
        sched = np.where(log > 0, log - np.uint32(G0), 0).astype(np.uint32)
        ot, os_, oT = orc.run_async(c, trait, surf, T0, G0, gens, sched)
    else:
        ot, os_, oT, _, _ = orc.run_buffered(c, trait, surf, T0, G0, gens, log)
    assert np.array_equal(t, ot) and np.array_equal(s, os_) and np.array_equal(T, oT), kw
