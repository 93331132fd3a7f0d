"""Float fitness (binary32 fitness word, sign-restricted Gaussian mutation) on
the GPU: bit-exact against the oracle in synchronous mode, and exact oracle
replay of logged free-running runs.  Every float step on both sides is one
correctly rounded IEEE operation, so the comparison is exact, not within a
tolerance."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
UNSUPPORTED = -6


@pytest.fixture(scope="module")
def hb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_10861_gb300 import _build, binding
    _build.build()
    return binding


def ocfg(orc, kw):
    return orc.Config(rows=kw["rows"], cols=kw["cols"], n=kw["n"],
                      tournament=kw.get("tournament", 5),
                      policy=orc.POLICY_NAMES[kw.get("policy", "tilted")],
                      bits=kw.get("bits", 1), W=kw.get("W", 2), interval=kw.get("interval", 1),
                      p_ben=kw.get("p_ben", 0.003), p_del=kw.get("p_del", 0.33),
                      seed=kw["seed"], coarsen=kw.get("coarsen", 1),
                      fitness=orc.FITNESS_FLOAT, sigma=kw["sigma"])


def gkw(kw):
    out = dict(tournament=5, policy="tilted", p_ben=0.003, p_del=0.33)
    out.update({k: v for k, v in kw.items() if k != "sigma"})
    out["fitness"] = "float"
    out["sigma"] = kw["sigma"]
    return out


SYNC = [
    dict(rows=8, cols=8, n=32, sigma=1.0, seed=1),
    dict(rows=5, cols=7, n=19, sigma=0.25, seed=2, policy="steady", bits=2),
    dict(rows=3, cols=4, n=32, sigma=3.0, seed=3, policy="hybrid", bits=2, tournament=2),
    dict(rows=6, cols=6, n=8, sigma=0.5, seed=4, policy="none", p_ben=0.2),
    dict(rows=4, cols=9, n=32, sigma=1.5, seed=5, coarsen=3, interval=2),
    dict(rows=1, cols=1, n=1, sigma=2.0, seed=6, tournament=1, p_ben=0.5, p_del=0.5),
]


@pytest.mark.parametrize("case", range(len(SYNC)))
def test_float_sync_bit_exact(hb, orc, case):
    kw = SYNC[case]
    c = ocfg(orc, kw)
    rng = np.random.default_rng(case)
    f = rng.normal(0, 2, c.agents).astype(np.float32)
    surf = rng.integers(0, 2**63, c.agents, dtype=np.uint64)
    if c.policy == orc.NONE:
        surf[:] = 0
    G0, gens = 11, 120
    want_t, want_s, _ = orc.run(c, trait=f.view(np.uint32), surf=surf, G0=G0, generations=gens)
    with hb.Grid(**gkw(kw)) as g:
        g.set_population(f.view(np.uint32), surf, G0)
        g.run(50)
        g.run(gens - 50)
        t, s = g.population()
    assert np.array_equal(t, want_t) and np.array_equal(s, want_s)
    assert (t.view(np.float32) != f).any()


def test_float_premigrated_run(hb, orc):
    kw = dict(rows=4, cols=4, n=32, sigma=1.0, seed=8)
    c = ocfg(orc, kw)
    trait, surf = orc.founders(c)
    m_t, m_s = orc.migrate(c, trait, surf, 0)
    want_t, want_s, _ = orc.run(c, trait=m_t, surf=m_s, G0=0, generations=40, premigrated=True)
    with hb.Grid(**gkw(kw)) as g:
        g.migrate()
        g.run(40)
        t, s = g.population()
    assert np.array_equal(t, want_t) and np.array_equal(s, want_s)


@pytest.mark.parametrize("mode", ["async", "buffered"])
def test_float_free_running_replays_exactly(hb, orc, mode):
    kw = dict(rows=8, cols=6, n=32, sigma=0.8, seed=9, policy="tilted")
    c = ocfg(orc, kw)
    f = np.zeros(c.agents, np.float32)
    surf = np.zeros(c.agents, np.uint64)
    G0, gens = 0, 150
    with hb.Grid(mode=mode, **gkw(kw)) as g:
        g.set_population(f.view(np.uint32), surf, G0)
        hb.hsga_set_async_log(g.handle, gens)
        g.run(gens)
        g.sync()
        t, s = g.population()
        T = g.counters()
        log = hb.hsga_get_async_log(g.handle, c.islands, gens)
    T0 = np.zeros(c.agents, np.uint32)
    if mode == "async":
        sched = np.where(log > 0, log - np.uint32(G0), 0).astype(np.uint32)
        ot, os_, oT = orc.run_async(c, f.view(np.uint32), surf, T0, G0, gens, sched)
    else:
        ot, os_, oT, _, _ = orc.run_buffered(c, f.view(np.uint32), surf, T0, G0, gens, log)
    assert np.array_equal(t, ot) and np.array_equal(s, os_) and np.array_equal(T, oT)
    # selection (tournament 5) spreads the rare beneficial amounts
    assert np.unique(t).size > 10 and (t.view(np.float32) > 0).any()


def test_float_config_rules(hb):
    ok = dict(rows=2, cols=2, n=32, tournament=5, fitness="float", sigma=1.0)
    with hb.Grid(**ok):
        pass
    for bad, status in [(dict(ok, n=33), -1),
                        (dict(ok, sigma=0.0), -1),
                        (dict(ok, kernel=hb.KERNEL_RESIDENT), UNSUPPORTED)]:
        with pytest.raises(hb.HsgaError) as e:
            hb.Grid(**bad)
        assert e.value.status == status
    with hb.Batch() as b:
        with pytest.raises(hb.HsgaError) as e:
            b.add(10, **ok)
        assert e.value.status == UNSUPPORTED
