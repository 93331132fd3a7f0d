"""Surfaces of several 64-bit words (128- and 256-bit fields) and 16-bit
differentiae on the GPU: populations, samples and reconstructions bit-exact
with the oracle."""
import numpy as np
import pytest

from oracle import phylo

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


DEFAULTS = dict(tournament=2, W=2, interval=1, p_ben=0.01, p_del=0.0, coarsen=1, words=1)


def gkw(kw):
    """The run's keyword arguments for the library, defaults filled in."""
    return {**DEFAULTS, **kw}


def ocfg(orc, kw):
    kw = gkw(kw)
    return orc.Config(rows=kw["rows"], cols=kw["cols"], n=kw["n"], tournament=kw["tournament"],
                      policy=orc.POLICY_NAMES[kw["policy"]], bits=kw["bits"], W=kw["W"],
                      interval=kw["interval"], p_ben=kw["p_ben"], p_del=kw["p_del"],
                      seed=kw["seed"], coarsen=kw["coarsen"],
                      fitness=orc.FITNESS_FLOAT if kw.get("fitness") == "float" else 0,
                      sigma=kw.get("sigma", 1.0), words=kw["words"])


CASES = [
    dict(rows=6, cols=5, n=32, policy="tilted", bits=1, words=4, seed=1),          # 256-bit field
    dict(rows=4, cols=4, n=32, policy="steady", bits=1, words=4, seed=2),
    dict(rows=3, cols=7, n=20, policy="stretched", bits=2, words=2, seed=3),
    dict(rows=5, cols=5, n=32, policy="hybrid", bits=4, words=4, tournament=5, seed=4),
    dict(rows=4, cols=6, n=16, policy="tilted", bits=16, words=4, W=1, seed=5),   # 16 x 16-bit
    dict(rows=4, cols=4, n=32, policy="trivial", bits=8, words=2, seed=6),
    dict(rows=6, cols=6, n=32, policy="tilted", bits=1, words=2, coarsen=3, interval=2, seed=7),
    dict(rows=4, cols=4, n=32, policy="tilted", bits=2, words=4, fitness="float", sigma=0.5,
         p_del=0.33, tournament=5, seed=8),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_wide_runs_bit_exact(hb, orc, case):
    kw = CASES[case]
    c = ocfg(orc, kw)
    rng = np.random.default_rng(case)
    trait = rng.integers(0, 5, c.agents).astype(np.uint32)
    if kw.get("fitness") == "float":
        trait = rng.normal(0, 1, c.agents).astype(np.float32).view(np.uint32)
    surf = rng.integers(0, 2**63, c.agents * c.words, dtype=np.uint64)
    G0, gens = 9, 150
    want_t, want_s, _ = orc.run(c, trait=trait, surf=surf, G0=G0, generations=gens)
    want_w, want_where = orc.sample(c, want_t, want_s, G0 + gens, min(10, c.islands))
    with hb.Grid(**gkw(kw)) as g:
        g.set_population(trait, surf, G0)
        g.run(60)
        g.run(gens - 60)
        t, s = g.population()
        w, where = g.sample(min(10, c.islands))
    assert np.array_equal(t, want_t) and np.array_equal(s, want_s)
    assert np.array_equal(w, want_w) and np.array_equal(where, want_where)


def test_wide_premigrated_run(hb, orc):
    kw = dict(rows=4, cols=4, n=32, policy="tilted", bits=1, words=4, seed=11)
    c = ocfg(orc, kw)
    trait, surf = orc.founders(c)
    m_t, m_s = orc.migrate(c, trait, surf, 0)
    want_t, want_s, _ = orc.run(c, trait=m_t, surf=m_s, G0=0, generations=30, premigrated=True)
    with hb.Grid(**gkw(kw)) as g:
        g.migrate()
        g.run(30)
        t, s = g.population()
    assert np.array_equal(t, want_t) and np.array_equal(s, want_s)


@pytest.mark.parametrize("kernel", [1, 2])
def test_sixteen_bit_differentiae_one_word(hb, orc, kernel):
    kw = dict(rows=4, cols=4, n=32, policy="tilted", bits=16, W=2, seed=12, kernel=kernel)
    c = ocfg(orc, kw)
    want_t, want_s, _ = orc.run(c, generations=200)
    with hb.Grid(**gkw(kw)) as g:
        g.run(200)
        t, s = g.population()
    assert np.array_equal(t, want_t) and np.array_equal(s, want_s)


@pytest.mark.parametrize("policy,bits,words,W,G", [(1, 1, 4, 2, 3000), (0, 1, 4, 2, 900),
                                                   (5, 2, 2, 2, 700), (1, 16, 4, 1, 500)])
def test_wide_reconstruction_matches_oracle(hb, orc, policy, bits, words, W, G):
    c = orc.Config(rows=6, cols=6, n=32, tournament=2, policy=policy, bits=bits, W=W,
                   interval=1, p_ben=0.01, seed=30 + policy, words=words)
    _, surf, _ = orc.run(c, generations=G)
    want = phylo.reconstruct(surf, policy, bits, W, G, words=words)
    parent, time, leaf = hb.hsga_reconstruct(surf, policy, bits, W, G, words=words)
    assert len(parent) == want.n_nodes
    mine = phylo.Tree(parent, time, leaf)
    assert phylo.sum_branch_length(mine) == phylo.sum_branch_length(want)
    rng = np.random.default_rng(0)
    for _ in range(400):
        a, b = (int(v) for v in rng.choice(c.agents, size=2, replace=False))
        assert phylo.pairwise_distance(mine, a, b) == phylo.pairwise_distance(want, a, b)


def test_wide_rules(hb):
    base = dict(rows=2, cols=2, n=32, policy="tilted", bits=1, words=4)
    for bad in [dict(base, mode="async"), dict(base, mode="buffered"),
                dict(base, kernel=hb.KERNEL_RESIDENT)]:
        with pytest.raises(hb.HsgaError) as e:
            hb.Grid(**bad)
        assert e.value.status == UNSUPPORTED
    with hb.Grid(**base) as g:
        with pytest.raises(hb.HsgaError) as e:
            hb.hsga_set_fossil_sampling(g.handle, 10, 2, 10)
        assert e.value.status == UNSUPPORTED
    with hb.Batch() as b:
        with pytest.raises(hb.HsgaError) as e:
            b.add(10, **base)
        assert e.value.status == UNSUPPORTED
