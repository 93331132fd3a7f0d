"""Fossil sampling during a run ("Distributed Phylogenetic Tracking":
genomes extracted during the run keep lineages that later go extinct in the
reconstruction): every fossil record equals the oracle's sampling of the
population at that generation, and fossils keep founding clades that the
end-state population has lost."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_10861_gb300 import _build, binding
    _build.build()
    return binding


@pytest.mark.parametrize("kernel", [1, 2])
def test_fossils_equal_oracle_and_keep_extinct_clades(hb, orc, kernel):
    kw = dict(rows=4, cols=4, n=32, tournament=1, policy="tilted", bits=1, seed=21)
    c = orc.Config(rows=4, cols=4, n=32, tournament=1, policy=orc.TILTED, bits=1, seed=21)
    tags = np.random.default_rng(3).integers(0, 2**16, size=c.agents).astype(np.uint32)
    zero = np.zeros(c.agents, dtype=np.uint64)
    every, k, G_end = 40, 8, 400
    with hb.Grid(kernel=kernel, **kw) as g:
        g.set_population(tags, zero, 0)
        hb.hsga_set_fossil_sampling(g.handle, every, k, capacity=64)
        g.run(150)
        g.run(G_end - 150)
        g.sync()
        words, where = hb.hsga_get_fossils(g.handle, 1000)
        st = g.stats()
        end_t, _ = g.population()
    assert st["fossils"] == 64 and st["fossils_dropped"] == (G_end // every) * k - 64
    t, s, G = tags, zero, 0
    for i in range(64 // k):
        t, s, _ = orc.run(c, t, s, G0=G, generations=every)
        G += every
        ow, owhere = orc.sample(c, t, s, G, k)
        assert np.array_equal(words[i * k:(i + 1) * k], ow)
        assert np.array_equal(where[i * k:(i + 1) * k], owhere)
        assert np.all(words[i * k:(i + 1) * k, 3] == G)
    # founding clades present among fossils but absent from the end state
    assert len(set(words[:, 0]) - set(end_t)) > 0
