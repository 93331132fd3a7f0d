"""GPU trie reconstruction against the oracle's reconstruction.

Trees are compared canonically: a rooted tree with node times is determined
by the multiset of (node time, set of samples below the node), which does
not depend on node numbering.  Inputs: surfaces from oracle runs (many
duplicates, every policy, differentia widths 1-8, temporal coarsening),
random surfaces, degenerate samples (one genome, identical genomes, no
deposition yet), and a 200,000-genome sample of a 16.8M-agent GPU run
(pairwise ancestor times, branch lengths and node counts against the oracle).
"""
import numpy as np
import pytest

from oracle import phylo

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_10861_gb300 import _build, binding
    _build.build()
    return binding


def canonical(parent, time, leaf_of_sample):
    parent = np.asarray(parent)
    n = len(parent)
    sample_of = {int(v): i for i, v in enumerate(leaf_of_sample)}
    below = [[] for _ in range(n)]
    for v in range(n):
        if v in sample_of:
            u = v
            s = sample_of[v]
            while u >= 0:
                below[u].append(s)
                u = int(parent[u])
    return sorted((int(time[v]), tuple(sorted(below[v]))) for v in range(n))


def check_valid(parent, time, leaf, k, T):
    n = len(parent)
    assert parent[0] == -1 and time[0] == -1 and n <= 2 * k + 1
    assert sorted(leaf.tolist()) == list(range(n - k, n))
    kids = np.bincount(parent[1:], minlength=n)
    internal = np.arange(1, n - k)
    assert (kids[internal] >= 2).all()                     # collapsed: no unifurcations
    assert (time[1:] >= time[parent[1:]]).all()            # times never fall away from the root
    assert (time[n - k:] == T).all()


RUNS = [
    dict(policy=0, bits=1, W=2, G=700, coarsen=1),
    dict(policy=1, bits=1, W=2, G=900, coarsen=1),
    dict(policy=2, bits=2, W=2, G=300, coarsen=1),
    dict(policy=5, bits=2, W=2, G=500, coarsen=1),
    dict(policy=3, bits=4, W=2, G=50, coarsen=1),
    dict(policy=1, bits=8, W=1, G=400, coarsen=1),
    dict(policy=0, bits=1, W=2, G=600, coarsen=3),
]


@pytest.mark.parametrize("case", range(len(RUNS)))
def test_matches_oracle_on_ga_surfaces(hb, orc, case):
    r = RUNS[case]
    c = orc.Config(rows=6, cols=6, n=32, tournament=2, policy=r["policy"], bits=r["bits"],
                   W=r["W"], interval=1, p_ben=0.01, seed=40 + case, coarsen=r["coarsen"])
    _, surf, _ = orc.run(c, generations=r["G"])
    want = phylo.reconstruct(surf, c.policy, c.bits, c.W, r["G"], r["coarsen"])
    parent, time, leaf = hb.hsga_reconstruct(surf, c.policy, c.bits, c.W, r["G"], r["coarsen"])
    check_valid(parent, time, leaf, len(surf), r["G"])
    assert canonical(parent, time, leaf) == canonical(want.parent, want.time,
                                                      want.leaf_of_sample)


def test_matches_oracle_on_random_surfaces(hb):
    rng = np.random.default_rng(3)
    surf = rng.integers(0, 2**63, 3000, dtype=np.uint64) << np.uint64(1)
    surf[100:200] = surf[0]                                 # a block of identical genomes
    for policy, bits, W, T in [(1, 1, 2, 5000), (0, 2, 2, 123), (2, 4, 1, 77)]:
        want = phylo.reconstruct(surf, policy, bits, W, T)
        parent, time, leaf = hb.hsga_reconstruct(surf, policy, bits, W, T)
        check_valid(parent, time, leaf, len(surf), T)
        assert canonical(parent, time, leaf) == canonical(want.parent, want.time,
                                                          want.leaf_of_sample)


@pytest.mark.parametrize("surf,T", [
    (np.array([12345], np.uint64), 100),                   # one genome
    (np.array([7, 7, 7, 7], np.uint64), 100),              # identical genomes
    (np.array([1, 2, 3], np.uint64), 0),                   # nothing deposited yet
    (np.array([0, 2**63], np.uint64), 1),                  # one deposition
])
def test_degenerate_samples(hb, surf, T):
    want = phylo.reconstruct(surf, 0, 1, 2, T)
    parent, time, leaf = hb.hsga_reconstruct(surf, 0, 1, 2, T)
    assert canonical(parent, time, leaf) == canonical(want.parent, want.time,
                                                      want.leaf_of_sample)


def test_rejects_bad_arguments(hb):
    with pytest.raises(hb.HsgaError):
        hb.hsga_reconstruct(np.zeros(0, np.uint64), 0, 1, 2, 10)
    with pytest.raises(hb.HsgaError):
        hb.hsga_reconstruct(np.zeros(4, np.uint64), "none", 1, 2, 10)
    with pytest.raises(hb.HsgaError):
        hb.hsga_reconstruct(np.zeros(4, np.uint64), 0, 3, 2, 10)


def test_large_sample_from_the_wafer_grid(hb):
    G, k = 300, 200_000
    with hb.Grid(rows=512, cols=1024, n=32, tournament=2, policy="tilted", bits=1, W=2,
                 p_ben=1e-3, seed=1) as g:
        g.run(G)
        _, s = g.population()
    pick = np.random.default_rng(0).choice(len(s), size=k, replace=False)
    surf = s[pick]
    parent, time, leaf = hb.hsga_reconstruct(surf, 1, 1, 2, G)
    check_valid(parent, time, leaf, k, G)
    want = phylo.reconstruct(surf, 1, 1, 2, G)
    assert len(parent) == want.n_nodes
    assert phylo.sum_branch_length(phylo.Tree(parent, time, leaf)) == \
        phylo.sum_branch_length(want)
    rng = np.random.default_rng(1)
    mine = phylo.Tree(parent, time, leaf)
    for _ in range(300):
        a, b = (int(v) for v in rng.choice(k, size=2, replace=False))
        assert phylo.pairwise_distance(mine, a, b) == phylo.pairwise_distance(want, a, b)
