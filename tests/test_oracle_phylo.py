"""Pins for the oracle's ancestry bounds, reconstruction and phylometrics.

* Hereditary stratigraphy (arXiv 2404.10861, "Distributed Phylogenetic
  Tracking"): differentiae deposited before two lineages split are shared,
  so a mismatch can only occur at or after the split; later differentiae are
  independent draws, so at the first retained time after the split two
  b-bit differentiae collide with probability 2^-b (the spurious-relatedness
  artifact the clade trial notes for 1-bit differentiae).  Checked against
  perfect pedigrees.
* Reconstruction and phylometrics: hand-built trees with known values, the
  brute-force pairwise distance, and the identity that fair-proportion
  evolutionary distinctiveness sums to the total branch length.
* The on-hardware trial's outcome: without adaptation, sum branch length and
  mean pairwise distance are larger than with it (one-sided Mann-Whitney U,
  the paper's test).
"""
import numpy as np
import pytest
from scipy import stats

from oracle import phylo


def test_pedigree_bounds_and_collision_rate(orc):
    rows = cols = 4
    n, bits, G = 32, 1, 2000
    c = orc.Config(rows=rows, cols=cols, n=n, tournament=2, policy=orc.STEADY,
                   bits=bits, W=2, interval=1, seed=1)
    trait, surf, par = orc.run(c, generations=G, track_parents=True)
    order, times = phylo.retained_order(c.policy, c.S, c.W, G)
    D = phylo.differentiae(surf, bits)[:, order]
    rng = np.random.default_rng(0)
    first_after = {}
    for _ in range(3000):
        x, y = rng.choice(c.agents, size=2, replace=False)
        d_true = phylo.true_mrca_generation(par, int(x), int(y))
        before = times < d_true
        assert np.array_equal(D[x, before], D[y, before])       # shared history
        t_prev, t_star = phylo.mrca_bounds(D[x], D[y], times)
        if t_star is not None:
            assert t_star >= d_true                             # hard bound
        _record_first_after(first_after, par, D, times, x, y, d_true)
    _assert_collision_rate(first_after, 2.0 ** -bits)


def _record_first_after(acc, par, D, times, x, y, d_true):
    """Remember the comparison at the first retained time after the split,
    keyed by the two agents that deposited those differentiae, so that pairs
    sharing both lineages there count once (their outcomes are identical)."""
    after = np.nonzero(times >= d_true)[0]
    if not len(after):
        return
    t1 = int(times[after[0]])
    ax = int(phylo.lineage(par, int(x))[t1 + 1])
    ay = int(phylo.lineage(par, int(y))[t1 + 1])
    assert ax != ay
    acc[(t1, min(ax, ay), max(ax, ay))] = int(D[x, after[0]] == D[y, after[0]])


def _assert_collision_rate(acc, p):
    # indicators [X_a == X_b] of iid uniform values are pairwise independent,
    # so the count of collisions has binomial variance
    trials, hits = len(acc), sum(acc.values())
    assert trials >= 60
    assert abs(hits - trials * p) < 4 * np.sqrt(trials * p * (1 - p)), (hits, trials)


def test_two_bit_collision_rate(orc):
    c = orc.Config(rows=4, cols=8, n=16, tournament=2, policy=orc.TILTED, bits=2,
                   W=2, interval=1, p_ben=0.002, seed=6)
    G = 600
    _, surf, par = orc.run(c, generations=G, track_parents=True)
    order, times = phylo.retained_order(c.policy, c.S, c.W, G)
    D = phylo.differentiae(surf, 2)[:, order]
    rng = np.random.default_rng(1)
    first_after = {}
    for _ in range(3000):
        x, y = rng.choice(c.agents, size=2, replace=False)
        d_true = phylo.true_mrca_generation(par, int(x), int(y))
        assert np.array_equal(D[x, times < d_true], D[y, times < d_true])
        _record_first_after(first_after, par, D, times, x, y, d_true)
    _assert_collision_rate(first_after, 0.25)


def _surfaces_from_sequences(seqs, order, bits):
    """Build surfaces whose differentiae, in retained-time order, are seqs."""
    out = np.zeros(len(seqs), dtype=np.uint64)
    for i, s in enumerate(seqs):
        v = 0
        for site, d in zip(order, s):
            v |= int(d) << (int(site) * bits)
        out[i] = v
    return out


def test_reconstruct_known_tree(orc):
    # steady, S=8, after T=8 depositions the retained times are 0..7 (site = time)
    T, bits = 8, 8
    order, times = phylo.retained_order(orc.STEADY, 8, 2, T)
    assert list(times) == list(range(8))
    seqs = [[1, 1, 1, 1, 1, 1, 1, 1],
            [1, 1, 1, 1, 1, 1, 1, 2],   # splits from 0 at time 7
            [1, 1, 1, 2, 2, 2, 2, 2],   # splits from {0,1} at time 3
            [3, 3, 3, 3, 3, 3, 3, 3]]   # splits from all at time 0
    surf = _surfaces_from_sequences(seqs, order, bits)
    tree = phylo.reconstruct(surf, orc.STEADY, bits, 2, T)
    # pairwise distance = 2 * (T - last shared time)
    want = {(0, 1): 2 * (8 - 6), (0, 2): 2 * (8 - 2), (1, 2): 2 * (8 - 2),
            (0, 3): 2 * (8 - (-1)), (1, 3): 18, (2, 3): 18}
    for (a, b), d in want.items():
        assert phylo.pairwise_distance(tree, a, b) == d
    m = phylo.phylometrics(tree)
    # edges: root(-1)->A(time 2)=3, A->B(time 6)=4, B->leaf0=2, B->leaf1=2,
    # A->leaf2=6, root->leaf3=9  => 26
    assert m["sum_branch_length"] == 26
    assert m["mean_pairwise_distance"] == pytest.approx(sum(want.values()) / 6)
    # internal nodes root, A, B; leaf depths 3,3,2,1
    assert m["sackin"] == 9
    # root: children A(3 leaves), leaf3(1) -> 2 ; A: B(2), leaf2(1) -> 1 ; B: 1,1 -> 0
    assert m["colless"] == 3
    ed = phylo.evolutionary_distinctiveness(tree)
    assert ed.sum() == pytest.approx(m["sum_branch_length"])
    assert ed[3] == pytest.approx(9.0)


def test_metrics_identities_random_trees(orc):
    rng = np.random.default_rng(4)
    for trial in range(5):
        T = 200
        surf = rng.integers(0, 4, size=40, dtype=np.uint64)   # shallow random
        surf = surf | (rng.integers(0, 2**62, size=40, dtype=np.uint64) << np.uint64(2)) * (trial % 2)
        tree = phylo.reconstruct(surf, orc.TILTED, 1, 2, T)
        m = phylo.phylometrics(tree)
        ed = phylo.evolutionary_distinctiveness(tree)
        assert ed.sum() == pytest.approx(m["sum_branch_length"])
        N = len(surf)
        brute = np.mean([phylo.pairwise_distance(tree, a, b)
                         for a in range(N) for b in range(a + 1, N)])
        assert m["mean_pairwise_distance"] == pytest.approx(brute)


def test_adaptive_vs_neutral_separation(orc):
    """On-hardware trial outcome: neutral phylogenies have larger sum branch
    length and mean pairwise distance than adaptive ones.  Mid-grid surface
    (32 two-bit differentiae, tilted), shrunk to a 16 x 16 torus and 3,000
    generations so the CPU finishes in seconds."""
    res = {True: [], False: []}
    G = 3000
    for adaptive in (True, False):
        for seed in range(1, 5):
            c = orc.Config(rows=16, cols=16, n=32, tournament=2, policy=orc.TILTED,
                           bits=2, W=2, interval=1, p_ben=1e-3 if adaptive else 0.0,
                           seed=seed)
            trait, surf, _ = orc.run(c, generations=G)
            words, _ = orc.sample(c, trait, surf, G, 256)
            s = words[:, 1].astype(np.uint64) | (words[:, 2].astype(np.uint64) << np.uint64(32))
            res[adaptive].append(phylo.phylometrics(phylo.reconstruct(s, c.policy, c.bits, c.W, G)))
    for key in ("sum_branch_length", "mean_pairwise_distance"):
        on = [m[key] for m in res[True]]
        off = [m[key] for m in res[False]]
        assert stats.mannwhitneyu(off, on, alternative="greater").pvalue < 0.05, (key, on, off)


def test_mixed_counts_bound_the_true_mrca(orc):
    # genome a sampled at G1, genome b at G2 > G1 of the same pedigree: every
    # generation both still retain from before their true common ancestry
    # must match, so the first mismatch is never earlier than it
    c = orc.Config(rows=3, cols=3, n=16, tournament=2, policy=orc.TILTED, bits=1, W=2,
                   interval=1, seed=3)
    G1, G2 = 700, 1300
    t1, s1, par1 = orc.run(c, generations=G1, track_parents=True)
    t2, s2, par2 = orc.run(c, trait=t1, surf=s1, G0=G1, generations=G2 - G1,
                           track_parents=True)
    rng = np.random.default_rng(1)
    hits = 0
    for _ in range(400):
        x, y = (int(v) for v in rng.integers(0, c.agents, size=2))
        z = int(phylo.lineage(par2, y)[0])                 # y's ancestor at G1
        d_true = G1 if z == x else phylo.true_mrca_generation(par1, x, z)
        t_prev, t_star = phylo.mrca_bounds_mixed(int(s1[x]), G1, int(s2[y]), G2, c.policy,
                                                 c.bits, c.W)
        assert t_star is None or t_star >= d_true
        hits += t_star is not None
    assert hits > 30


def test_mixed_distance_equals_tree_distance_at_equal_counts(orc):
    c = orc.Config(rows=2, cols=2, n=16, tournament=2, policy=orc.STEADY, bits=1, W=2,
                   interval=1, seed=5)
    G = 900
    _, surf, _ = orc.run(c, generations=G)
    tree = phylo.reconstruct(surf, c.policy, c.bits, c.W, G)
    rng = np.random.default_rng(2)
    for _ in range(100):
        a, b = (int(v) for v in rng.choice(c.agents, size=2, replace=False))
        m, _ = phylo.mrca_bounds_mixed(int(surf[a]), G, int(surf[b]), G, c.policy, c.bits, c.W)
        assert 2 * G - 2 * m == phylo.pairwise_distance(tree, a, b)
