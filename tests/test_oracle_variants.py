"""Pins for the surface variants the paper suggests ("Distributed
Phylogenetic Tracking": a hybrid giving half the annotation space to each of
steady and tilted; "Surface Algorithm Benchmark": coarsening the temporal
resolution by annotating only every k-th generation)."""
import numpy as np
import pytest
from scipy import stats

from oracle import phylo
from paper_2404_10861_gb300 import inputs

HYBRID = 5


@pytest.mark.parametrize("S,W", [(64, 2), (32, 2), (16, 2), (64, 4)])
def test_hybrid_halves_are_steady_and_tilted(orc, S, W):
    for T in list(range(0, 300)) + [1000, 4097, 65536]:
        got = orc.lookup(HYBRID, S, W, T)
        assert list(got[:S // 2]) == list(orc.lookup(orc.STEADY, S // 2, W, T))
        assert list(got[S // 2:]) == list(orc.lookup(orc.TILTED, S // 2, W, T))


@pytest.mark.parametrize("T", [77, 79])
def test_hybrid_deposits_two_independent_differentiae(orc, T):
    """Hybrid deposition T writes the steady half (sites [0, S/2); it may
    discard, as at T = 77) and the tilted half (sites [S/2, S)): the steady
    field from the low b bits of word 3 of the child's replication block, the
    tilted one from the b bits at bit 16 of it.  Nothing else changes, and the
    two values are independent and uniform."""
    c = orc.Config(rows=16, cols=16, n=32, policy=HYBRID, bits=2, interval=0, seed=3)
    trait, surf = inputs.small_trait_population(c.agents, seed=2)
    S, half = 32, 16
    _, child, par = orc.run(c, trait, surf, G0=T, generations=1, track_parents=True)
    parent = surf[par[0].astype(np.int64)]
    sa = orc.site(orc.STEADY, half, 2, T)               # == half: discarded
    sb = half + orc.site(orc.TILTED, half, 2, T)
    assert (sa == half) == (T == 77)
    mask = np.uint64(3 << (2 * sb))
    if sa < half:
        mask |= np.uint64(3 << (2 * sa))
    assert np.all(((child ^ parent) & ~mask) == 0)
    vb = ((child >> np.uint64(2 * sb)) & np.uint64(3)).astype(np.int64)
    assert stats.chisquare(np.bincount(vb, minlength=4)).pvalue > 1e-4      # uniform
    if sa < half:
        va = ((child >> np.uint64(2 * sa)) & np.uint64(3)).astype(np.int64)
        table = np.zeros((4, 4))
        np.add.at(table, (va, vb), 1)
        assert stats.chi2_contingency(table).pvalue > 1e-4                  # independent
    key = (c.seed & 0xFFFFFFFF, c.seed >> 32)
    for a in range(0, c.agents, 7):
        i, j = divmod(a, c.n)
        w3 = int(orc.philox4x32(key, (j, i, T, 1))[3])
        assert int(vb[a]) == (w3 >> 16) & 3, a
        if sa < half:
            assert int(va[a]) == w3 & 3, a


@pytest.mark.parametrize("k", [2, 3, 8])
def test_coarsening_deposits_every_kth_generation(orc, k):
    c = orc.Config(rows=8, cols=8, n=16, policy=orc.TILTED, bits=1, interval=0, seed=4,
                   coarsen=k)
    trait, surf = inputs.random_population(c.agents, seed=k, trait_max=3)
    for G in range(0, 3 * k + 1):
        _, child, par = orc.run(c, trait, surf, G0=G, generations=1, track_parents=True)
        parent = surf[par[0].astype(np.int64)]
        changed = child ^ parent
        if G % k:
            assert not changed.any()
        else:
            s_ = orc.site(orc.TILTED, 64, 2, G // k)
            assert np.all((changed & ~np.uint64(1 << s_)) == 0)
            assert changed.any()


def test_coarsened_ancestry_bounds(orc):
    """With coarsening the retained times are generations t k; mismatches
    still only occur at or after the true split."""
    k = 4
    c = orc.Config(rows=4, cols=4, n=16, policy=orc.TILTED, bits=1, seed=8, coarsen=k)
    G = 600
    _, surf, par = orc.run(c, generations=G, track_parents=True)
    order, times = phylo.retained_order(c.policy, 64, 2, G, coarsen=k)
    assert np.all(times % k == 0)
    D = phylo.differentiae(surf, 1)[:, order]
    rng = np.random.default_rng(0)
    for _ in range(400):
        x, y = rng.choice(c.agents, size=2, replace=False)
        d_true = phylo.true_mrca_generation(par, int(x), int(y))
        assert np.array_equal(D[x, times < d_true], D[y, times < d_true])


@pytest.mark.parametrize("policy,bits,words,W", [(1, 1, 4, 2), (0, 2, 2, 2), (2, 16, 4, 1),
                                                 (5, 4, 2, 2), (3, 8, 4, 2)])
def test_wide_surfaces_hold_their_ancestors_draws(orc, policy, bits, words, W):
    """Surfaces of several 64-bit words (up to the 256-bit field): every
    retained differentia is the value its own ancestor drew when it was
    deposited (word 3 of the Philox block of the child on the lineage, bits
    16.. for the hybrid policy's tilted half), found by walking the pedigree
    and recomputing the draw; selection never depends on the surface, so
    traits equal those of the one-word run."""
    from oracle import phylo
    c = orc.Config(rows=3, cols=3, n=8, tournament=2, policy=policy, bits=bits, W=W,
                   interval=1, p_ben=0.05, seed=21, words=words)
    G = 300
    trait, surf, par = orc.run(c, generations=G, track_parents=True)
    narrow = orc.Config(**{**c.__dict__, "words": 1, "bits": 1, "W": 2, "policy": 0})
    t1, _, _ = orc.run(narrow, generations=G)
    assert np.array_equal(trait, t1)
    S = 64 * words // bits
    times = orc.lookup(policy, S, W, G)
    D = phylo.differentiae(surf, bits, words)
    key = (c.seed & 0xFFFFFFFF, c.seed >> 32)
    half = S // 2
    rng = np.random.default_rng(0)
    checked = 0
    for x in rng.choice(c.agents, size=12, replace=False):
        line = phylo.lineage(par, int(x))
        for site, t in enumerate(times):
            if t < 0:
                continue
            child = int(line[t + 1])                     # the lineage's child born at t
            w3 = int(orc.philox4x32(key, (child % c.n, child // c.n, int(t), 1))[3])
            second = policy == 5 and site >= half
            want = ((w3 >> 16) if second else w3) & ((1 << bits) - 1)
            assert D[x, site] == want, (x, site, t)
            checked += 1
    assert checked >= 12 * 8
