"""Pins for the oracle's genetic-algorithm steps (arXiv 2404.10861, section
"Asynchronous Island-model Genetic Algorithm"), each against something other
than the oracle itself: closed forms of tournament selection and of the
Wright-Fisher coalescent, binomial mutation counts, the uniform random
von-Neumann-neighbour migration, exact bit-level statements about the
deposition, and the hereditary-stratigraphy ancestry bounds of section
"Distributed Phylogenetic Tracking" checked against perfect pedigrees.
"""
import numpy as np
import pytest
from scipy import stats

from paper_2404_10861_gb300 import inputs


def cfg(orc, **kw):
    base = dict(rows=4, cols=4, n=32, tournament=2, policy=orc.STEADY, bits=1,
                W=2, interval=1, p_ben=0.0, p_del=0.0, seed=1)
    base.update(kw)
    return orc.Config(**base)


# ---------------------------------------------------------------- a4 ---

@pytest.mark.parametrize("t", [1, 2, 3, 5, 6])
def test_tournament_matches_closed_form(orc, t):
    """Tournament of t candidates drawn with replacement among n distinct
    fitnesses: the rank-r parent (0 = least fit) wins with probability
    ((r+1)^t - r^t) / n^t."""
    c = cfg(orc, rows=16, cols=16, n=16, tournament=t, interval=0, seed=11 + t)
    trait, surf = inputs.permutation_traits(c.islands, c.n, seed=t)
    _, _, par = orc.run(c, trait, surf, G0=5, generations=1, track_parents=True)
    parent_rank = trait[par[0].astype(np.int64)]
    counts = np.bincount(parent_rank, minlength=c.n)
    r = np.arange(c.n, dtype=np.float64)
    p = ((r + 1) ** t - r ** t) / c.n ** t
    keep = p * counts.sum() >= 5
    exp = p[keep] * counts.sum()
    obs = counts[keep]
    chi = ((obs - exp) ** 2 / exp).sum()
    assert stats.chi2.sf(chi, keep.sum() - 1) > 1e-4
    # isolated islands: a parent is always a member of the child's island
    assert np.all(par[0] // c.n == np.arange(c.agents) // c.n)


def test_neutral_selection_is_wright_fisher(orc):
    """All fitnesses tied: every child picks a uniform parent, so two children
    of one island share a parent with probability 1/n (the Wright-Fisher
    coalescence rate)."""
    c = cfg(orc, rows=32, cols=32, n=8, interval=0, seed=5)
    _, _, par = orc.run(c, generations=3, track_parents=True)
    shared = total = 0
    for g in range(3):
        p = par[g].reshape(c.islands, c.n)
        eq = p[:, :, None] == p[:, None, :]
        iu = np.triu_indices(c.n, 1)
        shared += eq[:, iu[0], iu[1]].sum()
        total += c.islands * len(iu[0])
    p_hat = shared / total
    # pairs within an island are correlated; 6 sigma of the binomial is lax
    assert abs(p_hat - 1 / c.n) < 6 * np.sqrt((1 / c.n) * (1 - 1 / c.n) / total) * 3


@pytest.mark.parametrize("t", [2, 5, 7])
def test_tournament_parent_is_the_fitter_candidate_first_on_ties(orc, t):
    """Step a4 per child j of island i at generation G: candidate 0 and 1 are
    floor(w n / 2^32) of words 0 and 1 of Philox(seed; j, i, G, 1), candidate
    c >= 2 of word (c - 2) mod 4 of Philox(seed; j, i, G, 2 + (c - 2) // 4);
    a later candidate replaces the best only if strictly fitter.  Few trait
    levels make ties between distinct candidates common, which the marginal
    parent law cannot show (it is the same whichever candidate keeps ties),
    and words reused across blocks would keep that law too."""
    c = cfg(orc, rows=4, cols=4, n=16, tournament=t, interval=0, seed=19 + t)
    key = (c.seed & 0xFFFFFFFF, c.seed >> 32)
    trait, surf = inputs.small_trait_population(c.agents, seed=4)
    G = 9
    _, _, par = orc.run(c, trait, surf, G0=G, generations=1, track_parents=True)
    ties = 0
    for a in range(c.agents):
        i, j = divmod(a, c.n)
        w = orc.philox4x32(key, (j, i, G, 1))
        words = [int(w[0]), int(w[1])]
        for b in range((t - 2 + 3) // 4):
            words += [int(x) for x in orc.philox4x32(key, (j, i, G, 2 + b))]
        cands = [(x * c.n) >> 32 for x in words[:t]]
        best = cands[0]
        for cand in cands[1:]:
            fb, fc = trait[i * c.n + best], trait[i * c.n + cand]
            ties += int(cand != best and fc == fb)
            if fc > fb:
                best = cand
        assert int(par[0][a]) == i * c.n + best, a
    assert ties > c.agents // 10


def test_neutral_traits_stay_zero(orc):
    c = cfg(orc, rows=4, cols=4, n=32)
    trait, _, _ = orc.run(c, generations=500)
    assert not trait.any()


# ---------------------------------------------------------------- a5 ---

def test_mutation_rates_binomial(orc):
    c = cfg(orc, rows=32, cols=32, n=32, interval=0, p_ben=0.1, p_del=0.2, seed=9)
    trait = np.full(c.agents, 1000, dtype=np.uint32)
    surf = np.zeros(c.agents, dtype=np.uint64)
    out, _, _ = orc.run(c, trait, surf, G0=0, generations=1)
    N = c.agents
    for value, p in ((1001, 0.1), (999, 0.2), (1000, 0.7)):
        k = int((out == value).sum())
        assert abs(k - N * p) < 5 * np.sqrt(N * p * (1 - p)), (value, k)


def test_mutation_saturates(orc):
    c = cfg(orc, rows=2, cols=2, n=16, interval=0, p_ben=1.0)
    top = np.full(c.agents, 0xFFFFFFFF, dtype=np.uint32)
    out, _, _ = orc.run(c, top, np.zeros(c.agents, np.uint64), generations=3)
    assert np.all(out == 0xFFFFFFFF)
    c = cfg(orc, rows=2, cols=2, n=16, interval=0, p_del=1.0)
    out, _, _ = orc.run(c, np.zeros(c.agents, np.uint32), np.zeros(c.agents, np.uint64),
                        generations=3)
    assert np.all(out == 0)
    c = cfg(orc, rows=2, cols=2, n=16, interval=0, p_ben=1.0)
    out, _, _ = orc.run(c, np.zeros(c.agents, np.uint32), np.zeros(c.agents, np.uint64),
                        generations=7)
    assert np.all(out == 7)


# ---------------------------------------------------------------- a6 ---

@pytest.mark.parametrize("policy,bits", [(0, 1), (1, 2), (2, 4), (3, 8), (1, 1)])
def test_deposit_touches_only_the_site(orc, policy, bits):
    """A child's surface equals its parent's except in bits
    [site*b, site*b+b) of the site chosen for T, whose value is uniform."""
    c = cfg(orc, rows=16, cols=16, n=32, policy=policy, bits=bits, interval=0, seed=4)
    S = 64 // bits
    trait, surf = inputs.small_trait_population(c.agents, seed=policy * 10 + bits)
    for T in (0, 5, S, 3 * S + 1, 1000):
        _, child, par = orc.run(c, trait, surf, G0=T, generations=1, track_parents=True)
        parent_surf = surf[par[0].astype(np.int64)]
        site = orc.site(policy, S, c.W, T)
        mask = np.uint64(0) if site == S else np.uint64(((1 << bits) - 1) << (site * bits))
        assert np.all(((child ^ parent_surf) & ~mask) == 0)
        if site < S:
            vals = ((child >> np.uint64(site * bits)) & np.uint64((1 << bits) - 1)).astype(np.int64)
            counts = np.bincount(vals, minlength=1 << bits)
            assert stats.chisquare(counts).pvalue > 1e-4


def test_child_takes_word_2_for_mutation_and_word_3_for_deposit(orc):
    """Per child j of island i at generation G, with (w0..w3) =
    Philox(seed; j, i, G, 1): the trait is the parent's, raised by one when
    w2 < floor(p_ben 2^32), else lowered by one when w2 < floor(p_ben 2^32) +
    floor(p_del 2^32) (saturating), and the surface is the parent's with the
    generation's site set to the low b bits of w3.  Rates and uniformity
    alone would not show which word feeds which step."""
    c = cfg(orc, rows=4, cols=4, n=16, policy=orc.TILTED, bits=2, interval=0,
            p_ben=0.3, p_del=0.3, seed=23)
    key = (c.seed & 0xFFFFFFFF, c.seed >> 32)
    trait, surf = inputs.small_trait_population(c.agents, seed=6)
    G = 21
    t2, s2, par = orc.run(c, trait, surf, G0=G, generations=1, track_parents=True)
    tb, td = int(0.3 * 2**32), int(0.3 * 2**32)
    site = orc.site(orc.TILTED, 32, c.W, G)
    mask = 3 << (2 * site)
    for a in range(c.agents):
        i, j = divmod(a, c.n)
        w = orc.philox4x32(key, (j, i, G, 1))
        p = int(par[0][a])
        want_t = int(trait[p])
        if int(w[2]) < tb:
            want_t = min(want_t + 1, 2**32 - 1)
        elif int(w[2]) < tb + td:
            want_t = max(want_t - 1, 0)
        want_s = (int(surf[p]) & ~mask) | ((int(w[3]) & 3) << (2 * site))
        assert int(t2[a]) == want_t and int(s2[a]) == want_s, a


def test_untracked_leaves_surface_alone(orc):
    c = cfg(orc, policy=orc.NONE, p_ben=0.05)
    trait, surf = inputs.random_population(c.agents, seed=3, trait_max=10)
    _, s2, par = orc.run(c, trait, surf, generations=1, track_parents=True)
    assert np.all(s2 == surf[par[0].astype(np.int64)])


# ------------------------------------------------------------- a1/a2 ---

def test_migration_copies_from_von_neumann_neighbours(orc):
    c = cfg(orc, rows=24, cols=32, n=32, seed=21)
    trait = np.arange(c.agents, dtype=np.uint32)          # unique markers
    surf = np.zeros(c.agents, dtype=np.uint64)
    t2, _ = orc.migrate(c, trait, surf, G=17)
    home = t2 // c.n
    isl = np.arange(c.agents) // c.n
    foreign = home != isl
    nb = np.array([[orc.neighbour(c, i, d) for d in range(4)] for i in range(c.islands)])
    # every immigrant comes from one of the four neighbours
    assert np.all((nb[isl[foreign]] == home[foreign][:, None]).any(axis=1))
    # ... the one whose emigrant was aimed at this island: direction w1 >> 30
    # of Philox(seed; 0xFFFFFFFF, source, G, 0) points from the source here
    key = (c.seed & 0xFFFFFFFF, c.seed >> 32)
    blocks = np.array([orc.philox4x32(key, (0xFFFFFFFF, i, 17, 0)) for i in range(c.islands)],
                      dtype=np.uint64)
    aim = (blocks[:, 1] >> np.uint64(30)).astype(np.int64)
    assert np.all(nb[home[foreign], aim[home[foreign]]] == isl[foreign])
    # ... and it is that source's member at slot floor(w0 n / 2^32)
    eslot = ((blocks[:, 0] * np.uint64(c.n)) >> np.uint64(32)).astype(np.int64)
    assert np.all(t2[foreign] % c.n == eslot[home[foreign]])
    # ... landing, from direction d, at slot floor(v_d n / 2^32) of the
    # receiver's Philox(seed; 0xFFFFFFFE, island, G, 0)
    place = np.array([orc.philox4x32(key, (0xFFFFFFFE, i, 17, 0)) for i in range(c.islands)],
                     dtype=np.uint64)
    recv = isl[foreign]
    d_in = (nb[recv] == home[foreign][:, None]).argmax(axis=1)
    pslot = ((place[recv, d_in] * np.uint64(c.n)) >> np.uint64(32)).astype(np.int64)
    assert np.all(np.nonzero(foreign)[0] % c.n == pslot)
    # an emigrant lands at most once (a copy is sent, not broadcast)
    vals, cnt = np.unique(t2[foreign], return_counts=True)
    assert cnt.max() == 1
    # the sender keeps its own copy unless an immigrant landed on that slot
    src_island = home[foreign]
    for v, si in zip(t2[foreign][:200], src_island[:200]):
        if v not in t2[si * c.n:(si + 1) * c.n]:
            assert foreign[si * c.n + (v % c.n)]
    # arrivals per island ~ Binomial(4, 1/4): each neighbour aims at one of
    # its four neighbours uniformly (slot collisions, prob ~1/n, aside)
    per_island = np.bincount(isl[foreign], minlength=c.islands)
    hist = np.bincount(per_island, minlength=5)[:5]
    p = stats.binom.pmf(np.arange(5), 4, 0.25)
    exp = p * c.islands
    keep = exp >= 5
    obs = hist[keep].astype(float)
    obs[-1] += hist[~keep].sum()
    chi = ((obs - exp[keep]) ** 2 / exp[keep]).sum()
    assert stats.chi2.sf(chi, keep.sum() - 1) > 1e-4
    # total arrivals: every island emits exactly one emigrant
    assert abs(foreign.sum() - c.islands) <= c.islands * 4 / c.n + 5 * np.sqrt(c.islands)


@pytest.mark.parametrize("rows,cols", [(1, 1), (1, 5), (2, 2), (2, 3), (3, 1)])
def test_degenerate_tori(orc, rows, cols):
    """Neighbours may coincide or be the island itself: each emigrant still
    lands exactly once, so each island count of markers changes by the
    arrivals only."""
    c = cfg(orc, rows=rows, cols=cols, n=8, seed=rows * 10 + cols)
    trait = np.arange(c.agents, dtype=np.uint32)
    for G in range(40):
        t2, _ = orc.migrate(c, trait, np.zeros(c.agents, np.uint64), G=G)
        changed = (t2 != trait).sum()
        assert changed <= c.islands
        # the multiset gains duplicates only from emigrant copies
        assert len(np.unique(t2)) >= c.agents - c.islands


def test_later_direction_wins_a_shared_slot(orc):
    """Step a2's order on a 1x2 torus with one agent per island: an island's
    N and S neighbours are itself and its E and W neighbours the other
    island, so its own emigrant and the other's can both land on its only
    slot.  Directions land in the order N, E, S, W, a later arrival
    overwrites an earlier one, and both emigrants are chosen before either
    lands; the generations scanned include both orders of arrival."""
    c = cfg(orc, rows=1, cols=2, n=1, seed=77)
    key = (c.seed & 0xFFFFFFFF, c.seed >> 32)
    trait = np.array([100, 200], np.uint32)
    orders = set()
    for G in range(400):
        sent = [int(orc.philox4x32(key, (0xFFFFFFFF, i, G, 0))[1]) >> 30 for i in range(2)]
        t2, _ = orc.migrate(c, trait, np.zeros(2, np.uint64), G)
        for i in range(2):
            src = [i, 1 - i, i, 1 - i]            # the N, E, S, W neighbours of island i
            arrivals = [a for a in range(4) if sent[src[a]] == (a + 2) % 4]
            want = trait[src[arrivals[-1]]] if arrivals else trait[i]
            assert t2[i] == want, (G, i, sent)
            if len(arrivals) == 2:
                orders.add(tuple(src[a] == i for a in arrivals))
    assert orders == {(True, False), (False, True)}


def test_explicit_migrate_then_premigrated_run_equals_run(orc):
    c = cfg(orc, rows=5, cols=7, n=12, p_ben=0.01, policy=orc.TILTED, bits=2, seed=3)
    trait, surf = inputs.small_trait_population(c.agents, seed=8)
    a = orc.run(c, trait, surf, G0=40, generations=9)
    t1, s1 = orc.migrate(c, trait, surf, G=40)
    b = orc.run(c, t1, s1, G0=40, generations=9, premigrated=True)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_migration_interval(orc):
    c = cfg(orc, rows=4, cols=4, n=8, interval=3, seed=2)
    trait = np.arange(c.agents, dtype=np.uint32)
    _, _, par = orc.run(c, trait, np.zeros(c.agents, np.uint64), generations=6,
                        track_parents=True)
    isl = np.arange(c.agents) // c.n
    for g in range(6):
        crosses = (par[g].astype(np.int64) // c.n != isl).any()
        assert crosses == (g % 3 == 0)


# ------------------------------------------------------------ cone ---

def test_cone_equals_full_grid(orc):
    c = cfg(orc, rows=11, cols=13, n=16, p_ben=0.05, p_del=0.05, policy=orc.TILTED,
            tournament=3, seed=77)
    full_t, full_s, _ = orc.run(c, generations=5)
    for r, col in ((0, 0), (5, 6), (10, 12), (3, 11)):
        t, s = orc.run_cone(c, r, col, generations=5)
        i = r * c.cols + col
        assert np.array_equal(t, full_t[i * c.n:(i + 1) * c.n])
        assert np.array_equal(s, full_s[i * c.n:(i + 1) * c.n])


# ---------------------------------------------------------------- a7 ---

def test_sample_follows_its_draws(orc):
    """Step a7 per sample: the j-th pick swaps position j with position
    j + floor(w0 (I - j) / 2^32) of the island list, w0 word 0 of
    Philox(seed; j, 0xFFFFFFFF, G, 3), and the genome taken from island i is
    its member at floor(w0 n / 2^32) of Philox(seed; 0xFFFFFFFD, i, G, 0)."""
    c = cfg(orc, rows=6, cols=7, n=12, seed=29)
    key = (c.seed & 0xFFFFFFFF, c.seed >> 32)
    trait = np.arange(c.agents, dtype=np.uint32)
    surf = np.zeros(c.agents, dtype=np.uint64)
    I = c.islands
    for G, k in ((0, 1), (5, 17), (77, I)):
        w, where = orc.sample(c, trait, surf, G, k)
        perm = list(range(I))
        for j in range(k):
            d = int(orc.philox4x32(key, (j, 0xFFFFFFFF, G, 3))[0])
            r = j + ((d * (I - j)) >> 32)
            perm[j], perm[r] = perm[r], perm[j]
        for j in range(k):
            isl = perm[j]
            slot = (int(orc.philox4x32(key, (0xFFFFFFFD, isl, G, 0))[0]) * c.n) >> 32
            assert (int(where[j, 0]), int(where[j, 1])) == (isl, slot), (G, j)
            assert int(w[j, 0]) == isl * c.n + slot


def test_sample_distinct_and_uniform(orc):
    c = cfg(orc, rows=2, cols=2, n=5, seed=13)
    trait = np.arange(c.agents, dtype=np.uint32)
    surf = np.zeros(c.agents, dtype=np.uint64)
    pairs, slots = [], []
    for G in range(2400):
        w, where = orc.sample(c, trait, surf, G, 2)
        assert where[0, 0] != where[1, 0]
        assert np.all(w[:, 0] == where[:, 0] * c.n + where[:, 1])
        assert np.all(w[:, 3] == G)
        pairs.append(where[0, 0] * 4 + where[1, 0])
        slots.extend(where[:, 1])
    counts = np.bincount(pairs, minlength=16)
    ordered = [a * 4 + b for a in range(4) for b in range(4) if a != b]
    assert stats.chisquare(counts[ordered]).pvalue > 1e-4
    assert stats.chisquare(np.bincount(slots, minlength=c.n)).pvalue > 1e-4
    with pytest.raises(ValueError):
        orc.sample(c, trait, surf, 0, 5)
    w, _ = orc.sample(c, trait, surf, 0, 4)
    assert sorted(w[:, 0] // c.n) == [0, 1, 2, 3]
