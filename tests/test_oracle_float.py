"""Pins for the oracle's float fitness model (the paper's 128-bit genome with a
binary32 fitness word and sign-restricted Gaussian mutation, "Methods ›
Genome Model" and "Results › On-hardware Trial").

* The mutation amount is |N(0, sigma^2)|: a Kolmogorov-Smirnov test against
  scipy's half-normal, its mean against sigma sqrt(2 / pi), beneficial
  amounts never negative and deleterious never positive.
* Selection compares fitness as floats: with negative fitness a comparison
  of the raw words as unsigned integers would pick the least fit.
* The free-running step (per-genome counters) and the synchronous step agree
  under the synchronous schedule.
"""
import numpy as np
import pytest
from scipy import stats


def one_generation_amounts(orc, seed, sigma, p_ben, p_del, islands=64):
    # one agent per island, no migration, no tracking: the child is its
    # parent (fitness 0) plus the signed mutation amount
    c = orc.Config(rows=islands, cols=islands, n=1, tournament=1, policy=orc.NONE, bits=1,
                   W=2, interval=0, p_ben=p_ben, p_del=p_del, seed=seed,
                   fitness=orc.FITNESS_FLOAT, sigma=sigma)
    t, _, _ = orc.run(c, generations=1)
    return t.view(np.float32).astype(np.float64)


def test_amounts_are_half_normal(orc):
    sigma = 2.5
    a = np.concatenate([one_generation_amounts(orc, s, sigma, 1.0, 0.0) for s in range(5)])
    assert (a >= 0).all()
    ks = stats.kstest(a, stats.halfnorm(scale=sigma).cdf)
    assert ks.pvalue > 1e-3, ks
    se = sigma * np.sqrt(1 - 2 / np.pi) / np.sqrt(len(a))
    assert abs(a.mean() - sigma * np.sqrt(2 / np.pi)) < 4 * se
    d = np.concatenate([one_generation_amounts(orc, s, sigma, 0.0, 1.0) for s in range(5, 8)])
    assert (d <= 0).all()
    assert stats.kstest(-d, stats.halfnorm(scale=sigma).cdf).pvalue > 1e-3


def test_mutation_probabilities_and_untouched_children(orc):
    a = one_generation_amounts(orc, 9, 1.0, 0.2, 0.3)
    frac_pos, frac_neg = (a > 0).mean(), (a < 0).mean()
    n = len(a)
    assert abs(frac_pos - 0.2) < 4 * np.sqrt(0.2 * 0.8 / n)
    assert abs(frac_neg - 0.3) < 4 * np.sqrt(0.3 * 0.7 / n)
    assert ((a == 0) == ~((a > 0) | (a < 0))).all()


def test_amount_bits_follow_the_stated_arithmetic(orc):
    # regression: the amount for one draw recomputed in numpy binary32
    seed, sigma = 3, 0.75
    a = one_generation_amounts(orc, seed, sigma, 1.0, 0.0, islands=4)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    c = np.float32(sigma / np.sqrt(24.0 + 1.0 / 12.0) / 16777216.0)
    for i in range(16):
        q = orc.philox4x32(key, (0, i, 0, 256))
        B = sum(bin(int(x)).count("1") for x in q[:3])
        g = (B - 48) * (1 << 24) + (int(q[3]) >> 8) - (1 << 23)
        want = np.abs(np.float32(g) * c)
        assert np.float32(a[i]) == want


def test_selection_compares_floats(orc):
    # p = 0: children are copies; a 64-candidate tournament over 4 agents
    # finds the fittest (-0.5) with probability 1 - (3/4)^64
    c = orc.Config(rows=2, cols=3, n=4, tournament=64, policy=orc.NONE, bits=1, W=2,
                   interval=0, seed=4, fitness=orc.FITNESS_FLOAT)
    f = np.tile(np.array([-3.0, -0.5, -7.0, -1.5], np.float32), c.islands)
    t, _, _ = orc.run(c, generations=1, trait=f.view(np.uint32),
                      surf=np.zeros(c.agents, np.uint64))
    assert (t.view(np.float32) == np.float32(-0.5)).all()


@pytest.mark.parametrize("policy", [0, 1, 5])
def test_free_running_step_matches_synchronous(orc, policy):
    c = orc.Config(rows=4, cols=3, n=8, tournament=5, policy=policy, bits=2, W=2, interval=1,
                   p_ben=0.05, p_del=0.33, seed=12, fitness=orc.FITNESS_FLOAT, sigma=0.5)
    rng = np.random.default_rng(1)
    f = rng.normal(0, 1, c.agents).astype(np.float32)
    surf = rng.integers(0, 2**63, c.agents, dtype=np.uint64)
    gens = 30
    st, ss, _ = orc.run(c, generations=gens, trait=f.view(np.uint32), surf=surf, G0=7)
    sched = orc.sync_schedule(c, 7, gens)
    at, as_, aT = orc.run_async(c, f.view(np.uint32), surf, np.full(c.agents, 7, np.uint32), 7,
                                gens, sched)
    assert np.array_equal(st, at) and np.array_equal(ss, as_)
    assert (aT == 7 + gens).all()
    assert (st.view(np.float32) != f).any()
