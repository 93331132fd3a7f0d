"""Clade-reconstruction trial (arXiv 2404.10861, "Results › Clade
Reconstruction Trial"): 3x3 islands, founders tagged with random 16-bit
identifiers that are inherited unchanged, neutral selection, one end-state
genome per island after 25, 50, 100 and 250 generations, trie reconstruction
from 1-bit tilted surfaces.  The paper's expectations:

* taxa of the same founding clade are reconstructed as closer relatives than
  taxa of different clades;
* the number of founding clades still present falls with duration.

The tag occupies the trait word; tournament size 1 makes selection neutral
(the tag never influences reproduction) and mutation is off, so the tag is
inherited unchanged.  The oracle version runs on the CPU; the GPU version
runs the same trial through the C-ABI and must equal the oracle bit-exactly.
"""
import numpy as np
import pytest
from scipy import stats

from oracle import phylo

DURATIONS = (25, 50, 100, 250)
REPLICATES = 30


def trial_config(orc, seed):
    return orc.Config(rows=3, cols=3, n=32, tournament=1, policy=orc.TILTED, bits=1, W=2,
                      interval=1, p_ben=0.0, p_del=0.0, seed=seed)


def founder_tags(agents, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(0, 2**16, size=agents).astype(np.uint32)


def analyse(orc, snapshots):
    """snapshots: {duration: (population traits, sampled words)} of one
    replicate -> (clades in population, clades among samples, mean distance
    same-tag, mean distance different-tag) per duration."""
    out = {}
    for G, (trait, words) in snapshots.items():
        tags = words[:, 0]
        surf = words[:, 1].astype(np.uint64) | (words[:, 2].astype(np.uint64) << np.uint64(32))
        tree = phylo.reconstruct(surf, orc.TILTED, 1, 2, G)
        same, diff = [], []
        for a in range(len(tags)):
            for b in range(a + 1, len(tags)):
                d = phylo.pairwise_distance(tree, a, b)
                (same if tags[a] == tags[b] else diff).append(d)
        out[G] = (len(np.unique(trait)), len(np.unique(tags)),
                  np.mean(same) if same else None, np.mean(diff) if diff else None)
    return out


def check_trial(results):
    # founding clades in the population never increase with time (exact)
    for rep in results:
        counts = [rep[G][0] for G in DURATIONS]
        assert all(a >= b for a, b in zip(counts, counts[1:])), counts
    # among the nine samples, the mean clade count falls with duration
    means = [np.mean([rep[G][1] for rep in results]) for G in DURATIONS]
    assert all(a > b for a, b in zip(means, means[1:])), means
    # same-clade pairs reconstruct as closer relatives than different-clade pairs
    pairs = [(rep[G][2], rep[G][3]) for rep in results for G in DURATIONS
             if rep[G][2] is not None and rep[G][3] is not None]
    assert len(pairs) >= 20
    same = np.array([p[0] for p in pairs])
    diff = np.array([p[1] for p in pairs])
    assert np.mean(same < diff) > 0.8
    assert stats.wilcoxon(same, diff, alternative="less").pvalue < 1e-3


def test_clade_trial_oracle(orc):
    results = []
    for rep in range(REPLICATES):
        c = trial_config(orc, seed=1000 + rep)
        trait = founder_tags(c.agents, rep)
        surf = np.zeros(c.agents, dtype=np.uint64)
        snaps, G = {}, 0
        for D in DURATIONS:
            trait, surf, _ = orc.run(c, trait, surf, G0=G, generations=D - G)
            G = D
            words, _ = orc.sample(c, trait, surf, G, 9)
            snaps[D] = (trait.copy(), words)
        results.append(analyse(orc, snaps))
    check_trial(results)


@pytest.mark.gpu
def test_clade_trial_gpu_equals_oracle(orc):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_10861_gb300 import _build, binding as hb
    _build.build()
    results = []
    for rep in range(REPLICATES):
        c = trial_config(orc, seed=1000 + rep)
        tags = founder_tags(c.agents, rep)
        zero = np.zeros(c.agents, dtype=np.uint64)
        snaps = {}
        with hb.Grid(rows=3, cols=3, n=32, tournament=1, policy="tilted", bits=1, W=2,
                     seed=1000 + rep) as g:
            g.set_population(tags, zero, 0)
            G = 0
            ot, os_ = tags, zero
            for D in DURATIONS:
                g.run(D - G)
                ot, os_, _ = orc.run(c, ot, os_, G0=G, generations=D - G)
                G = D
                t, s = g.population()
                assert np.array_equal(t, ot) and np.array_equal(s, os_)
                words, where = g.sample(9)
                ow, _ = orc.sample(c, ot, os_, G, 9)
                assert np.array_equal(words, ow)
                snaps[D] = (t, words)
        results.append(analyse(orc, snaps))
    check_trial(results)
