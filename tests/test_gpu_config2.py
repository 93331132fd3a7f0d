"""The mid-grid workload at its stated size on the GPU: 64 x 64 islands x 32
agents, 32 two-bit differentiae under each of the steady, tilted and
stretched policies, tournament 2, synchronous migration every generation,
100,000 generations, seeds 1-8, with adaptation on (beneficial mutation
probability 1e-3, +1 to the trait) and off (0): 48 runs.

The outcome the paper reports for its on-hardware trial ("Results ›
On-hardware Trial"): without adaptation the reconstructed phylogenies are
longer; selective sweeps shorten them.  Per policy, every island's sampled
genome (4,096 per run) is reconstructed (the oracle's trie) and a one-sided
Mann-Whitney U test over the 8 seeds must find sum branch length and mean
pairwise distance larger with adaptation off (alpha 0.05).  Colless and
Sackin indices are computed and reported beside them.  When the environment
variable HSGA_REPORT_DIR names a directory, the per-run phylometrics are
written there as config2_phylometrics.json.
"""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GENS = 100_000
SEEDS = range(1, 9)
POLICIES = ("steady", "tilted", "stretched")
KEYS = ("sum_branch_length", "mean_pairwise_distance", "colless", "sackin")


@pytest.fixture(scope="module")
def hb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_10861_gb300 import _build, binding
    _build.build()
    return binding


@pytest.fixture(scope="module")
def runs(hb, orc):
    """Phylometrics of all 48 runs: {(policy, adaptive): [dict per seed]}."""
    from oracle import phylo
    out = {}
    for policy in POLICIES:
        for adaptive in (True, False):
            res = []
            for seed in SEEDS:
                kw = dict(rows=64, cols=64, n=32, tournament=2, policy=policy, bits=2, W=2,
                          interval=1, p_ben=1e-3 if adaptive else 0.0, p_del=0.0, seed=seed)
                with hb.Grid(**kw) as g:
                    g.run(GENS)
                    g.sync()
                    assert g.stats()["generation"] == GENS
                    words, _ = g.sample(64 * 64)            # one genome per island
                    trait, _ = g.population()
                s = words[:, 1].astype(np.uint64) | (words[:, 2].astype(np.uint64) << np.uint64(32))
                tree = phylo.reconstruct(s, orc.POLICY_NAMES[policy], 2, 2, GENS)
                m = {k: float(v) for k, v in phylo.phylometrics(tree).items()}
                m.update(seed=seed, mean_trait=float(trait.mean()), nodes=int(tree.n_nodes))
                res.append(m)
            out[(policy, adaptive)] = res
    report = os.environ.get("HSGA_REPORT_DIR")
    if report:
        os.makedirs(report, exist_ok=True)
        with open(os.path.join(report, "config2_phylometrics.json"), "w") as f:
            json.dump({f"{p}/{'adaptive' if a else 'neutral'}": v for (p, a), v in out.items()},
                      f, indent=1)
    return out


@pytest.mark.parametrize("policy", POLICIES)
def test_adaptation_shortens_phylogenies(runs, policy):
    from scipy import stats
    on, off = runs[(policy, True)], runs[(policy, False)]
    assert all(m["mean_trait"] > 0 for m in on)           # beneficial mutations spread
    assert all(m["mean_trait"] == 0 for m in off)          # neutral: traits stay 0
    for key in ("sum_branch_length", "mean_pairwise_distance"):
        a = [m[key] for m in on]
        b = [m[key] for m in off]
        p = stats.mannwhitneyu(b, a, alternative="greater").pvalue
        assert p < 0.05, (policy, key, a, b, p)
    for key in ("colless", "sackin"):
        assert all(m[key] >= 0 for m in on + off)
