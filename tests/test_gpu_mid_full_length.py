"""The mid-grid workload bit-exact at its full length: 64 x 64 islands x 32
agents, 32 two-bit differentiae, tournament 2, synchronous migration every
generation, 100,000 generations from founders, seeds 1 and 2, under each of
the steady, tilted and stretched policies with adaptation on (beneficial
mutation probability 1e-3) and off: 12 runs of 1.3e10 replications each.

The GPU runs them on the kernel a user gets for this size (the resident
kernel, tiles of islands per block), in uneven calls so that launches end
and restart mid-run; every trait and surface word of the final population
must equal the oracle's.  The oracle's 12 runs (about five minutes each on
one core) start in spawned worker processes before the GPU runs, one
process per run up to the host's cores.
"""
import os

import numpy as np
import pytest

from conftest import oracle_config

pytestmark = pytest.mark.gpu

GENS = 100_000
CHUNKS = (1, 33_333, 66_666)
SEEDS = (1, 2)
POLICIES = ("steady", "tilted", "stretched")
CASES = [(pol, adaptive, seed) for pol in POLICIES for adaptive in (True, False)
         for seed in SEEDS]


def run_kw(policy, adaptive, seed):
    return dict(rows=64, cols=64, n=32, tournament=2, policy=policy, bits=2, W=2, interval=1,
                p_ben=1e-3 if adaptive else 0.0, p_del=0.0, seed=seed)


@pytest.fixture(scope="module")
def hb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_10861_gb300 import _build, binding
    _build.build()
    return binding


@pytest.fixture(scope="module")
def oracle_runs(orc):
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    workers = max(1, min(len(CASES), (os.cpu_count() or 2) - 1))
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        jobs = {case: ex.submit(orc.run, oracle_config(orc, run_kw(*case)), None, None, 0, GENS)
                for case in CASES}
        yield jobs


@pytest.fixture(scope="module")
def gpu_runs(hb, oracle_runs):
    out = {}
    for case in CASES:
        with hb.Grid(**run_kw(*case)) as g:
            for n in CHUNKS:
                g.run(n)
            g.sync()
            assert g.stats()["generation"] == GENS
            out[case] = g.population()
    return out


@pytest.mark.parametrize("case", CASES, ids=[f"{p}-{'adaptive' if a else 'neutral'}-seed{s}"
                                             for p, a, s in CASES])
def test_mid_grid_full_length_bit_exact(gpu_runs, oracle_runs, case):
    t, s = gpu_runs[case]
    want_t, want_s, _ = oracle_runs[case].result()
    assert np.array_equal(t, want_t), f"traits: {int((t != want_t).sum())} differ"
    assert np.array_equal(s, want_s), f"surfaces: {int((s != want_s).sum())} differ"
    if case[1]:
        assert t.max() > 0      # adaptation on: beneficial mutations spread
    else:
        assert t.max() == 0     # neutral: traits stay 0
