"""Whole-population parity at the configurations' full sizes, through the
C-ABI, bit-exact (all arithmetic is integer):

* the wafer-shaped grid (512 x 1024 islands x 32 agents = 16,777,216 agents,
  tilted 64 x 1-bit surface, tournament 2, p_ben 1e-3) in the launch
  configuration the benchmark times (the streamed kernel), from a uniformly
  random population at G0 = 2^20 - 37, 64 generations split into uneven
  calls: every trait and every surface word equal to the oracle's run of the
  whole grid, then a 10,000-genome sample equal to the oracle's sampling;
* the mid grid (64 x 64 islands x 32 agents, 32 two-bit differentiae,
  p_ben 1e-3) for 10,000 generations from founders under each of the steady,
  tilted and stretched policies, on the resident kernel (the default for this
  size) and the streamed kernel.

The oracle runs in spawned worker processes while the GPU works.
"""
import numpy as np
import pytest

from conftest import oracle_config
from paper_2404_10861_gb300 import inputs

pytestmark = pytest.mark.gpu

WAFER = dict(rows=512, cols=1024, n=32, tournament=2, policy="tilted", bits=1, W=2,
             interval=1, p_ben=1e-3, p_del=0.0, seed=1)
WAFER_G0 = 2**20 - 37
WAFER_CHUNKS = (1, 20, 43)
MID_GENS = 10_000
MID_CHUNKS = (1, 4_321, 5_678)
POLICIES = ("steady", "tilted", "stretched")


def mid_kw(policy):
    return dict(rows=64, cols=64, n=32, tournament=2, policy=policy, bits=2, W=2, interval=1,
                p_ben=1e-3, p_del=0.0, seed=2)


@pytest.fixture(scope="module")
def hb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_10861_gb300 import _build, binding
    _build.build()
    return binding


@pytest.fixture(scope="module")
def wafer_start():
    return inputs.random_population(512 * 1024 * 32, seed=2024)


@pytest.fixture(scope="module")
def oracle_results(orc, oracle_pool, wafer_start):
    """Oracle runs submitted up front (they take tens of seconds each)."""
    jobs = {}
    c = oracle_config(orc, WAFER)
    jobs["wafer"] = oracle_pool.submit(orc.run, c, wafer_start[0], wafer_start[1], WAFER_G0,
                                       sum(WAFER_CHUNKS))
    for pol in POLICIES:
        jobs[pol] = oracle_pool.submit(orc.run, oracle_config(orc, mid_kw(pol)), None, None, 0,
                                       MID_GENS)
    return jobs


def first_difference(got, want):
    bad = np.nonzero(got != want)[0]
    return f"{len(bad)} differ, first at agents {bad[:5]}"


def test_wafer_whole_population_bit_exact(hb, orc, oracle_results, wafer_start):
    import torch
    hb.use_torch_allocator()
    try:
        stream = torch.cuda.Stream()
        with hb.Grid(stream=stream.cuda_stream, kernel=hb.KERNEL_STREAMED, **WAFER) as g:
            g.set_population(wafer_start[0], wafer_start[1], WAFER_G0)
            for n in WAFER_CHUNKS:
                g.run(n)
            g.sync()
            assert g.stats()["generation"] == WAFER_G0 + sum(WAFER_CHUNKS)
            t, s = g.population()
            w, where = g.sample(10_000)
    finally:
        hb.use_default_allocator()
    want_t, want_s, _ = oracle_results["wafer"].result()
    assert np.array_equal(t, want_t), "traits: " + first_difference(t, want_t)
    assert np.array_equal(s, want_s), "surfaces: " + first_difference(s, want_s)
    # the run moved every island: traits changed and the founders' random
    # surfaces were overwritten site by site
    assert np.count_nonzero(t != wafer_start[0]) > 0.9 * len(t)
    assert np.count_nonzero(s != wafer_start[1]) > 0.9 * len(s)
    c = oracle_config(orc, WAFER)
    ow, owhere = orc.sample(c, want_t, want_s, WAFER_G0 + sum(WAFER_CHUNKS), 10_000)
    assert np.array_equal(w, ow)
    assert np.array_equal(where, owhere)


@pytest.mark.parametrize("policy", POLICIES)
@pytest.mark.parametrize("kernel", ["resident_grid", "streamed"])
def test_mid_grid_10k_generations_bit_exact(hb, orc, oracle_results, policy, kernel):
    kid = {"resident_grid": hb.KERNEL_RESIDENT_GRID, "streamed": hb.KERNEL_STREAMED}[kernel]
    with hb.Grid(kernel=kid, **mid_kw(policy)) as g:
        for n in MID_CHUNKS:
            g.run(n)
        g.sync()
        assert g.stats()["generation"] == MID_GENS
        t, s = g.population()
    want_t, want_s, _ = oracle_results[policy].result()
    assert np.array_equal(t, want_t), "traits: " + first_difference(t, want_t)
    assert np.array_equal(s, want_s), "surfaces: " + first_difference(s, want_s)
    assert t.max() > 0                      # adaptation on: beneficial mutations spread
