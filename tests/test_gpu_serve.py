"""Continuous batching: requests that arrive while others run are admitted
as memory frees up, their work overlaps on the device, and every result is
the same as running the request alone (bit-exact sampled surfaces); the
smaller requests' results also equal the oracle's run and sampling of the
same request."""
import numpy as np
import pytest

from conftest import oracle_config

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_10861_gb300 import _build, binding
    _build.build()
    return binding


def oracle_result(config, generations, k):
    """The oracle's run of one request from founders and its sample (runs in
    a worker process)."""
    import oracle
    c = oracle_config(oracle, config)
    t, s, _ = oracle.run(c, generations=generations)
    return oracle.sample(c, t, s, generations, k)


def test_served_results_equal_alone_and_oracle_under_memory_cap(hb, orc, oracle_pool):
    from paper_2404_10861_gb300 import serve
    reqs = serve.poisson_requests(24, rate=4000.0, seed=5, gen_scale=50,
                                  agents_range=(1024, 65536), sample_k=64)
    small = {r.rid: oracle_pool.submit(oracle_result, r.config, r.generations, r.sample_k)
             for r in reqs if r.agents * r.generations <= 3 * 10**7}
    assert len(small) >= 8
    biggest = max(hb.hsga_run_footprint(hb.make_config(**r.config)) for r in reqs)
    cap = biggest               # the largest request only fits alone: admission must wait
    res_b, st_b = serve.serve(reqs, memory_cap=cap, slice_ticks=64)
    res_a, _ = serve.serve_alone(reqs)
    assert len(res_b) == len(reqs) == len(res_a)
    assert st_b["peak_concurrent_runs"] >= 2          # work overlapped
    assert st_b["admissions_deferred"] > 0            # the cap bound
    by_id = {r.rid: r for r in res_a}
    for r in res_b:
        a = by_id[r.rid]
        assert np.array_equal(r.words, a.words), r.rid
        assert np.array_equal(r.where, a.where), r.rid
        assert r.finished >= r.admitted >= r.arrival - 1e-6
        if r.rid in small:
            ow, owhere = small[r.rid].result()
            assert np.array_equal(r.words, ow), ("oracle", r.rid)
            assert np.array_equal(r.where, owhere), ("oracle", r.rid)
    summ = serve.summarize(res_b, st_b)
    assert summ["latency_p99_s"] >= summ["latency_p50_s"] > 0


def test_large_requests_advance_on_their_own_grid_beside_the_batch(hb, orc, oracle_pool):
    """Requests of at least 2^20 agents run one at a time on a grid of their
    own, on a second stream beside the batch; every result equals the
    request run alone, and the first large one also the oracle's."""
    import torch
    from paper_2404_10861_gb300 import serve
    small = serve.poisson_requests(10, rate=4000.0, seed=7, gen_scale=100,
                                   agents_range=(1024, 16384), sample_k=64)
    big = dict(rows=256, cols=128, n=32, tournament=2, policy="tilted", bits=1, W=2,
               interval=1, p_ben=1e-3, p_del=0.0)                 # 2^20 agents
    bigs = [serve.Request(100 + i, 0.0005 * i, dict(big, seed=77 + i), 120 + 40 * i, 64)
            for i in range(2)]
    want = oracle_pool.submit(oracle_result, bigs[0].config, bigs[0].generations, 64)
    reqs = small + bigs
    stream, large = torch.cuda.Stream(), torch.cuda.Stream()
    res_b, st_b = serve.serve(reqs, memory_cap=1 << 36, slice_ticks=32,
                              stream=stream.cuda_stream, large_stream=large.cuda_stream)
    res_a, _ = serve.serve_alone(reqs)
    assert len(res_b) == len(reqs) == len(res_a)
    assert st_b["peak_concurrent_large_runs"] == 1
    by_id = {r.rid: r for r in res_a}
    for r in res_b:
        assert np.array_equal(r.words, by_id[r.rid].words), r.rid
        assert np.array_equal(r.where, by_id[r.rid].where), r.rid
    ow, owhere = want.result()
    got = {r.rid: r for r in res_b}[bigs[0].rid]
    assert np.array_equal(got.words, ow) and np.array_equal(got.where, owhere)
