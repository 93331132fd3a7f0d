"""The allocation-free entry point, hsga_run_generations_noalloc, against the
ordinary grid entry points.

Callers that must not allocate device memory (a process under a fixed
memory budget, code running inside another framework's allocator) advance
their own device planes with hsga_run_generations_noalloc; its scratch lives
in an array built into the library.  Its results must equal what a grid
created with hsga_init_grid produces from the same state, bit for bit (the
tolerance every parity test here uses), on two calls in a row — the second
call reuses the scratch the first one left behind.

This file is named to be collected last, so that a run that stops at the
first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2404_10861_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_10861_gb300 import _build, binding
    _build.build()
    return binding


@pytest.mark.parametrize("kw", [
    dict(rows=64, cols=64, n=32, tournament=2, policy="tilted", bits=2, p_ben=1e-3, seed=2),
    dict(rows=6, cols=9, n=40, tournament=3, policy="steady", bits=1, p_ben=0.01, p_del=0.01,
         interval=2, seed=7),
])
def test_noalloc_matches_grid_entry_points_twice(hb, kw):
    import torch
    cfg = hb.make_config(**kw)
    agents = cfg.rows * cfg.cols * cfg.agents_per_island
    trait, surf = inputs.small_trait_population(agents, seed=3, levels=5)
    G0, n1, n2 = 1000, 37, 150
    stream = torch.cuda.Stream()

    # existing entry points: a grid that owns its memory
    with hb.Grid(stream=stream.cuda_stream, **kw) as g:
        g.set_population(trait, surf, G0)
        g.run(n1)
        g.sync()
        want1 = g.population()
        g.run(n2)
        g.sync()
        want2 = g.population()

    # allocation-free entry point on caller-owned device planes, two calls
    td = torch.from_numpy(trait.view(np.int32)).cuda()
    sd = torch.from_numpy(surf.view(np.int64)).cuda()
    torch.cuda.synchronize()
    hb.hsga_run_generations_noalloc(cfg, G0, n1, td, sd, stream.cuda_stream)
    got1 = (td.cpu().numpy().view(np.uint32).copy(), sd.cpu().numpy().view(np.uint64).copy())
    hb.hsga_run_generations_noalloc(cfg, G0 + n1, n2, td, sd, stream.cuda_stream)
    got2 = (td.cpu().numpy().view(np.uint32), sd.cpu().numpy().view(np.uint64))
    for got, want in ((got1, want1), (got2, want2)):
        assert np.array_equal(got[0], want[0])
        assert np.array_equal(got[1], want[1])


def test_noalloc_rejects_oversized_grid_and_host_planes(hb):
    import torch
    big = hb.make_config(rows=128, cols=128, n=32)          # 16384 islands > 8192
    t = torch.zeros(128 * 128 * 32, dtype=torch.int32, device="cuda")
    s = torch.zeros(128 * 128 * 32, dtype=torch.int64, device="cuda")
    with pytest.raises(hb.HsgaError) as e:
        hb.hsga_run_generations_noalloc(big, 0, 1, t, s)
    assert e.value.status == -1
    small = hb.make_config(rows=4, cols=4, n=32)
    th = np.zeros(512, dtype=np.uint32)
    sh = np.zeros(512, dtype=np.uint64)
    with pytest.raises(hb.HsgaError) as e:
        hb.hsga_run_generations_noalloc(small, 0, 1, th, sh)
    assert e.value.status == -1


def test_noalloc_rejects_generation_counts_that_wrap(hb):
    """G + n is checked without forming a sum that could wrap around in 64
    bits: a G near 2^64 with one more generation must be refused, not run at
    a truncated generation."""
    import torch
    cfg = hb.make_config(rows=4, cols=4, n=32)
    t = torch.zeros(512, dtype=torch.int32, device="cuda")
    s = torch.zeros(512, dtype=torch.int64, device="cuda")
    for G, n in ((2**64 - 1, 1), (2**63, 2**63), (1, 2**64 - 1), (2**32 - 65, 1)):
        with pytest.raises(hb.HsgaError) as e:
            hb.hsga_run_generations_noalloc(cfg, G, n, t, s)
        assert e.value.status == -1, (G, n)
    hb.hsga_run_generations_noalloc(cfg, 2**32 - 66, 1, t, s)   # the largest G + n allowed


def test_noalloc_planes_must_be_on_the_current_device(hb):
    """The scratch array's address is the current device's, so planes that
    live on another device are refused before any launch.  With one GPU the
    current device's own planes are accepted; with two, planes on device 1
    are refused while device 0 is current."""
    import torch
    cfg = hb.make_config(rows=4, cols=4, n=32)
    torch.cuda.set_device(0)
    t0 = torch.zeros(512, dtype=torch.int32, device="cuda:0")
    s0 = torch.zeros(512, dtype=torch.int64, device="cuda:0")
    hb.hsga_run_generations_noalloc(cfg, 0, 3, t0, s0)
    if torch.cuda.device_count() < 2:
        return
    t1 = torch.zeros(512, dtype=torch.int32, device="cuda:1")
    s1 = torch.zeros(512, dtype=torch.int64, device="cuda:1")
    with pytest.raises(hb.HsgaError) as e:
        hb.hsga_run_generations_noalloc(cfg, 0, 3, t1, s1)
    assert e.value.status == -1
