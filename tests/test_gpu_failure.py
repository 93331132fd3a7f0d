"""Failure detection without a GPU fault: the bounded waits the resident
kernel applies to its neighbours' stamped records (one thread's, and the
warp-wide form of the tiled exchange), run on a record that nothing writes,
must each end with HSGA_ERR_WAIT_TIMEOUT near their limit and leave the
context usable; on a record that carries the stamp they must return at
once."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
WAIT_TIMEOUT = -5


@pytest.fixture(scope="module")
def hb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_10861_gb300 import _build, binding
    _build.build()
    return binding


def test_unmet_wait_times_out_and_context_survives(hb, orc):
    import torch
    record = torch.zeros(4, dtype=torch.int64, device="cuda")
    limit = 20_000_000                                      # 20 ms
    status, waited = hb.hsga_wait_probe(record, 1, limit)
    assert status == WAIT_TIMEOUT
    assert 2 * limit <= waited < 2 * limit + 200_000_000   # both forms ran out
    record.copy_(torch.tensor([(3 << 32) | v for v in (11, 12, 13, 2)], dtype=torch.int64))
    status, waited = hb.hsga_wait_probe(record, 3, limit)
    assert status == 0 and waited < limit
    record[1] = (4 << 32) | 12                              # one word of a newer record
    status, waited = hb.hsga_wait_probe(record, 3, limit)
    assert status == WAIT_TIMEOUT and waited >= 2 * limit
    record[1] = (3 << 32) | 12
    record[2] = (2 << 32) | 13                              # one word of an older record
    status, _ = hb.hsga_wait_probe(record, 3, limit)
    assert status == WAIT_TIMEOUT
    # the context still runs kernels: a resident grid against the oracle
    kw = dict(rows=4, cols=4, n=32, tournament=2, policy="steady", bits=1, seed=1)
    c = orc.Config(rows=4, cols=4, n=32, tournament=2, policy=orc.STEADY, bits=1, W=2,
                   interval=1, seed=1)
    want_t, want_s, _ = orc.run(c, generations=50)
    with hb.Grid(kernel=hb.KERNEL_RESIDENT_GRID, **kw) as g:
        g.run(50)
        g.sync()
        t, s = g.population()
    assert np.array_equal(t, want_t) and np.array_equal(s, want_s)


def test_probe_argument_checks(hb):
    import torch
    record = torch.zeros(4, dtype=torch.int64, device="cuda")
    with pytest.raises(hb.HsgaError):
        hb.hsga_wait_probe(record, 1, 2_000_000_000)        # over the 1 s cap
    with pytest.raises(hb.HsgaError):
        hb.hsga_wait_probe(np.zeros(4, np.uint64), 1, 1000)  # host memory


def test_synchronous_calls_refuse_a_capturing_stream(hb, orc):
    """Calls that must wait for their stream return HSGA_ERR_NOT_CAPTURABLE
    when that stream is being captured into a CUDA graph, before touching it,
    so the capture stays valid and the grid keeps working afterwards."""
    import ctypes
    import torch
    NOT_CAPTURABLE = -7
    stream = torch.cuda.Stream()
    kw = dict(rows=8, cols=8, n=32, tournament=2, policy="tilted", bits=1, p_ben=1e-3, seed=3)
    c = orc.Config(rows=8, cols=8, n=32, tournament=2, policy=orc.TILTED, bits=1, W=2,
                   interval=1, p_ben=1e-3, seed=3)
    with hb.Grid(stream=stream.cuda_stream, **kw) as g:
        g.run(20)
        g.sync()
        words = np.zeros((4, 4), dtype=np.uint32)
        where = np.zeros((4, 2), dtype=np.uint32)
        t = np.zeros(c.agents, dtype=np.uint32)
        s = np.zeros(c.agents, dtype=np.uint64)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(stream):
            graph.capture_begin(capture_error_mode="thread_local")
            try:
                st_sync = hb.lib().hsga_synchronize(g.handle)
                st_sample = hb.lib().hsga_sample_surfaces(
                    g.handle, 4, ctypes.c_void_p(words.ctypes.data),
                    ctypes.c_void_p(where.ctypes.data))
                st_get = hb.lib().hsga_get_population(
                    g.handle, ctypes.c_void_p(t.ctypes.data), ctypes.c_void_p(s.ctypes.data))
            finally:
                graph.capture_end()
        assert (st_sync, st_sample, st_get) == (NOT_CAPTURABLE,) * 3
        g.run(15)
        g.sync()
        got = g.population()
    want = orc.run(c, generations=35)[:2]
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
