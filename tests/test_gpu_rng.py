"""The kernels' counter-based generator against the oracle's independent
Philox4x32-10: every word of a 2^24-counter sweep, and sweeps over the
reserved slot words (emigrant, immigrant, sample) and the largest counters."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_10861_gb300 import _build, binding
    _build.build()
    return binding


def device_sweep(hb, seed, c0, count, c1, c2, c3):
    import torch
    out = torch.empty((count, 4), dtype=torch.int32, device="cuda")
    hb.hsga_philox_device(seed, c0, count, c1, c2, c3, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32)


def test_two_to_the_24_counters(hb, orc):
    seed = 0xDEADBEEF12345678
    got = device_sweep(hb, seed, 0, 1 << 24, 17, 4242, 1)
    want = orc.philox_sweep(seed, 0, 1 << 24, 17, 4242, 1)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("c0,c1,c2,c3", [(2**32 - 65536, 0xFFFFFFFF, 123, 0),
                                         (0, 0xFFFFFFFE, 2**32 - 1, 0),
                                         (5, 0xFFFFFFFF, 77, 3),
                                         (1000, 524287, 999999, 256)])
def test_reserved_and_extreme_counters(hb, orc, c0, c1, c2, c3):
    got = device_sweep(hb, 7, c0, 65536, c1, c2, c3)
    assert np.array_equal(got, orc.philox_sweep(7, c0, 65536, c1, c2, c3))


def test_throughput_kernel_draws_the_same_blocks(hb, orc):
    """The kernel that measures the generator's throughput evaluates the same
    blocks as the oracle: per thread, the xor of every word of its blocks."""
    import torch
    threads, m, c2, c3 = 300, 37, 0xABCDEF, 9          # a ragged block, m not a multiple of 4
    seed = 0x0123456789ABCDEF
    out = torch.zeros(threads, dtype=torch.int32, device="cuda")
    hb.hsga_philox_throughput(seed, threads, m, c2, c3, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint32)
    for t in list(range(0, threads, 7)) + [threads - 1]:
        want = np.bitwise_xor.reduce(orc.philox_sweep(seed, 0, m, t, c2, c3).reshape(-1))
        assert got[t] == want, t
