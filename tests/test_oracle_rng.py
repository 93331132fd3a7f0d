"""Pins for the oracle's Philox4x32-10 (Salmon et al., SC'11).

The oracle's round function is one macro instantiated at 32- and 64-bit words.
* The 64-bit instance must reproduce numpy.random.Philox (a library
  Philox4x64-10): this pins the round structure and key schedule.
* The 32-bit instance must reproduce triton's Philox4x32-10 (run by triton's
  CPU interpreter): this pins the 32-bit multipliers.
* The Weyl key increments are the fractional parts of the golden ratio and
  sqrt(3) scaled by 2^32 / 2^64 (closed forms from the Philox paper).
* Statistical checks: bit frequencies and floor(w*n/2^32) index uniformity.
"""
import os
import subprocess
import sys
import textwrap
from decimal import Decimal, getcontext

import numpy as np
import pytest


@pytest.mark.parametrize("key,ctr", [((0, 0), (0, 0, 0, 0)),
                                     ((5, 7), (3, 0, 0, 0)),
                                     ((2**64 - 1, 12345), (2**64 - 2, 1, 2**63, 9)),
                                     ((0xDEADBEEF, 0xFEEDFACECAFEBEEF), (1, 2, 3, 4))])
def test_philox4x64_matches_numpy(orc, key, ctr):
    # numpy increments the counter before producing a block
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64),
                          counter=np.array(ctr, dtype=np.uint64))
    want = bg.random_raw(4)
    c1 = (ctr[0] + 1) % 2**64
    carry = 1 if c1 == 0 else 0
    got = orc.philox4x64(key, (c1, (ctr[1] + carry) % 2**64, ctr[2], ctr[3]))
    assert [int(x) for x in got] == [int(x) for x in want]


def test_weyl_constants_closed_form():
    getcontext().prec = 60
    phi_frac = (Decimal(5).sqrt() - 1) / 2          # golden ratio - 1
    sqrt3_frac = Decimal(3).sqrt() - 1
    assert int(phi_frac * 2**32) == 0x9E3779B9
    assert int(sqrt3_frac * 2**32) == 0xBB67AE85
    assert int(phi_frac * 2**64) == 0x9E3779B97F4A7C15
    assert int(sqrt3_frac * 2**64) == 0xBB67AE8584CAA73B
    src = open(os.path.join(os.path.dirname(__file__), "..", "oracle", "hsga_oracle.c")).read()
    for c in ("0x9E3779B9u", "0xBB67AE85u", "0x9E3779B97F4A7C15ull", "0xBB67AE8584CAA73Bull"):
        assert c in src


_TRITON_SCRIPT = textwrap.dedent("""
    import os, sys, json
    os.environ["TRITON_INTERPRET"] = "1"
    import torch, triton, triton.language as tl
    from triton.language.random import philox

    @triton.jit
    def k(out, seed, c0p, c1p, c2p, c3p, N: tl.constexpr):
        i = tl.arange(0, N)
        c0 = tl.load(c0p + i); c1 = tl.load(c1p + i); c2 = tl.load(c2p + i); c3 = tl.load(c3p + i)
        a, b, c, d = philox(seed, c0, c1, c2, c3)
        tl.store(out + i * 4 + 0, a); tl.store(out + i * 4 + 1, b)
        tl.store(out + i * 4 + 2, c); tl.store(out + i * 4 + 3, d)

    cases = json.loads(sys.argv[1])
    res = []
    for seed, ctr in cases:
        cs = [torch.tensor([ctr[j]], dtype=torch.int64).to(torch.uint32) for j in range(4)]
        out = torch.zeros(4, dtype=torch.int64).to(torch.uint32)
        k[(1,)](out, seed, *cs, N=1)
        res.append([int(x) & 0xFFFFFFFF for x in out.to(torch.int64).tolist()])
    print(json.dumps(res))
""")


def test_philox4x32_matches_triton_interpreter(orc, tmp_path):
    pytest.importorskip("triton")
    import json
    cases = [(0, [0, 0, 0, 0]), (1, [0, 0xFFFFFFFF, 7, 1]),
             (0xFFFFFFFFFFFFFFFF, [0xFFFFFFFF] * 4),
             (0x299F31D0A4093822, [0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344]),
             (12345678901234, [31, 524287, 999999, 3])]
    script = tmp_path / "tri.py"
    script.write_text(_TRITON_SCRIPT)
    r = subprocess.run([sys.executable, str(script), json.dumps(cases)],
                       capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + r.stderr[-300:])
    got_triton = json.loads(r.stdout.strip().splitlines()[-1])
    for (seed, ctr), want in zip(cases, got_triton):
        got = orc.philox4x32((seed & 0xFFFFFFFF, seed >> 32), ctr)
        assert [int(x) for x in got] == want, (seed, ctr)


def test_philox_bits_and_index_uniform(orc):
    # 4096 blocks x 4 words: every bit position ~ Bernoulli(1/2)
    words = np.array([orc.philox4x32((1, 0), (j, 3, 5, 1)) for j in range(4096)],
                     dtype=np.uint64).reshape(-1)
    bits = ((words[:, None] >> np.arange(32, dtype=np.uint64)) & np.uint64(1)).astype(np.float64)
    freq = bits.mean(axis=0)
    sd = np.sqrt(0.25 / len(words))
    assert np.all(np.abs(freq - 0.5) < 5 * sd)
    # floor(w * n / 2^32) over n = 32: chi-square vs uniform
    from scipy import stats
    idx = (words * np.uint64(32)) >> np.uint64(32)
    counts = np.bincount(idx.astype(np.int64), minlength=32)
    assert stats.chisquare(counts).pvalue > 1e-4


def test_philox_sweep_matches_single_calls(orc):
    key = 0x0123456789ABCDEF
    for c0, c1, c2, c3 in [(0, 3, 5, 1), (2**32 - 64, 0xFFFFFFFF, 7, 0),
                           (1000, 0xFFFFFFFE, 2**31, 256)]:
        bulk = orc.philox_sweep(key, c0, 64, c1, c2, c3)
        for i in range(64):
            one = orc.philox4x32((key & 0xFFFFFFFF, key >> 32), (c0 + i, c1, c2, c3))
            assert [int(x) for x in one] == bulk[i].tolist()


def test_philox_uniform_over_2_to_24_words(orc):
    """2^22 blocks (2^24 words): every bit ~ Bernoulli(1/2) within 5 sigma and
    floor(w n / 2^32) uniform for n = 5, 32, 100 (chi-square)."""
    from scipy import stats
    w = orc.philox_sweep(1, 0, 1 << 22, 9, 11, 1).reshape(-1).astype(np.uint64)
    sd = np.sqrt(0.25 / len(w))
    for b in range(32):
        f = ((w >> np.uint64(b)) & np.uint64(1)).mean()
        assert abs(f - 0.5) < 5 * sd, b
    for n in (5, 32, 100):
        idx = ((w * np.uint64(n)) >> np.uint64(32)).astype(np.int64)
        assert stats.chisquare(np.bincount(idx, minlength=n)).pvalue > 1e-4, n
