"""The C-ABI library without a GPU: it loads, exports every symbol that
include/hsga.h declares, and its host-side functions (site function, closed-
form timestamp lookup, argument validation) agree with the oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hb():
    from paper_2404_10861_gb300 import _build, binding
    _build.build()
    return binding


def declared_functions():
    src = open(os.path.join(ROOT, "include", "hsga.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(hsga_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_exports_every_declared_symbol(hb):
    names = declared_functions()
    assert len(names) >= 17
    lib = ctypes.CDLL(hb.library_path())
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(hb._SIGS), "binding must cover exactly the header"
    assert hb.lib().hsga_version() == 100
    assert hb.lib().hsga_status_string(-5) == b"bounded device wait timed out"


@pytest.mark.parametrize("policy", [0, 1, 2, 3, 5])
def test_site_matches_oracle(hb, orc, policy):
    rng = np.random.default_rng(policy)
    Ts = list(range(5000)) + [int(x) for x in rng.integers(0, 2**32 - 2, 3000)]
    for S, W in ((8, 2), (16, 4), (32, 2), (64, 2), (64, 1), (64, 4), (128, 2), (256, 2),
                 (256, 4)):
        if policy == 5 and (S // 2) // W < 2:
            continue
        for T in Ts[::7]:
            assert hb.hsga_site(policy, S, W, T) == orc.site(policy, S, W, T), (S, W, T)


@pytest.mark.parametrize("policy", [0, 1, 2, 3, 5])
def test_closed_form_lookup_matches_bruteforce(hb, orc, policy):
    """Timestamps are deduced from (site, T) alone; the closed form must equal
    the brute-force last-writer replay."""
    for S, W in ((8, 2), (16, 2), (32, 2), (64, 2), (32, 4), (64, 4), (16, 1), (128, 2),
                 (256, 2), (256, 4), (4, 1)):
        if policy == 5 and (S // 2) // W < 2:
            continue
        Ts = list(range(0, 600)) + [1023, 1024, 1025, 4095, 4096, 4097, 65535, 65536, 99999,
                                    100000, 123457, 262143, 1000000]
        for T in Ts:
            got = hb.hsga_lookup(policy, S, W, T)
            want = orc.lookup(policy, S, W, T)
            assert np.array_equal(got, want), (policy, S, W, T, got, want)


def test_config_validation_needs_no_gpu(hb):
    bad = [dict(rows=0), dict(n=0), dict(n=65), dict(tournament=0), dict(bits=3),
           dict(policy=7), dict(policy="tilted", W=3), dict(policy="tilted", bits=8, W=8), dict(policy="stretched", W=0),
           dict(p_ben=0.7, p_del=0.5), dict(p_ben=-0.1), dict(kernel=9),
           dict(policy="hybrid", bits=8, W=4), dict(policy=6),
           dict(fitness="float", sigma=0.0), dict(fitness="float", sigma=-1.0),
           dict(fitness="float", sigma=1.0, n=33), dict(mode="buffered", n=33),
           dict(mode="buffered", coarsen=2), dict(words=3), dict(words=8),
           dict(words=2, n=33), dict(words=4, policy="none"), dict(bits=32),
           dict(bits=16, policy="tilted", W=4)]
    for kw in bad:
        cfg = hb.make_config(**kw)
        out = ctypes.c_void_p()
        assert hb.lib().hsga_init_grid(ctypes.byref(cfg), None, ctypes.byref(out)) == -1, kw
    assert hb.lib().hsga_lookup(0, 12, 2, 5, None) == -1
    cfg = hb.make_config(fitness="float", sigma=1.0)
    cfg.fitness = 2                                        # not a fitness model
    out = ctypes.c_void_p()
    assert hb.lib().hsga_init_grid(ctypes.byref(cfg), None, ctypes.byref(out)) == -1
