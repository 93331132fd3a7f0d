"""Pins for the oracle's surface site-selection functions.

The paper fixes properties, not formulas (section "Surface-based Hereditary
Stratigraphy Algorithms" and "Distributed Phylogenetic Tracking"): a
fixed-size buffer written in place, pruning only by overwrite, timestamps
recoverable from (site, T), "steady" spreading retained time points evenly
over history, "tilted" favouring recent ones.  Each test below replays the
site function deposition by deposition (brute force) and checks one such
property, or the structural statement of the reading it implements.
"""
import numpy as np
import pytest

STEADY, TILTED, STRETCHED, TRIVIAL = 0, 1, 2, 3


def replay(orc, policy, S, W, N):
    """Yield (n, retained times sorted) after n = 1..N depositions."""
    times = -np.ones(S, dtype=np.int64)
    for n in range(1, N + 1):
        s = orc.site(policy, S, W, n - 1)
        assert 0 <= s <= S
        if s < S:
            times[s] = n - 1
        yield n, times.copy()


def level(t, L):
    h = ((t + 1) & -(t + 1)).bit_length() - 1
    return min(h, L - 1)


def test_trivial_is_modulo(orc):
    for S in (8, 32, 64):
        for T in list(range(300)) + [2**31 + 5, 2**32 - 2]:
            assert orc.site(TRIVIAL, S, 2, T) == T % S


@pytest.mark.parametrize("S", [4, 8, 16, 32, 64])
def test_steady_even_spread(orc, S):
    s = S.bit_length() - 1
    N = 4096 if S <= 16 else 8192
    for n, times in replay(orc, STEADY, S, 2, N):
        kept = np.sort(times[times >= 0])
        if n <= S:
            assert list(kept) == list(range(n))           # fills in order
            continue
        assert len(kept) == S                              # no wasted space
        e = max(0, (n - 1).bit_length() - s)
        want = {m * 2**e - 1 for m in range(1, n // 2**e + 1)}
        assert want <= set(int(x) for x in kept)          # multiples of 2^e kept
        pts = np.concatenate([[-1], kept, [n]])
        assert np.diff(pts).max() * S / n < 2.0            # gap < 2N/S


@pytest.mark.parametrize("S,W", [(8, 2), (16, 2), (32, 2), (64, 2), (32, 4), (64, 4), (16, 1)])
def test_tilted_keeps_last_W_per_level_and_recency(orc, S, W):
    L = S // W
    N = 4096
    horizon = W * 2 ** (L - 1)
    per_level = {}
    for n, times in replay(orc, TILTED, S, W, N):
        t = n - 1
        per_level.setdefault(level(t, L), []).append(t)
        kept = set(int(x) for x in times[times >= 0])
        assert t in kept                                    # newest always kept
        want = set()
        for lv in per_level.values():
            want.update(lv[-W:])
        assert kept == want
        if n <= horizon:
            pts = np.sort(np.array(sorted(kept) + [-1]))
            gaps = np.diff(pts)
            ages = (n - 1) - pts[1:]
            ok = ages > 0
            assert np.all(gaps[ok] - 1 <= 2.0 / (2 * W - 1) * ages[ok] + 1e-9)


@pytest.mark.parametrize("S,W", [(8, 2), (16, 2), (32, 2), (64, 2), (64, 4), (32, 1)])
def test_stretched_keeps_first_W_per_level(orc, S, W):
    L = S // W
    per_level = {}
    for n, times in replay(orc, STRETCHED, S, W, 4096):
        t = n - 1
        per_level.setdefault(level(t, L), []).append(t)
        kept = np.sort(times[times >= 0])
        want = set()
        for lv in per_level.values():
            want.update(lv[:W])
        assert set(int(x) for x in kept) == want
        pts = np.concatenate([[-1], kept])
        gaps = np.diff(pts)
        assert np.all(gaps - 1 <= (kept + 1) / (W + 1) + 1e-9)   # dense early history


@pytest.mark.parametrize("policy", [STEADY, TILTED, STRETCHED, TRIVIAL])
def test_lookup_matches_replay(orc, policy):
    for S in (8, 64):
        last = None
        for n, times in replay(orc, policy, S, 2, 1500):
            last = times
            if n in (1, 7, 64, 65, 100, 1023, 1024, 1500):
                assert list(orc.lookup(policy, S, 2, n)) == list(times)
        assert last is not None


def test_site_in_range_large_T(orc):
    rng = np.random.default_rng(3)
    for T in rng.integers(0, 2**32 - 2, size=2000):
        for policy in (STEADY, TILTED, STRETCHED, TRIVIAL):
            for S in (8, 32, 64):
                assert 0 <= orc.site(policy, S, 2, int(T)) <= S
