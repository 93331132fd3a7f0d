"""Pins for the oracle's buffered free-running migration replay.

The paper's WSE islands exchange genomes through per-neighbour buffers with
completion flags (section "Asynchronous Island-model Genetic Algorithm":
one-genome send buffers, four-genome receive buffers, the main cycle copies
completed receive buffers into the population, then refills completed send
buffers, then evolves).  The oracle replays a logged run in causal order.
It is pinned here by

* a case worked by hand (one island that is its own neighbour, one agent,
  every child one step fitter): the trait lags the generation count by one
  for every four immigrations;
* an independent event simulation written in this file, which runs the
  protocol in real-time order (islands advance one generation at a time in a
  random interleaving, each seeing only what has been sent so far, sometimes
  missing it) and writes the log; the oracle's causal replay of that log must
  reproduce the simulation's population, counters, channels and waiting
  buffers exactly;
* logs that break the protocol (a skipped post number, a take before its
  post, a post before its acknowledgement) must be rejected.
"""
import numpy as np
import pytest


def cfg(orc, **kw):
    base = dict(rows=3, cols=4, n=8, tournament=2, policy=orc.TILTED, bits=1, W=2,
                interval=1, p_ben=0.05, p_del=0.02, seed=11)
    base.update(kw)
    return orc.Config(**base)


def test_self_neighbour_one_agent_by_hand(orc):
    # 1x1 torus: all four neighbours are the island itself; n = 1, so every
    # draw picks slot 0; p_ben = 1 adds one to every child.  Generation g
    # takes post g (sent at g - 1) on every channel and posts again, so each
    # channel's buffer fills at g = 4, 8, 12, ... and then holds posts sent
    # at g - 4 .. g - 1; placement leaves the last, sent at g - 1, whose
    # trait is one behind.  After N generations the trait (and the counter,
    # which also grows by one per generation and is carried by the copy) is
    # N - floor((N - 1) / 4).
    c = orc.Config(rows=1, cols=1, n=1, tournament=1, policy=orc.NONE, bits=1, W=2,
                   interval=1, p_ben=1.0, p_del=0.0, seed=7)
    for N in (1, 4, 5, 13, 40):
        log = np.zeros((1, N, 4), np.uint32)
        for g in range(N):
            log[0, g, :] = (g << 1) | 1
        t, s, T, chan, _ = orc.run_buffered(c, np.zeros(1, np.uint32), np.zeros(1, np.uint64),
                                            np.zeros(1, np.uint32), 0, N, log)
        assert int(t[0]) == N - (N - 1) // 4 and int(T[0]) == int(t[0]), N
        assert np.all(chan[0, :, 0] == N) and np.all(chan[0, :, 1] == N - 1)
        assert np.all(chan[0, :, 2] == (N - 1) % 4)


def _uindex(w, n):
    return (int(w) * n) >> 32


def simulate(orc, c, trait, surf, tcount, G0, gens, seed, p_miss=0.3, speed=None):
    """The protocol in real-time order.  Returns the final state and the log."""
    rng = np.random.default_rng(seed)
    I, n = c.islands, c.n
    key = (c.seed & 0xFFFFFFFF, c.seed >> 32)
    trait, surf, tcount = trait.copy(), surf.copy(), tcount.copy()
    nb = np.array([[orc.neighbour(c, i, d) for d in range(4)] for i in range(I)])
    mail = np.zeros((I, 4, 4), np.uint32)     # genome in flight per channel
    posts = np.zeros((I, 4), np.int64)        # posts made on channel (i, d)
    ack = np.zeros((I, 4), np.int64)          # last post of (i, d) its receiver took
    taken = np.zeros((I, 4), np.int64)        # last post taken from direction d
    count = np.zeros((I, 4), np.int64)
    buf = np.zeros((I, 4, 4, 4), np.uint32)
    done = np.zeros(I, np.int64)
    log = np.zeros((I, gens, 4), np.uint32)
    speed = np.ones(I) if speed is None else np.asarray(speed, float)
    while (done < gens).any():
        live = np.nonzero(done < gens)[0]
        i = int(rng.choice(live, p=speed[live] / speed[live].sum()))
        g = int(done[i])
        G = G0 + g
        if c.interval > 0 and G % c.interval == 0:
            for d in range(4):
                src, sd = int(nb[i, d]), (d + 2) % 4
                if posts[src, sd] > taken[i, d] and rng.random() >= p_miss:
                    k = taken[i, d] + 1
                    buf[i, d, count[i, d]] = mail[src, sd]
                    count[i, d] += 1
                    taken[i, d] = k
                    ack[src, sd] = k
                    log[i, g, d] |= np.uint32(k << 1)
            for d in range(4):
                if count[i, d] == 4:
                    v = orc.philox4x32(key, (0xFFFFFFFE, i, G, 1 + d))
                    for j in range(4):
                        a = i * n + _uindex(v[j], n)
                        h = buf[i, d, j]
                        trait[a] = h[0]
                        surf[a] = np.uint64(int(h[1]) | (int(h[2]) << 32))
                        tcount[a] = h[3]
                    count[i, d] = 0
            w = orc.philox4x32(key, (0xFFFFFFFF, i, G, 0))
            for d in range(4):
                if ack[i, d] == posts[i, d] and rng.random() >= p_miss:
                    a = i * n + _uindex(w[d], n)
                    s = int(surf[a])
                    mail[i, d] = (trait[a], s & 0xFFFFFFFF, s >> 32, tcount[a])
                    posts[i, d] += 1
                    log[i, g, d] |= np.uint32(1)
        orc.island_step(c, i, G, trait, surf, tcount)
        done[i] += 1
    chan = np.stack([posts, taken, count], axis=-1).astype(np.uint32)
    return trait, surf, tcount, chan, buf, log


SHAPES = [
    dict(rows=3, cols=4, n=8),
    dict(rows=1, cols=5, n=6, tournament=3, policy=2),          # N/S neighbour is itself
    dict(rows=2, cols=2, n=4, tournament=5, policy=5, bits=2),  # hybrid, both wraps
    dict(rows=4, cols=3, n=32, interval=2, policy=0),
    dict(rows=1, cols=1, n=3, policy=3, bits=4),
]


@pytest.mark.parametrize("shape", range(len(SHAPES)))
def test_replay_matches_event_simulation(orc, shape):
    c = cfg(orc, **SHAPES[shape])
    rng = np.random.default_rng(shape)
    trait = rng.integers(0, 6, c.agents).astype(np.uint32)
    surf = rng.integers(0, 2**63, c.agents, dtype=np.uint64)
    tcount = np.full(c.agents, 50, np.uint32)
    gens = 40
    speed = rng.uniform(0.3, 1.0, c.islands)                  # uneven island clocks
    st, ss, sT, schan, sbuf, log = simulate(orc, c, trait, surf, tcount, 50, gens, shape,
                                            speed=speed)
    assert (log >> 1).max() > 4                               # buffers filled and placed
    ot, os_, oT, ochan, obuf = orc.run_buffered(c, trait, surf, tcount, 50, gens, log)
    assert np.array_equal(ot, st) and np.array_equal(os_, ss) and np.array_equal(oT, sT)
    assert np.array_equal(ochan, schan)
    waiting = np.arange(4)[None, None, :] < ochan[:, :, 2:3]
    assert np.array_equal(obuf[waiting], sbuf[waiting])
    # nothing is lost: every post but the one in flight has been taken
    nb = np.array([[orc.neighbour(c, i, d) for d in range(4)] for i in range(c.islands)])
    for i in range(c.islands):
        for d in range(4):
            lag = int(ochan[i, d, 0]) - int(ochan[nb[i, d], (d + 2) % 4, 1])
            assert lag in (0, 1)


def test_broken_logs_are_rejected(orc):
    c = cfg(orc)
    rng = np.random.default_rng(3)
    trait = np.zeros(c.agents, np.uint32)
    surf = np.zeros(c.agents, np.uint64)
    tcount = np.zeros(c.agents, np.uint32)
    _, _, _, _, _, log = simulate(orc, c, trait, surf, tcount, 0, 20, 5)
    orc.run_buffered(c, trait, surf, tcount, 0, 20, log)      # the valid log replays
    takes = np.argwhere((log >> 1) > 1)
    i, g, d = takes[0]
    bad = log.copy()
    bad[i, g, d] += 2                                         # skips a post number
    with pytest.raises(ValueError):
        orc.run_buffered(c, trait, surf, tcount, 0, 20, bad)
    bad = log.copy()
    bad[:, :, :] &= np.uint32(1)
    bad[0, 0, 0] |= np.uint32(1 << 1)                         # takes before any post
    with pytest.raises(ValueError):
        orc.run_buffered(c, trait, surf, tcount, 0, 20, bad)
    bad = np.zeros_like(log)
    bad[:, 0, :] = 1
    bad[:, 1, :] = 1                                          # posts again without an ack
    with pytest.raises(ValueError):
        orc.run_buffered(c, trait, surf, tcount, 0, 20, bad)
