"""GPU parity: the CUDA path, called through the C-ABI, against the CPU oracle
on identical seeded inputs.  All arithmetic is integer, so the bar is
bit-exact on every genome word (traits, 64-bit surfaces), every sampled
record and every (island, slot) index.

Cases: the tiny workload in full (4x4 islands x 32 agents, steady 64x1-bit
surface, 2,000 generations); a prefix of the mid-grid workload (64x64 x 32,
32 two-bit differentiae) under every policy with adaptation on and off;
ragged and degenerate shapes (1x1, 1xC, Rx1 tori, 1, 17, 33, 64 agents,
tournaments of 1..7, every differentia width); explicit migration;
checkpoint/resume; sampling through both sampler paths; and the full
wafer-shaped grid (512x1024 x 32 = 16.8M agents, the benchmark's launch
configuration) checked island by island against the oracle's dependency-cone
runs, plus properties that hold at any size.
"""
import numpy as np
import pytest

from paper_2404_10861_gb300 import inputs

pytestmark = pytest.mark.gpu

KERNELS = {"streamed": 1, "resident": 2, "resident_grid": 3}


@pytest.fixture(scope="module")
def hb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_10861_gb300 import _build, binding
    _build.build()
    return binding


def oracle_cfg(orc, kw):
    pol = kw.get("policy", "steady")
    pol = orc.POLICY_NAMES[pol] if isinstance(pol, str) else pol
    return orc.Config(rows=kw.get("rows", 4), cols=kw.get("cols", 4), n=kw.get("n", 32),
                      tournament=kw.get("tournament", 2), policy=pol, bits=kw.get("bits", 1),
                      W=kw.get("W", 2), interval=kw.get("interval", 1),
                      p_ben=kw.get("p_ben", 0.0), p_del=kw.get("p_del", 0.0),
                      seed=kw.get("seed", 1), coarsen=kw.get("coarsen", 1))


def gpu_run(hb, kw, kernel, trait=None, surf=None, G0=0, chunks=(1,)):
    g = hb.Grid(kernel=KERNELS[kernel], **kw)
    try:
        if trait is not None:
            g.set_population(trait, surf, G0)
        for c in chunks:
            g.run(c)
        g.sync()
        st = g.stats()
        t, s = g.population()
        return t, s, st
    finally:
        g.close()


def assert_same(a, b, what):
    ta, sa = a
    tb, sb = b
    bad_t = np.nonzero(ta != tb)[0]
    bad_s = np.nonzero(sa != sb)[0]
    assert len(bad_t) == 0, f"{what}: {len(bad_t)} traits differ, first at agent {bad_t[:5]}"
    assert len(bad_s) == 0, f"{what}: {len(bad_s)} surfaces differ, first at agent {bad_s[:5]}"


@pytest.mark.parametrize("kernel", ["streamed", "resident", "resident_grid"])
def test_tiny_workload_full_run(hb, orc, kernel):
    kw = dict(rows=4, cols=4, n=32, tournament=2, policy="steady", bits=1, p_ben=0.0, seed=1)
    want = orc.run(oracle_cfg(orc, kw), generations=2000)[:2]
    t, s, st = gpu_run(hb, kw, kernel, chunks=(1, 99, 1900))
    assert st["generation"] == 2000
    assert st["kernel"] == KERNELS[kernel]            # tiny grid: one block when resident
    assert_same((t, s), want, f"tiny/{kernel}")
    assert not t.any()                      # neutral: traits stay 0
    assert s.any()


@pytest.mark.parametrize("kernel", ["streamed", "resident"])
@pytest.mark.parametrize("policy", ["steady", "tilted", "stretched"])
@pytest.mark.parametrize("p_ben", [1e-3, 0.0])
def test_mid_grid_prefix(hb, orc, kernel, policy, p_ben):
    kw = dict(rows=64, cols=64, n=32, tournament=2, policy=policy, bits=2, p_ben=p_ben, seed=2)
    G = 120
    want = orc.run(oracle_cfg(orc, kw), generations=G)[:2]
    t, s, _ = gpu_run(hb, kw, kernel, chunks=(G,))
    assert_same((t, s), want, f"mid/{kernel}/{policy}/{p_ben}")


EDGE = [
    dict(rows=1, cols=1, n=32),
    dict(rows=1, cols=5, n=17, tournament=3),
    dict(rows=3, cols=1, n=33, tournament=5, policy="tilted", bits=2),
    dict(rows=2, cols=2, n=64, tournament=7, policy="stretched", bits=4, W=4),
    dict(rows=5, cols=7, n=1, tournament=2, policy="trivial", bits=8),
    dict(rows=6, cols=9, n=24, tournament=1, policy="none", p_ben=0.05),
    dict(rows=4, cols=6, n=32, tournament=2, policy="tilted", bits=1, W=1, interval=3,
         p_ben=0.01, p_del=0.02),
    dict(rows=7, cols=3, n=48, tournament=6, policy="steady", bits=8, interval=0, p_ben=0.1,
         p_del=0.1),
    dict(rows=9, cols=11, n=31, tournament=4, policy="tilted", bits=4, W=2, p_ben=0.5, p_del=0.5),
    dict(rows=2, cols=3, n=40, tournament=2, policy="steady", bits=1, p_del=1.0),
    dict(rows=6, cols=7, n=32, tournament=2, policy="hybrid", bits=1, W=2, p_ben=0.01),
    dict(rows=5, cols=5, n=20, tournament=3, policy="hybrid", bits=2, W=4, coarsen=3),
    dict(rows=4, cols=9, n=32, tournament=2, policy="tilted", bits=1, coarsen=5, p_ben=0.02),
    dict(rows=3, cols=3, n=64, tournament=2, policy="steady", bits=4, coarsen=2, interval=2),
]


@pytest.mark.parametrize("kernel", ["streamed", "resident", "resident_grid"])
@pytest.mark.parametrize("case", range(len(EDGE)))
def test_edge_shapes_from_random_states(hb, orc, kernel, case):
    kw = dict(EDGE[case], seed=100 + case)
    c = oracle_cfg(orc, kw)
    if case % 2:
        trait, surf = inputs.random_population(c.agents, seed=case)
    else:
        trait, surf = inputs.small_trait_population(c.agents, seed=case, levels=3)
    if kw.get("policy") == "none":
        surf = np.zeros_like(surf)
    for G0 in (0, 63, 1023, 2**20 - 5):
        want = orc.run(c, trait, surf, G0=G0, generations=37)[:2]
        t, s, _ = gpu_run(hb, kw, kernel, trait, surf, G0=G0, chunks=(5, 32))
        assert_same((t, s), want, f"edge{case}/{kernel}/G0={G0}")


@pytest.mark.parametrize("kernel", ["streamed", "resident", "resident_grid"])
def test_explicit_migrate_then_run(hb, orc, kernel):
    kw = dict(rows=5, cols=8, n=20, tournament=2, policy="tilted", bits=2, p_ben=0.02, seed=9)
    c = oracle_cfg(orc, kw)
    trait, surf = inputs.small_trait_population(c.agents, seed=5)
    G0 = 77
    g = hb.Grid(kernel=KERNELS[kernel], **kw)
    try:
        g.set_population(trait, surf, G0)
        g.migrate()
        g.sync()
        mt, ms = orc.migrate(c, trait, surf, G0)
        assert_same(g.population(), (mt, ms), "migrate")
        with pytest.raises(hb.HsgaError):
            g.migrate()                                  # already migrated this generation
        g.run(11)
        g.sync()
        want = orc.run(c, mt, ms, G0=G0, generations=11, premigrated=True)[:2]
        assert_same(g.population(), want, "migrate+run")
    finally:
        g.close()


@pytest.mark.parametrize("kernel", ["streamed", "resident"])
def test_checkpoint_resume_is_bit_identical(hb, kernel):
    kw = dict(rows=16, cols=16, n=32, policy="tilted", bits=1, p_ben=1e-3, seed=3,
              kernel=KERNELS[kernel])
    a = hb.Grid(**kw)
    b = hb.Grid(**kw)
    try:
        a.run(300)
        blob = hb.hsga_save(a.handle)
        a.run(200)
        a.sync()
        b.run(1)
        hb.hsga_load(b.handle, blob)
        assert b.stats()["generation"] == 300
        b.run(200)
        b.sync()
        assert_same(a.population(), b.population(), "resume")
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("k", [0, 1, 10, 256, 1000])
def test_sample_matches_oracle(hb, orc, k):
    kw = dict(rows=32, cols=32, n=32, policy="steady", bits=1, p_ben=1e-3, seed=4)
    c = oracle_cfg(orc, kw)
    trait, surf = inputs.random_population(c.agents, seed=11)
    G = 4321
    g = hb.Grid(**kw)
    try:
        g.set_population(trait, surf, G)
        w, where = g.sample(k)
        if k:
            ow, owhere = orc.sample(c, trait, surf, G, k)
            assert np.array_equal(w, ow)
            assert np.array_equal(where, owhere)
        with pytest.raises(hb.HsgaError):
            g.sample(c.islands + 1)
        w, where = g.sample(c.islands)                 # every island exactly once
        assert sorted(where[:, 0]) == list(range(c.islands))
    finally:
        g.close()


def test_sample_large_k_serial_path(hb, orc):
    kw = dict(rows=128, cols=128, n=8, policy="tilted", bits=1, seed=8)
    c = oracle_cfg(orc, kw)
    trait, surf = inputs.random_population(c.agents, seed=12)
    g = hb.Grid(**kw)
    try:
        g.set_population(trait, surf, 99)
        for k in (12288, 12289, 16384):
            w, where = g.sample(k)
            ow, owhere = orc.sample(c, trait, surf, 99, k)
            assert np.array_equal(w, ow), k
            assert np.array_equal(where, owhere), k
    finally:
        g.close()


def test_sites_kernel_matches_oracle(hb, orc):
    import torch
    out = torch.zeros(70000, dtype=torch.int32, device="cuda")
    for policy in (0, 1, 2, 3):
        for S, W in ((64, 2), (32, 2), (16, 4), (8, 1)):
            for T0 in (0, 2**31 - 1000, 2**32 - 70002):
                hb.hsga_sites_device(policy, S, W, T0, 70000, out)
                torch.cuda.synchronize()
                got = out.cpu().numpy().astype(np.int64) & 0xFFFFFFFF
                for i in list(range(0, 70000, 97)) + [69999]:
                    assert got[i] == orc.site(policy, S, W, T0 + i), (policy, S, W, T0 + i)


def test_torch_allocator_and_stream(hb, orc):
    import torch
    hb.use_torch_allocator()
    try:
        stream = torch.cuda.Stream()
        kw = dict(rows=8, cols=8, n=32, policy="tilted", bits=2, p_ben=1e-3, seed=5)
        c = oracle_cfg(orc, kw)
        trait, surf = inputs.small_trait_population(c.agents, seed=2)
        g = hb.Grid(stream=stream.cuda_stream, **kw)
        try:
            td = torch.from_numpy(trait.view(np.int32)).cuda()
            sd = torch.from_numpy(surf.view(np.int64)).cuda()
            torch.cuda.synchronize()
            g.set_population(td, sd, 10)                  # device sources
            g.run(25)
            to = torch.empty_like(td)
            so = torch.empty_like(sd)
            hb.hsga_get_population(g.handle, to, so)     # device destinations
            g.sync()
            got = (to.cpu().numpy().view(np.uint32), so.cpu().numpy().view(np.uint64))
            assert_same(got, orc.run(c, trait, surf, G0=10, generations=25)[:2], "torch")
            words = torch.zeros((64, 4), dtype=torch.int32, device="cuda")
            where = torch.zeros((64, 2), dtype=torch.int32, device="cuda")
            hb.hsga_sample_surfaces(g.handle, 64, words, where)   # device outputs
            g.sync()
            ow, owhere = orc.sample(c, got[0], got[1], 35, 64)
            assert np.array_equal(words.cpu().numpy().view(np.uint32), ow)
            assert np.array_equal(where.cpu().numpy().view(np.uint32), owhere)
        finally:
            g.close()
    finally:
        hb.use_default_allocator()


def test_kernel_choice(hb):
    g = hb.Grid(rows=64, cols=64, n=32)
    try:
        assert g.stats()["kernel"] == 3                   # mid grid: cooperative resident grid
    finally:
        g.close()
    g = hb.Grid(rows=4, cols=4, n=32)
    try:
        assert g.stats()["kernel"] == 2                   # tiny grid: one resident block
    finally:
        g.close()


# ------------------------------------------------ wafer-shaped workload ---
WAFER = dict(rows=512, cols=1024, n=32, tournament=2, policy="tilted", bits=1, p_ben=1e-3,
             seed=1)


@pytest.fixture(scope="module")
def wafer(hb):
    g = hb.Grid(kernel=KERNELS["streamed"], **WAFER)
    yield g
    g.close()


def test_wafer_grid_cones(hb, orc, wafer):
    """Full size, the benchmark's kernel: islands sampled over the torus
    (corners, edges, interior) against exact dependency-cone oracle runs."""
    c = oracle_cfg(orc, WAFER)
    G = 6
    wafer.set_population(*inputs.founders(c.agents), 0)
    wafer.run(G)
    wafer.sync()
    t, s = wafer.population()
    rng = np.random.default_rng(0)
    picks = [(0, 0), (0, 1023), (511, 0), (511, 1023), (255, 512), (1, 1)]
    picks += [(int(r), int(q)) for r, q in zip(rng.integers(0, 512, 24), rng.integers(0, 1024, 24))]
    for r, q in picks:
        ot, os_ = orc.run_cone(c, r, q, G)
        i = r * c.cols + q
        assert np.array_equal(t[i * c.n:(i + 1) * c.n], ot), (r, q)
        assert np.array_equal(s[i * c.n:(i + 1) * c.n], os_), (r, q)


def test_wafer_grid_properties_after_long_run(hb, orc, wafer):
    """Properties at any size: each generation adds at most one to a trait;
    sites never written hold no bits; sampled records agree with the
    population they came from."""
    c = oracle_cfg(orc, WAFER)
    wafer.set_population(*inputs.founders(c.agents), 0)
    G = 300
    wafer.run(G)
    wafer.sync()
    t, s = wafer.population()
    assert 0 < t.mean() <= t.max() <= G                  # at most +1 per generation
    times = orc.lookup(c.policy, c.S, c.W, G)
    empty = np.nonzero(times < 0)[0]
    mask = np.uint64(sum(1 << int(p) for p in empty))
    assert not np.any(s & mask)
    w, where = wafer.sample(10000)
    ow, owhere = orc.sample(c, t, s, G, 10000)
    assert np.array_equal(w, ow)
    assert np.array_equal(where, owhere)
