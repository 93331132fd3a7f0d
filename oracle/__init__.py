"""CPU oracle for the tracking-enabled island-model GA (arXiv 2404.10861).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg are the only callers.  The product
package never imports this module, and this module never imports the
product package; they share no code.

The arithmetic lives in ``hsga_oracle.c`` (plain C, single-threaded, built
with gcc by :func:`build`); this file only marshals numpy arrays through
ctypes.  Every function names the step of the paper's generational cycle
(section "Asynchronous Island-model Genetic Algorithm") that it follows; the
C source states the readings used where the paper is silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hsga_oracle.c")
_LIB = os.path.join(_HERE, "libhsga_oracle.so")

STEADY, TILTED, STRETCHED, TRIVIAL, NONE, HYBRID = 0, 1, 2, 3, 4, 5
POLICY_NAMES = {"steady": STEADY, "tilted": TILTED, "stretched": STRETCHED,
                "trivial": TRIVIAL, "none": NONE, "hybrid": HYBRID}
FITNESS_TRAIT, FITNESS_FLOAT = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable C: x86_64 and aarch64)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        # -ffp-contract=off: every float operation is rounded on its own
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-Wall", "-Wextra", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Cfg(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_uint32), ("cols", ctypes.c_uint32),
                ("n", ctypes.c_uint32), ("tournament", ctypes.c_uint32),
                ("policy", ctypes.c_uint32), ("bits", ctypes.c_uint32),
                ("W", ctypes.c_uint32), ("interval", ctypes.c_uint32),
                ("p_ben", ctypes.c_double), ("p_del", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("coarsen", ctypes.c_uint32),
                ("fitness", ctypes.c_uint32), ("sigma", ctypes.c_double),
                ("words", ctypes.c_uint32), ("pad", ctypes.c_uint32)]


@dataclass
class Config:
    """One run's parameters, in the paper's vocabulary.

    rows x cols toroidal island grid, ``n`` agents per island, tournament size,
    surface policy, differentia bit width (S = 64 / bits surface sites),
    sites per level W (tilted / stretched), migration interval (0 = none),
    beneficial / deleterious mutation probabilities, the Philox seed, and
    the annotation interval (temporal coarsening: deposit every coarsen-th
    generation), and the fitness model: FITNESS_TRAIT (unsigned integer,
    mutations of one) or FITNESS_FLOAT (binary32, sign-restricted Gaussian
    mutation amounts of standard deviation ``sigma``), and the surface width
    in 64-bit words (``words``: S = 64 words / bits sites; surfaces are flat
    agent-major arrays of agents x words uint64).
    """
    rows: int = 4
    cols: int = 4
    n: int = 32
    tournament: int = 2
    policy: int = STEADY
    bits: int = 1
    W: int = 2
    interval: int = 1
    p_ben: float = 0.0
    p_del: float = 0.0
    seed: int = 1
    coarsen: int = 1
    fitness: int = 0
    sigma: float = 1.0
    words: int = 1

    @property
    def islands(self) -> int:
        return self.rows * self.cols

    @property
    def agents(self) -> int:
        return self.rows * self.cols * self.n

    @property
    def S(self) -> int:
        return 64 // self.bits

    def _c(self) -> _Cfg:
        return _Cfg(self.rows, self.cols, self.n, self.tournament, self.policy,
                    self.bits, self.W, self.interval, self.p_ben, self.p_del,
                    self.seed, self.coarsen, self.fitness, self.sigma, self.words, 0)


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        u32, u64, i32, i64 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32, ctypes.c_int64
        P = ctypes.POINTER
        _lib.orc_philox4x32_10.argtypes = [u32, u32, P(u32), P(u32)]
        _lib.orc_philox4x64_10.argtypes = [u64, u64, P(u64), P(u64)]
        _lib.orc_site.argtypes = [u32, u32, u32, u64]
        _lib.orc_site.restype = u32
        _lib.orc_lookup.argtypes = [u32, u32, u32, u64, P(i64)]
        _lib.orc_neighbour.argtypes = [P(_Cfg), u32, u32]
        _lib.orc_neighbour.restype = u32
        _lib.orc_emigrate.argtypes = [P(_Cfg), u32, P(u32), P(u32), P(u64), u64, P(u32)]
        _lib.orc_immigrate.argtypes = [P(_Cfg), u32, P(u32), P(i32), ctypes.c_void_p,
                                       P(u32), P(u64), P(u32), u64, ctypes.c_void_p]
        _lib.orc_select.argtypes = [P(_Cfg), u32, P(u32), ctypes.c_void_p, P(u32), P(u64),
                                    ctypes.c_void_p, u64, u64, P(u32), P(u64), ctypes.c_void_p]
        _lib.orc_run_grid.argtypes = [P(_Cfg), P(u32), P(u64), u64, u64, ctypes.c_int,
                                      ctypes.c_void_p]
        _lib.orc_run_grid.restype = ctypes.c_int
        _lib.orc_migrate_grid.argtypes = [P(_Cfg), P(u32), P(u64), u64]
        _lib.orc_migrate_grid.restype = ctypes.c_int
        _lib.orc_run_cone.argtypes = [P(_Cfg), u32, u32, u32, u64, u64, u32, P(u32), P(u64)]
        _lib.orc_run_cone.restype = ctypes.c_int
        _lib.orc_sample_grid.argtypes = [P(_Cfg), P(u32), P(u64), u64, u32, P(u32),
                                         ctypes.c_void_p]
        _lib.orc_sample_grid.restype = ctypes.c_int
        _lib.orc_run_async.argtypes = [P(_Cfg), P(u32), P(u64), P(u32), u64, u32, P(u32)]
        _lib.orc_run_async.restype = ctypes.c_int
        _lib.orc_philox_sweep.argtypes = [u64, u32, u32, u32, u32, u32, P(u32)]
        _lib.orc_philox_sweep.restype = None
        _lib.orc_island_step.argtypes = [P(_Cfg), u32, u64, P(u32), P(u64), P(u32)]
        _lib.orc_island_step.restype = ctypes.c_int
        _lib.orc_run_buffered.argtypes = [P(_Cfg), P(u32), P(u64), P(u32), u64, u32, P(u32),
                                          P(u32), P(u32)]
        _lib.orc_run_buffered.restype = ctypes.c_int
    return _lib


def _p(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _vp(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


# ----------------------------------------------------------------- RNG ---

def philox4x32(key, counter) -> np.ndarray:
    """Philox4x32-10 block (Salmon et al. SC'11); key = (k0, k1)."""
    c = np.ascontiguousarray(counter, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(int(key[0]), int(key[1]), _p(c, ctypes.c_uint32),
                            _p(out, ctypes.c_uint32))
    return out


def philox4x64(key, counter) -> np.ndarray:
    """The same rounds at 64-bit words (pins the round structure)."""
    c = np.ascontiguousarray(counter, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().orc_philox4x64_10(int(key[0]), int(key[1]), _p(c, ctypes.c_uint64),
                            _p(out, ctypes.c_uint64))
    return out


# ------------------------------------------------------------- surface ---

def site(policy: int, S: int, W: int, T: int) -> int:
    """Site written by deposition T (S means: discarded)."""
    return int(lib().orc_site(policy, S, W, T))


def lookup(policy: int, S: int, W: int, T: int) -> np.ndarray:
    """Deposition time held by every site after T depositions (-1 = empty)."""
    out = np.zeros(S, dtype=np.int64)
    lib().orc_lookup(policy, S, W, T, _p(out, ctypes.c_int64))
    return out


# ------------------------------------------------------------------ GA ---

def founders(cfg: Config):
    """Founding population: every trait 0, every surface empty (all zero)."""
    return (np.zeros(cfg.agents, dtype=np.uint32),
            np.zeros(cfg.agents * cfg.words, dtype=np.uint64))


def run(cfg: Config, trait=None, surf=None, G0: int = 0, generations: int = 1,
        premigrated: bool = False, track_parents: bool = False):
    """Synchronous run of ``generations`` full cycles from generation G0.

    Returns (trait, surf, parents); parents is (generations, agents) uint64 of
    pre-migration parent indices, or None.
    """
    if trait is None:
        trait, surf = founders(cfg)
    trait = np.ascontiguousarray(trait, dtype=np.uint32).copy()
    surf = np.ascontiguousarray(surf, dtype=np.uint64).copy()
    parents = (np.zeros((generations, cfg.agents), dtype=np.uint64)
               if track_parents else None)
    c = cfg._c()
    rc = lib().orc_run_grid(ctypes.byref(c), _p(trait, ctypes.c_uint32),
                            _p(surf, ctypes.c_uint64), G0, generations,
                            int(premigrated), _vp(parents))
    if rc != 0:
        raise MemoryError("oracle run failed")
    return trait, surf, parents


def migrate(cfg: Config, trait, surf, G: int):
    """Explicit emigrate + immigrate (steps a1, a2) of generation G."""
    trait = np.ascontiguousarray(trait, dtype=np.uint32).copy()
    surf = np.ascontiguousarray(surf, dtype=np.uint64).copy()
    c = cfg._c()
    if lib().orc_migrate_grid(ctypes.byref(c), _p(trait, ctypes.c_uint32),
                              _p(surf, ctypes.c_uint64), G) != 0:
        raise MemoryError("oracle migrate failed")
    return trait, surf


def run_cone(cfg: Config, row: int, col: int, generations: int, G0: int = 0,
             trait0: int = 0, surf0: int = 0):
    """One island's agents after ``generations`` cycles from a uniform state,
    computed on its dependency cone only (exact at any torus size)."""
    t = np.zeros(cfg.n, dtype=np.uint32)
    s = np.zeros(cfg.n * cfg.words, dtype=np.uint64)
    c = cfg._c()
    rc = lib().orc_run_cone(ctypes.byref(c), row, col, trait0, surf0, G0,
                            generations, _p(t, ctypes.c_uint32),
                            _p(s, ctypes.c_uint64))
    if rc != 0:
        raise ValueError(f"cone run failed ({rc})")
    return t, s


def sample(cfg: Config, trait, surf, G: int, k: int):
    """Step a7: k sampled genomes (k x (2 + 2 words) words: trait, surface
    words as (low, high) pairs, G) and their (island, slot)."""
    trait = np.ascontiguousarray(trait, dtype=np.uint32)
    surf = np.ascontiguousarray(surf, dtype=np.uint64)
    words = np.zeros((k, 2 + 2 * cfg.words), dtype=np.uint32)
    where = np.zeros((k, 2), dtype=np.uint32)
    c = cfg._c()
    rc = lib().orc_sample_grid(ctypes.byref(c), _p(trait, ctypes.c_uint32),
                               _p(surf, ctypes.c_uint64), G, k,
                               _p(words, ctypes.c_uint32), _vp(where))
    if rc == -2:
        raise ValueError("k exceeds the number of islands")
    if rc != 0:
        raise MemoryError("oracle sample failed")
    return words, where


# ------------------------------------------------- free-running migration ---

def run_async(cfg: Config, trait, surf, tcount, G0: int, generations: int, schedule):
    """Free-running migration replayed from a schedule (see hsga_oracle.c):
    schedule[island, g, d] = 1 + the neighbour generation whose emigrant the
    island took from direction d at its generation g (0 = none).  Genomes
    carry their own deposition counters ``tcount``.  Returns (trait, surf,
    tcount)."""
    trait = np.ascontiguousarray(trait, dtype=np.uint32).copy()
    surf = np.ascontiguousarray(surf, dtype=np.uint64).copy()
    tcount = np.ascontiguousarray(tcount, dtype=np.uint32).copy()
    sched = np.ascontiguousarray(schedule, dtype=np.uint32).reshape(-1)
    if sched.size != cfg.islands * generations * 4:
        raise ValueError("schedule must be islands x generations x 4")
    c = cfg._c()
    rc = lib().orc_run_async(ctypes.byref(c), _p(trait, ctypes.c_uint32),
                             _p(surf, ctypes.c_uint64), _p(tcount, ctypes.c_uint32), G0,
                             generations, _p(sched, ctypes.c_uint32))
    if rc == -3:
        raise ValueError("schedule inconsistent with the emigrants' directions or causality")
    if rc != 0:
        raise MemoryError("oracle async run failed")
    return trait, surf, tcount


def philox_sweep(seed: int, c0: int, count: int, c1: int, c2: int, c3: int) -> np.ndarray:
    """Philox4x32-10 blocks for counters (c0 + i, c1, c2, c3): (count, 4) uint32."""
    out = np.zeros((count, 4), dtype=np.uint32)
    lib().orc_philox_sweep(seed, c0, count, c1, c2, c3, _p(out, ctypes.c_uint32))
    return out


def island_step(cfg: Config, island: int, G: int, trait, surf, tcount) -> None:
    """One generation (a3-a6) of one island with per-genome deposition
    counters, in place on the whole-grid arrays (uint32, uint64, uint32,
    C-contiguous)."""
    for a, t in ((trait, np.uint32), (surf, np.uint64), (tcount, np.uint32)):
        if a.dtype != t or not a.flags.c_contiguous:
            raise TypeError("island_step works in place on contiguous arrays")
    c = cfg._c()
    if lib().orc_island_step(ctypes.byref(c), island, G, _p(trait, ctypes.c_uint32),
                             _p(surf, ctypes.c_uint64), _p(tcount, ctypes.c_uint32)):
        raise MemoryError("oracle island step failed")


def run_buffered(cfg: Config, trait, surf, tcount, G0: int, generations: int, log):
    """Buffered free-running migration (per-neighbour emigration buffers of
    one genome, immigration buffers of four) replayed from a log (see
    hsga_oracle.c): log[island, g, d] = (post number taken from direction d)
    << 1 | (1 if the island posted toward d).  Returns (trait, surf, tcount,
    chan, inbuf): chan[island, d] = (posts made toward d, last post number
    taken from d, genomes waiting), inbuf[island, d, j] = (trait, surface lo,
    surface hi, T) of waiting genome j."""
    trait = np.ascontiguousarray(trait, dtype=np.uint32).copy()
    surf = np.ascontiguousarray(surf, dtype=np.uint64).copy()
    tcount = np.ascontiguousarray(tcount, dtype=np.uint32).copy()
    lg = np.ascontiguousarray(log, dtype=np.uint32).reshape(-1)
    if lg.size != cfg.islands * generations * 4:
        raise ValueError("log must be islands x generations x 4")
    chan = np.zeros((cfg.islands, 4, 3), dtype=np.uint32)
    inbuf = np.zeros((cfg.islands, 4, 4, 4), dtype=np.uint32)
    c = cfg._c()
    rc = lib().orc_run_buffered(ctypes.byref(c), _p(trait, ctypes.c_uint32),
                                _p(surf, ctypes.c_uint64), _p(tcount, ctypes.c_uint32), G0,
                                generations, _p(lg, ctypes.c_uint32),
                                _p(chan, ctypes.c_uint32), _p(inbuf, ctypes.c_uint32))
    if rc == -3:
        raise ValueError("log breaks the buffered protocol or its causality")
    if rc != 0:
        raise MemoryError("oracle buffered run failed")
    return trait, surf, tcount, chan, inbuf


def sync_schedule(cfg: Config, G0: int, generations: int) -> np.ndarray:
    """The schedule under which free-running migration reproduces the
    synchronous run: at generation g every island takes, from each neighbour,
    that neighbour's generation-g emigrant if it was aimed at the island."""
    I = cfg.islands
    out = np.zeros((I, generations, 4), dtype=np.uint32)
    for g in range(generations):
        G = G0 + g
        if not (cfg.interval > 0 and G % cfg.interval == 0):
            continue
        dirs = np.array([int(philox4x32((cfg.seed & 0xFFFFFFFF, cfg.seed >> 32),
                                        (0xFFFFFFFF, i, G, 0))[1]) >> 30 for i in range(I)])
        for i in range(I):
            for d in range(4):
                nb = neighbour(cfg, i, d)
                if dirs[nb] == (d + 2) % 4:
                    out[i, g, d] = g + 1
    return out


# ------------------------------------------- pieces for band decomposition ---

def emigrate(cfg: Config, gid, trait, surf, G: int) -> np.ndarray:
    """Step a1 for local islands with global ids ``gid``: (n_local, 4 + 2 words)
    records (trait, direction, source index low/high, surface words)."""
    gid = np.ascontiguousarray(gid, dtype=np.uint32)
    rec = np.zeros((len(gid), 4 + 2 * cfg.words), dtype=np.uint32)
    c = cfg._c()
    lib().orc_emigrate(ctypes.byref(c), len(gid), _p(gid, ctypes.c_uint32),
                       _p(np.ascontiguousarray(trait, dtype=np.uint32), ctypes.c_uint32),
                       _p(np.ascontiguousarray(surf, dtype=np.uint64), ctypes.c_uint64),
                       G, _p(rec, ctypes.c_uint32))
    return rec


def immigrate_select(cfg: Config, gid, nbr, active, trait, surf, rec, G: int):
    """Steps a2-a6 for the active local islands; returns the children."""
    gid = np.ascontiguousarray(gid, dtype=np.uint32)
    nbr = np.ascontiguousarray(nbr, dtype=np.int32)
    active = np.ascontiguousarray(active, dtype=np.uint8)
    trait = np.ascontiguousarray(trait, dtype=np.uint32).copy()
    surf = np.ascontiguousarray(surf, dtype=np.uint64).copy()
    rec = np.ascontiguousarray(rec, dtype=np.uint32)
    c = cfg._c()
    if cfg.interval > 0 and G % cfg.interval == 0:
        lib().orc_immigrate(ctypes.byref(c), len(gid), _p(gid, ctypes.c_uint32),
                            _p(nbr, ctypes.c_int32), _vp(active),
                            _p(trait, ctypes.c_uint32), _p(surf, ctypes.c_uint64),
                            _p(rec, ctypes.c_uint32), G, None)
    t2, s2 = trait.copy(), surf.copy()
    lib().orc_select(ctypes.byref(c), len(gid), _p(gid, ctypes.c_uint32), _vp(active),
                     _p(trait, ctypes.c_uint32), _p(surf, ctypes.c_uint64), None, G, G,
                     _p(t2, ctypes.c_uint32), _p(s2, ctypes.c_uint64), None)
    return t2, s2


def neighbour(cfg: Config, island: int, d: int) -> int:
    c = cfg._c()
    return int(lib().orc_neighbour(ctypes.byref(c), island, d))
