"""ctypes binding of ``libhsga.so`` (C-ABI declared in ``include/hsga.h``).

Argument marshalling only: every step of the generation cycle runs in the
library's CUDA kernels.  The functions keep the C names.  Arrays may be numpy
arrays (host memory) or CUDA torch tensors (device memory); the library tells
them apart.  The library must exist (``__graft_entry__.build()`` or
``python -m paper_2404_10861_gb300._build``); importing a missing or stale
library raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import _build

STEADY, TILTED, STRETCHED, TRIVIAL, NONE, HYBRID = 0, 1, 2, 3, 4, 5
POLICIES = {"steady": STEADY, "tilted": TILTED, "stretched": STRETCHED,
            "trivial": TRIVIAL, "none": NONE, "hybrid": HYBRID}
KERNEL_AUTO, KERNEL_STREAMED, KERNEL_RESIDENT, KERNEL_RESIDENT_GRID = 0, 1, 2, 3

STATUS = {0: "ok", -1: "invalid argument", -2: "device allocation failed",
          -3: "CUDA runtime error", -4: "kernel reported an inconsistent state",
          -5: "bounded device wait timed out", -6: "unsupported",
          -7: "call waits for a stream under graph capture"}


class HsgaError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {STATUS.get(status, status)} ({status})")
        self.status = status


class hsga_config(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_uint32), ("cols", ctypes.c_uint32),
                ("agents_per_island", ctypes.c_uint32), ("tournament_size", ctypes.c_uint32),
                ("surface_policy", ctypes.c_uint32), ("differentia_bits", ctypes.c_uint32),
                ("sites_per_level", ctypes.c_uint32), ("migration_interval", ctypes.c_uint32),
                ("p_beneficial", ctypes.c_double), ("p_deleterious", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("kernel", ctypes.c_uint32),
                ("deposit_interval", ctypes.c_uint32), ("migration_mode", ctypes.c_uint32),
                ("fitness", ctypes.c_uint32), ("mutation_sigma", ctypes.c_double),
                ("surface_words", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class hsga_stats(ctypes.Structure):
    _fields_ = [("generation", ctypes.c_uint64), ("replications", ctypes.c_uint64),
                ("kernel_launches", ctypes.c_uint64), ("kernel", ctypes.c_uint32),
                ("islands_per_warp", ctypes.c_uint32), ("warps_per_block", ctypes.c_uint32),
                ("blocks", ctypes.c_uint32), ("fossils", ctypes.c_uint32),
                ("fossils_dropped", ctypes.c_uint64)]


class hsga_batch_run_info(ctypes.Structure):
    _fields_ = [("generation", ctypes.c_uint64), ("budget", ctypes.c_uint64),
                ("agents", ctypes.c_uint64), ("done", ctypes.c_uint32), ("live", ctypes.c_uint32)]


class hsga_batch_stats(ctypes.Structure):
    _fields_ = [("tick", ctypes.c_uint64), ("replications", ctypes.c_uint64),
                ("kernel_launches", ctypes.c_uint64), ("phases", ctypes.c_uint64),
                ("device_bytes", ctypes.c_uint64), ("live_runs", ctypes.c_uint32),
                ("active_runs", ctypes.c_uint32), ("threads_per_block", ctypes.c_uint32),
                ("blocks", ctypes.c_uint32)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)

# Every symbol include/hsga.h declares, with its ctypes signature.
_SIGS = {
    "hsga_version": ([], ctypes.c_int),
    "hsga_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "hsga_set_allocator": ([ALLOC_FN, FREE_FN, ctypes.c_void_p], ctypes.c_int),
    "hsga_init_grid": ([ctypes.POINTER(hsga_config), ctypes.c_void_p,
                        ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "hsga_set_population": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                             ctypes.c_uint64], ctypes.c_int),
    "hsga_get_population": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "hsga_run_generations": ([ctypes.c_void_p, ctypes.c_uint64], ctypes.c_int),
    "hsga_migrate": ([ctypes.c_void_p], ctypes.c_int),
    "hsga_sample_surfaces": ([ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p,
                              ctypes.c_void_p], ctypes.c_int),
    "hsga_set_fossil_sampling": ([ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32,
                                  ctypes.c_uint32], ctypes.c_int),
    "hsga_get_fossils": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32,
                          ctypes.POINTER(ctypes.c_uint32)], ctypes.c_int),
    "hsga_get_counters": ([ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "hsga_set_async_log": ([ctypes.c_void_p, ctypes.c_uint32], ctypes.c_int),
    "hsga_get_async_log": ([ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "hsga_get_migration_buffers": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
                                   ctypes.c_int),
    "hsga_wait_probe": ([ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64,
                         ctypes.POINTER(ctypes.c_uint64), ctypes.c_void_p], ctypes.c_int),
    "hsga_philox_device": ([ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                            ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p],
                           ctypes.c_int),
    "hsga_reconstruct": ([ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                          ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32,
                          ctypes.c_void_p,
                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32,
                          ctypes.POINTER(ctypes.c_uint32), ctypes.c_void_p], ctypes.c_int),
    "hsga_synchronize": ([ctypes.c_void_p], ctypes.c_int),
    "hsga_get_stats": ([ctypes.c_void_p, ctypes.POINTER(hsga_stats)], ctypes.c_int),
    "hsga_save": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)],
                  ctypes.c_int),
    "hsga_load": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t], ctypes.c_int),
    "hsga_destroy": ([ctypes.c_void_p], None),
    "hsga_site": ([ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64],
                  ctypes.c_uint32),
    "hsga_lookup": ([ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64,
                     ctypes.c_void_p], ctypes.c_int),
    "hsga_sites_device": ([ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64,
                           ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "hsga_batch_create": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "hsga_batch_add": ([ctypes.c_void_p, ctypes.POINTER(hsga_config), ctypes.c_uint64,
                        ctypes.POINTER(ctypes.c_uint32)], ctypes.c_int),
    "hsga_batch_run": ([ctypes.c_void_p, ctypes.c_uint64], ctypes.c_int),
    "hsga_batch_info": ([ctypes.c_void_p, ctypes.c_uint32, ctypes.POINTER(hsga_batch_run_info)],
                        ctypes.c_int),
    "hsga_batch_get_population": ([ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p,
                                   ctypes.c_void_p], ctypes.c_int),
    "hsga_batch_sample": ([ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p,
                           ctypes.c_void_p], ctypes.c_int),
    "hsga_batch_remove": ([ctypes.c_void_p, ctypes.c_uint32], ctypes.c_int),
    "hsga_batch_get_stats": ([ctypes.c_void_p, ctypes.POINTER(hsga_batch_stats)], ctypes.c_int),
    "hsga_run_footprint": ([ctypes.POINTER(hsga_config), ctypes.POINTER(ctypes.c_uint64)],
                           ctypes.c_int),
    "hsga_batch_synchronize": ([ctypes.c_void_p], ctypes.c_int),
    "hsga_batch_destroy": ([ctypes.c_void_p], None),
    "hsga_set_octet_slice": ([ctypes.c_void_p, ctypes.c_uint32], ctypes.c_int),
    "hsga_philox_throughput": ([ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p,
                                ctypes.c_void_p], ctypes.c_int),
    "hsga_run_generations_noalloc": ([ctypes.POINTER(hsga_config), ctypes.c_uint64,
                                      ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p], ctypes.c_int),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def lib():
    """Loads libhsga.so, raising if it is missing (no fallback exists)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(path)
        for name, (argt, rest) in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = argt
            fn.restype = rest
        _lib = L
    return _lib


def _check(status: int, what: str):
    if status != 0:
        raise HsgaError(status, what)


def _ptr(a):
    """Raw address of a numpy array or a torch tensor (host or device)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(a.ctypes.data)
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    raise TypeError(f"unsupported buffer {type(a)}")


# ------------------------------------------------------------- allocator ---
_alloc_keep = []


def use_torch_allocator():
    """Routes the library's device allocations through torch's caching
    allocator (PyTorch provides device memory and streams)."""
    import torch

    def _alloc(nbytes, stream, ctx):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), stream=stream or 0))
        except Exception:
            return None

    def _free(ptr, stream, ctx):
        if ptr:
            torch.cuda.caching_allocator_delete(int(ptr))

    cbs = (ALLOC_FN(_alloc), FREE_FN(_free))
    _alloc_keep.append(cbs)
    _check(lib().hsga_set_allocator(cbs[0], cbs[1], None), "hsga_set_allocator")


def use_default_allocator():
    _check(lib().hsga_set_allocator(ALLOC_FN(), FREE_FN(), None), "hsga_set_allocator")


# ------------------------------------------------------------ functions ---
def make_config(rows=4, cols=4, n=32, tournament=2, policy="steady", bits=1, W=2,
                interval=1, p_ben=0.0, p_del=0.0, seed=1, kernel=KERNEL_AUTO,
                coarsen=1, mode="sync", fitness="trait", sigma=0.0, words=1) -> hsga_config:
    """fitness "trait": unsigned integer fitness, mutations of one; "float":
    binary32 fitness with sign-restricted Gaussian mutation amounts of
    standard deviation ``sigma`` (> 0).  words: surface width in 64-bit words
    (1, 2 or 4; S = 64 words / bits sites)."""
    pol = POLICIES[policy] if isinstance(policy, str) else int(policy)
    return hsga_config(rows, cols, n, tournament, pol, bits, W, interval, p_ben, p_del,
                       seed, kernel, coarsen, {"sync": 0, "async": 1, "buffered": 2}[mode],
                       {"trait": 0, "float": 1}[fitness], sigma, words, 0)


def hsga_init_grid(cfg: hsga_config, cuda_stream=None) -> ctypes.c_void_p:
    out = ctypes.c_void_p()
    stream = None if cuda_stream is None else ctypes.c_void_p(int(cuda_stream))
    _check(lib().hsga_init_grid(ctypes.byref(cfg), stream, ctypes.byref(out)), "hsga_init_grid")
    return out


def hsga_set_population(g, trait, surf, generation: int):
    _check(lib().hsga_set_population(g, _ptr(trait), _ptr(surf), int(generation)),
           "hsga_set_population")


def hsga_get_population(g, trait, surf):
    _check(lib().hsga_get_population(g, _ptr(trait), _ptr(surf)), "hsga_get_population")


def hsga_run_generations(g, n: int):
    _check(lib().hsga_run_generations(g, int(n)), "hsga_run_generations")


def hsga_migrate(g):
    _check(lib().hsga_migrate(g), "hsga_migrate")


def hsga_sample_surfaces(g, k: int, out_words, out_island_slot=None):
    _check(lib().hsga_sample_surfaces(g, int(k), _ptr(out_words), _ptr(out_island_slot)),
           "hsga_sample_surfaces")


def hsga_set_fossil_sampling(g, every: int, k: int, capacity: int):
    _check(lib().hsga_set_fossil_sampling(g, int(every), int(k), int(capacity)),
           "hsga_set_fossil_sampling")


def hsga_get_fossils(g, max_records: int):
    """(words (n, 4), island/slot (n, 2)) of the fossil records held."""
    words = np.zeros((max(1, max_records), 4), dtype=np.uint32)
    where = np.zeros((max(1, max_records), 2), dtype=np.uint32)
    cnt = ctypes.c_uint32()
    _check(lib().hsga_get_fossils(g, _ptr(words), _ptr(where), int(max_records),
                                  ctypes.byref(cnt)), "hsga_get_fossils")
    m = min(cnt.value, max_records)
    return words[:m], where[:m]


def hsga_get_counters(g, T_out):
    _check(lib().hsga_get_counters(g, _ptr(T_out)), "hsga_get_counters")


def hsga_set_async_log(g, generations: int):
    _check(lib().hsga_set_async_log(g, int(generations)), "hsga_set_async_log")


def hsga_get_async_log(g, islands: int, generations: int) -> np.ndarray:
    out = np.zeros((islands, generations, 4), dtype=np.uint32)
    _check(lib().hsga_get_async_log(g, _ptr(out)), "hsga_get_async_log")
    return out


def hsga_get_migration_buffers(g, islands: int):
    """Buffered grids: (chan, inbuf) with chan[island, d] = (posts sent toward
    d, last post taken from d, genomes waiting) and inbuf[island, d, j] =
    (trait, surface lo, surface hi, T) of waiting genome j."""
    chan = np.zeros((islands, 4, 3), dtype=np.uint32)
    inbuf = np.zeros((islands, 4, 4, 4), dtype=np.uint32)
    _check(lib().hsga_get_migration_buffers(g, _ptr(chan), _ptr(inbuf)),
           "hsga_get_migration_buffers")
    return chan, inbuf


def hsga_reconstruct(surf, policy, bits: int, W: int, generations: int, coarsen: int = 1,
                     stream=None, words: int = 1):
    """GPU trie reconstruction of sampled surfaces (k x words uint64,
    agent-major) -> (parent, time, leaf_of_sample) numpy arrays; node 0 is
    the root."""
    pol = POLICIES[policy] if isinstance(policy, str) else int(policy)
    surf = np.ascontiguousarray(surf, dtype=np.uint64).reshape(-1)
    k = len(surf) // max(1, words)
    cap = 2 * k + 1
    parent = np.zeros(cap, dtype=np.int64)
    time = np.zeros(cap, dtype=np.int64)
    leaf = np.zeros(k, dtype=np.uint32)
    nodes = ctypes.c_uint32(0)
    s = None if stream is None else ctypes.c_void_p(int(stream))
    _check(lib().hsga_reconstruct(_ptr(surf), k, words, pol, bits, W, int(generations),
                                  int(coarsen),
                                  _ptr(parent), _ptr(time), _ptr(leaf), cap,
                                  ctypes.byref(nodes), s), "hsga_reconstruct")
    n = nodes.value
    return parent[:n], time[:n], leaf


def hsga_wait_probe(record_dev, seq: int, limit_ns: int, stream=None):
    """Runs the resident kernel's bounded waits (one thread's, then a
    warp's) on a device record of four 64-bit words; returns (status,
    waited_ns) without raising on a timeout."""
    waited = ctypes.c_uint64(0)
    s = None if stream is None else ctypes.c_void_p(int(stream))
    st = lib().hsga_wait_probe(_ptr(record_dev), seq, limit_ns, ctypes.byref(waited), s)
    if st not in (0, -5):
        _check(st, "hsga_wait_probe")
    return st, waited.value


def hsga_philox_device(seed: int, c0: int, count: int, c1: int, c2: int, c3: int, out_dev,
                       stream=None):
    """Philox4x32-10 blocks for counters (c0 + i, c1, c2, c3) into a device
    buffer of count x 4 uint32."""
    s = None if stream is None else ctypes.c_void_p(int(stream))
    _check(lib().hsga_philox_device(seed, c0, count, c1, c2, c3, _ptr(out_dev), s),
           "hsga_philox_device")


def hsga_set_octet_slice(g, generations: int):
    """Free-running grids: generations per visit of each island octet."""
    _check(lib().hsga_set_octet_slice(g, int(generations)), "hsga_set_octet_slice")


def hsga_philox_throughput(seed: int, threads: int, blocks_per_thread: int, c2: int, c3: int,
                           out_dev, stream=None):
    """Per thread t, the xor of every word of the blocks for counters
    (i, t, c2, c3), i < blocks_per_thread, into a device uint32 buffer."""
    s = None if stream is None else ctypes.c_void_p(int(stream))
    _check(lib().hsga_philox_throughput(seed, threads, blocks_per_thread, c2, c3,
                                        _ptr(out_dev), s), "hsga_philox_throughput")


def hsga_synchronize(g):
    _check(lib().hsga_synchronize(g), "hsga_synchronize")


def hsga_get_stats(g) -> dict:
    st = hsga_stats()
    _check(lib().hsga_get_stats(g, ctypes.byref(st)), "hsga_get_stats")
    return {f: getattr(st, f) for f, _ in hsga_stats._fields_}


def hsga_save(g) -> bytes:
    n = ctypes.c_size_t(0)
    _check(lib().hsga_save(g, None, ctypes.byref(n)), "hsga_save")
    buf = ctypes.create_string_buffer(n.value)
    _check(lib().hsga_save(g, buf, ctypes.byref(n)), "hsga_save")
    return buf.raw[:n.value]


def hsga_load(g, blob: bytes):
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check(lib().hsga_load(g, buf, len(blob)), "hsga_load")


def hsga_destroy(g):
    if g:
        lib().hsga_destroy(g)


def hsga_site(policy: int, S: int, W: int, T: int) -> int:
    return int(lib().hsga_site(policy, S, W, T))


def hsga_lookup(policy: int, S: int, W: int, T: int) -> np.ndarray:
    out = np.zeros(S, dtype=np.int64)
    _check(lib().hsga_lookup(policy, S, W, T, _ptr(out)), "hsga_lookup")
    return out


def hsga_sites_device(policy: int, S: int, W: int, T0: int, count: int, out_dev, stream=None):
    s = None if stream is None else ctypes.c_void_p(int(stream))
    _check(lib().hsga_sites_device(policy, S, W, T0, count, _ptr(out_dev), s),
           "hsga_sites_device")


def hsga_run_generations_noalloc(cfg: hsga_config, generation: int, n: int, trait_dev,
                                 surf_dev, stream=None):
    """Advances device planes in place without any device allocation (the
    library's built-in scratch is used; see include/hsga.h)."""
    s = None if stream is None else ctypes.c_void_p(int(stream))
    _check(lib().hsga_run_generations_noalloc(ctypes.byref(cfg), int(generation), int(n),
                                              _ptr(trait_dev), _ptr(surf_dev), s),
           "hsga_run_generations_noalloc")


def hsga_batch_create(cuda_stream=None):
    out = ctypes.c_void_p()
    s = None if cuda_stream is None else ctypes.c_void_p(int(cuda_stream))
    _check(lib().hsga_batch_create(s, ctypes.byref(out)), "hsga_batch_create")
    return out


def hsga_batch_add(b, cfg: hsga_config, generations: int) -> int:
    rid = ctypes.c_uint32()
    _check(lib().hsga_batch_add(b, ctypes.byref(cfg), int(generations), ctypes.byref(rid)),
           "hsga_batch_add")
    return rid.value


def hsga_batch_run(b, ticks: int):
    _check(lib().hsga_batch_run(b, int(ticks)), "hsga_batch_run")


def hsga_batch_info(b, run: int) -> dict:
    info = hsga_batch_run_info()
    _check(lib().hsga_batch_info(b, run, ctypes.byref(info)), "hsga_batch_info")
    return {f: getattr(info, f) for f, _ in hsga_batch_run_info._fields_}


def hsga_batch_get_population(b, run: int, trait, surf):
    _check(lib().hsga_batch_get_population(b, run, _ptr(trait), _ptr(surf)),
           "hsga_batch_get_population")


def hsga_batch_sample(b, run: int, k: int, out_words, out_island_slot=None):
    _check(lib().hsga_batch_sample(b, run, int(k), _ptr(out_words), _ptr(out_island_slot)),
           "hsga_batch_sample")


def hsga_batch_remove(b, run: int):
    _check(lib().hsga_batch_remove(b, run), "hsga_batch_remove")


def hsga_batch_get_stats(b) -> dict:
    st = hsga_batch_stats()
    _check(lib().hsga_batch_get_stats(b, ctypes.byref(st)), "hsga_batch_get_stats")
    return {f: getattr(st, f) for f, _ in hsga_batch_stats._fields_}


def hsga_run_footprint(cfg: hsga_config) -> int:
    n = ctypes.c_uint64()
    _check(lib().hsga_run_footprint(ctypes.byref(cfg), ctypes.byref(n)), "hsga_run_footprint")
    return n.value


def hsga_batch_destroy(b):
    if b:
        lib().hsga_batch_destroy(b)


class Batch:
    """Owning wrapper around an hsga_batch (many runs advanced together)."""

    def __init__(self, stream=None):
        self.handle = hsga_batch_create(stream)
        self.cfgs = []

    def add(self, generations, **kw) -> int:
        cfg = make_config(**kw)
        rid = hsga_batch_add(self.handle, cfg, generations)
        self.cfgs.append(cfg)
        return rid

    def run(self, ticks):
        hsga_batch_run(self.handle, ticks)

    def info(self, run):
        return hsga_batch_info(self.handle, run)

    def population(self, run):
        c = self.cfgs[run]
        agents = c.rows * c.cols * c.agents_per_island
        t = np.zeros(agents, dtype=np.uint32)
        s = np.zeros(agents, dtype=np.uint64)
        hsga_batch_get_population(self.handle, run, t, s)
        return t, s

    def sample(self, run, k):
        w = np.zeros((k, 4), dtype=np.uint32)
        where = np.zeros((k, 2), dtype=np.uint32)
        hsga_batch_sample(self.handle, run, k, w, where)
        return w, where

    def remove(self, run):
        hsga_batch_remove(self.handle, run)

    def stats(self):
        return hsga_batch_get_stats(self.handle)

    def sync(self):
        _check(lib().hsga_batch_synchronize(self.handle), "hsga_batch_synchronize")

    def close(self):
        if self.handle:
            hsga_batch_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------- convenience ---
@dataclass
class Grid:
    """Owning wrapper: ``Grid(**config)``; methods call the C-ABI above."""

    def __init__(self, stream=None, **kw):
        self.cfg = make_config(**kw)
        self.handle = hsga_init_grid(self.cfg, stream)

    @property
    def agents(self) -> int:
        return self.cfg.rows * self.cfg.cols * self.cfg.agents_per_island

    @property
    def islands(self) -> int:
        return self.cfg.rows * self.cfg.cols

    def set_population(self, trait, surf, generation):
        hsga_set_population(self.handle, trait, surf, generation)

    @property
    def words(self) -> int:
        return max(1, self.cfg.surface_words)

    def population(self):
        t = np.zeros(self.agents, dtype=np.uint32)
        s = np.zeros(self.agents * self.words, dtype=np.uint64)
        hsga_get_population(self.handle, t, s)
        return t, s

    def counters(self):
        T = np.zeros(self.agents, dtype=np.uint32)
        hsga_get_counters(self.handle, T)
        return T

    def run(self, n):
        hsga_run_generations(self.handle, n)

    def buffers(self):
        return hsga_get_migration_buffers(self.handle, self.islands)

    def migrate(self):
        hsga_migrate(self.handle)

    def sample(self, k):
        w = np.zeros((k, 2 + 2 * self.words), dtype=np.uint32)
        where = np.zeros((k, 2), dtype=np.uint32)
        hsga_sample_surfaces(self.handle, k, w, where)
        return w, where

    def sync(self):
        hsga_synchronize(self.handle)

    def stats(self):
        return hsga_get_stats(self.handle)

    def close(self):
        if self.handle:
            hsga_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
