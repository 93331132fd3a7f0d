"""Continuous-batching server for evolution experiments.

Requests (one island-model GA run each: grid, agents per island, policy,
adaptation, generation budget) arrive over time.  The server keeps admitted
runs resident on the device inside one batch (``hsga_batch_*``, which
advances every active run by one generation per tick in one launch),
admits waiting requests whenever their device-memory footprint fits under a
cap, advances the batch in slices of generations, and when a run finishes
returns its sampled surfaces (step a7) and frees its memory.  Requests that
arrive while others are on the GPU join between slices, so their work
overlaps.

Admission is size-aware.  A run of at least ``large_agents`` agents keeps
the whole GPU busy on its own; at most ``max_large`` of those run at a time,
first come first served among them, while smaller requests are admitted in
arrival order as soon as they fit, never queueing behind a large one.  A
large run advances on a grid of its own (the single-run kernels, which
stream a large grid faster than the batch's tick kernel) on a second stream
beside the batch, in slices of the same length as the batch's, so it runs
at nearly its speed alone; the small runs, which alone would leave the GPU
idle between their short generations, overlap with it in the batch.
``serve_alone`` is the reference policy: the same stream served one request
at a time, each on its own grid.

Every run's result is the same whether it ran alone or in the mix (the batch
engine is bit-identical to a lone grid); tests check that on sampled output.
"""
from __future__ import annotations

import math
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import binding as hb


@dataclass
class Request:
    rid: int
    arrival: float            # seconds after the stream starts
    config: dict              # keyword arguments of binding.make_config
    generations: int
    sample_k: int

    @property
    def agents(self) -> int:
        return self.config["rows"] * self.config["cols"] * self.config["n"]


@dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    finished: float
    replications: int
    words: np.ndarray = field(repr=False)
    where: np.ndarray = field(repr=False)

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def splitmix64(x: int) -> int:
    x = (x + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
    x = ((x ^ (x >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
    x = ((x ^ (x >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
    return x ^ (x >> 31)


def poisson_requests(count: int, rate: float, seed: int = 5, gen_scale: int = 1,
                     agents_range=(1024, 4_194_304), gens_range=(1000, 100_000),
                     sample_k: int = 10_000, n: int = 32):
    """The served-experiments stream: Poisson arrivals at `rate` per second;
    agents log-uniform over agents_range mapped to n agents per island on a
    near-square torus (rows = 2^floor(log2 sqrt(islands)), cols =
    ceil(islands / rows)); generations log-uniform over gens_range divided by
    gen_scale; random policy (steady / tilted / stretched) and adaptive flag."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += float(rng.exponential(1.0 / rate))
        agents = math.exp(rng.uniform(math.log(agents_range[0]), math.log(agents_range[1])))
        islands = max(1, math.ceil(agents / n))
        rows = 2 ** int(math.floor(math.log2(math.sqrt(islands))))
        cols = math.ceil(islands / rows)
        gens = int(math.exp(rng.uniform(math.log(gens_range[0]), math.log(gens_range[1]))))
        gens = max(1, gens // gen_scale)
        policy = str(rng.choice(["steady", "tilted", "stretched"]))
        p_ben = 1e-3 if rng.random() < 0.5 else 0.0
        cfg = dict(rows=rows, cols=cols, n=n, tournament=2, policy=policy, bits=1, W=2,
                   interval=1, p_ben=p_ben, p_del=0.0, seed=splitmix64((seed << 32) | i))
        out.append(Request(i, t, cfg, gens, min(sample_k, rows * cols)))
    return out


def _wait_until(t0: float, rel: float):
    while time.perf_counter() - t0 < rel:
        time.sleep(min(0.0005, max(0.0, rel - (time.perf_counter() - t0))))


def serve(requests, memory_cap: int, slice_ticks: int = 256, stream=None,
          large_agents: int | None = 1 << 20, max_large: int = 1, large_apart: bool = True,
          large_stream=None):
    """Continuous batching with size-aware admission (module docstring);
    large_agents=None admits every request first come, first served.
    large_apart=False keeps large runs inside the batch too.  large_stream:
    the stream of the large runs' grids (default: `stream`, which serialises
    them with the batch).  Returns (results, stats)."""
    pending = deque(sorted(requests, key=lambda r: r.arrival))
    waiting: list = []                 # arrived, not admitted, in arrival order
    running = {}                       # batch run id -> (request, admitted time, footprint)
    apart = {}                         # request id -> [request, admitted, footprint, grid, done]
    results = []
    in_use = 0
    peak_runs = 0
    peak_large = 0
    blocked = 0                        # admissions deferred by the memory cap
    grid_launches = 0
    if large_stream is None:
        large_stream = stream

    def is_large(req):
        return large_agents is not None and req.agents >= large_agents

    def finish(req, admitted, words, where):
        results.append(Result(req.rid, req.arrival, admitted, time.perf_counter() - t0,
                              req.agents * req.generations, words, where))

    with hb.Batch(stream=stream) as batch:
        t0 = time.perf_counter()
        while pending or waiting or running or apart:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            large_now = len(apart) + sum(1 for req, _, _ in running.values() if is_large(req))
            i = 0
            while i < len(waiting):
                req = waiting[i]
                if is_large(req) and large_now >= max_large:
                    i += 1                 # waits for the large slot; later requests may pass
                    continue
                fp = hb.hsga_run_footprint(hb.make_config(**req.config))
                if fp > memory_cap:
                    raise ValueError(f"request {req.rid} needs {fp} bytes, over the cap")
                if in_use + fp > memory_cap:
                    blocked += 1
                    break                  # memory goes to requests in arrival order
                waiting.pop(i)
                admitted = time.perf_counter() - t0
                if large_apart and is_large(req):
                    apart[req.rid] = [req, admitted, fp, hb.Grid(stream=large_stream,
                                                                 **req.config), 0]
                else:
                    rid = batch.add(req.generations, **req.config)
                    running[rid] = (req, admitted, fp)
                in_use += fp
                large_now += is_large(req)
            peak_runs = max(peak_runs, len(running) + len(apart))
            peak_large = max(peak_large, large_now)
            if not running and not apart:
                if pending:
                    _wait_until(t0, pending[0].arrival)
                continue
            # one slice: the large runs' grids and the batch advance side by side
            for a in apart.values():
                n = min(slice_ticks, a[0].generations - a[4])
                a[3].run(n)
                a[4] += n
            if running:
                remaining = min(req.generations - batch.info(rid)["generation"]
                                for rid, (req, _, _) in running.items())
                batch.run(max(1, min(slice_ticks, remaining)))
            for a in apart.values():
                a[3].sync()
            batch.sync()          # one slice in flight: arrivals join at the next slice
            for key in [k for k, a in apart.items() if a[4] >= a[0].generations]:
                req, admitted, fp, g, _ = apart.pop(key)
                words, where = g.sample(req.sample_k)              # synchronous
                grid_launches += g.stats()["kernel_launches"]
                g.close()
                finish(req, admitted, words, where)
                in_use -= fp
            for rid in [r for r in running if batch.info(r)["done"]]:
                req, admitted, fp = running.pop(rid)
                words, where = batch.sample(rid, req.sample_k)       # synchronous
                finish(req, admitted, words, where)
                batch.remove(rid)
                in_use -= fp
        elapsed = time.perf_counter() - t0
        st = batch.stats()
    return results, {"elapsed_s": elapsed, "peak_concurrent_runs": peak_runs,
                     "peak_concurrent_large_runs": peak_large,
                     "admissions_deferred": blocked,
                     "kernel_launches": st["kernel_launches"] + grid_launches,
                     "ticks": st["tick"]}


def serve_alone(requests, stream=None):
    """Reference policy: first come, first served, one run at a time."""
    results = []
    t0 = time.perf_counter()
    for req in sorted(requests, key=lambda r: r.arrival):
        _wait_until(t0, req.arrival)
        start = time.perf_counter() - t0
        with hb.Grid(stream=stream, **req.config) as g:
            g.run(req.generations)
            words, where = g.sample(req.sample_k)
        results.append(Result(req.rid, req.arrival, start, time.perf_counter() - t0,
                              req.agents * req.generations, words, where))
    return results, {"elapsed_s": time.perf_counter() - t0}


def summarize(results, stats) -> dict:
    lat = np.array([r.latency for r in results])
    reps = sum(r.replications for r in results)
    el = stats["elapsed_s"]
    out = {"completed": len(results), "runs_per_hour": len(results) * 3600.0 / el,
           "agent_replications_per_s": reps / el,
           "latency_p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
           "latency_p99_s": float(np.percentile(lat, 99)) if len(lat) else None}
    out.update(stats)
    return out
