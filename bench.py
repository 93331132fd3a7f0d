"""Benchmark: agent replications per second of the island-model GA hot path
(arXiv 2404.10861) on the wafer-shaped workload: 512 x 1024 toroidal islands
x 32 agents = 16,777,216 agents, 3 x uint32 genomes (trait + 64-bit tilted
surface of 1-bit differentiae), tournament 2, beneficial mutation 1e-3,
synchronous migration every generation (the bit-exact mode).

One step = GENS_PER_STEP (1,000) generations of steps a1-a6 over the whole
grid plus step a7 (10,000 sampled genomes).  Inputs live in HBM: the
population is 201 MB per plane, larger than the 129 MB L2, so no flush is
needed between launches.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  For N > 1 (torchrun) every rank runs an
independent replica (its own seed): the island grid is replicated, not
sharded, on this machine; timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

ROWS, COLS, N_AGENTS = 512, 1024, 32
GENS_PER_STEP = 1000
SAMPLE_K = 10000
WORKLOAD = dict(rows=ROWS, cols=COLS, n=N_AGENTS, tournament=2, policy="tilted", bits=1, W=2,
                interval=1, p_ben=1e-3, p_del=0.0)
AGENTS = ROWS * COLS * N_AGENTS
# Algorithmic HBM bytes of one streamed generation launch: every agent's
# 12-byte genome read once and its child's written once, plus one 12-byte
# emigrant gather per island.
BYTES_PER_LAUNCH = AGENTS * 24 + ROWS * COLS * 12


def config_json(world: int = 1):
    """The workload, the same on both arms (each arm's step is described
    beside it, under "step")."""
    return {"workload": "wafer-shaped island GA, sync migration (512x1024 islands x 32 agents)",
            "islands": ROWS * COLS, "agents": AGENTS, "agents_per_island": N_AGENTS,
            "genome": "3 x uint32 (trait + 64-bit tilted surface, 1-bit differentiae)",
            "tournament": 2, "p_beneficial": 1e-3, "migration": "synchronous, every generation",
            "l2": "inputs larger than L2 (201 MB per population plane)",
            "parallelism": f"replicas{world}"}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


KERNEL_SOURCES = ["paper_2404_10861_gb300/csrc/hsga_device.cuh",
                  "paper_2404_10861_gb300/csrc/hsga_island.cuh",
                  "paper_2404_10861_gb300/csrc/hsga_internal.h",
                  "paper_2404_10861_gb300/csrc/hsga_kernels.cu",
                  "paper_2404_10861_gb300/csrc/hsga_stage.cuh",
                  "paper_2404_10861_gb300/csrc/hsga_staged.cu"]
PROFILE = os.path.join(ROOT, "profiles", "step_streamed_wafer.md")
FREE_RUNNING_SOURCES = ["paper_2404_10861_gb300/csrc/hsga_device.cuh",
                        "paper_2404_10861_gb300/csrc/hsga_island.cuh",
                        "paper_2404_10861_gb300/csrc/hsga_async.cu"]
FREE_RUNNING_PROFILE = os.path.join(ROOT, "profiles", "step_free_running_wafer.md")


def kernel_source_hash(sources=KERNEL_SOURCES) -> str:
    import hashlib
    h = hashlib.sha256()
    for f in sources:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def profiled_traffic(key="dram_bytes_per_launch", profile=PROFILE, sources=KERNEL_SOURCES):
    """DRAM bytes (the `key` field) from a committed ncu summary, or None when
    the kernel sources changed since that capture."""
    try:
        fields = {}
        for line in open(profile):
            if ":" in line and line.strip().startswith(("source_sha256", key)):
                k, v = line.strip().strip("`").split(":", 1)
                fields[k.strip()] = v.strip().strip("`")
        if fields.get("source_sha256") != kernel_source_hash(sources):
            return None
        return int(fields[key])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.out = None

    def __enter__(self):
        try:
            self.out = open(f"/tmp/hsga_clocks_{os.getpid()}.csv", "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.out:
            self.out.close()

    def summary(self):
        path = f"/tmp/hsga_clocks_{os.getpid()}.csv"
        try:
            rows = [l.strip().split(", ") for l in open(path) if l.strip()]
            os.unlink(path)
        except Exception:
            return None
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except Exception:
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(n_gpus: int):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    return rank, world, local


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_config(seed: int):
    import oracle
    return oracle.Config(rows=ROWS, cols=COLS, n=N_AGENTS, tournament=2, policy=oracle.TILTED,
                         bits=1, W=2, interval=1, p_ben=1e-3, seed=seed)


def _oracle_replica_run(job):
    """One host core's replica: the workload's first `generations`
    generations from founders with its own seed.  Returns wall-clock start
    and end (comparable across processes)."""
    seed, generations = job
    import oracle
    oracle.build()
    cfg = oracle_config(seed)
    t0 = time.time()
    oracle.run(cfg, generations=generations)
    return t0, time.time()


def cpu_baseline_oracle(generations: int = 12):
    """The oracle as it stands (plain single-threaded C) on every host core
    at once: one independent replica of the workload per core (own seed),
    each running its first `generations` generations from founders.  The
    pool is spawned, never forked, because CUDA is initialised already."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    cores = host_cores()
    jobs = [(1 + i, generations) for i in range(cores)]
    with mp.get_context("spawn").Pool(cores) as pool:
        spans = pool.map(_oracle_replica_run, jobs, chunksize=1)
    per_core = [AGENTS * generations / (b - a) for a, b in spans]
    wall = max(b for _, b in spans) - min(a for a, _ in spans)
    total = AGENTS * generations * cores
    return {"value": total / wall, "unit": "agent replications/s", "cores": cores,
            "kind": "oracle", "per_core": statistics.median(per_core),
            "sample": f"one replica per host core ({cores} processes, seeds 1..{cores}), each "
                      f"{generations} generations of the full 16.8M-agent grid from founders "
                      f"({total:.3g} replications in {wall:.1f} s wall; median "
                      f"{statistics.median(per_core):.3g} replications/s per core)"}


def _oracle_replica_server(conn, seed):
    """Reference-arm worker: holds one replica of the workload and advances
    it one generation per request, replying with the seconds it took."""
    import oracle
    oracle.build()
    cfg = oracle_config(seed)
    trait, surf = oracle.founders(cfg)
    G = 0
    while True:
        if conn.recv() is None:
            break
        t0 = time.perf_counter()
        trait, surf, _ = oracle.run(cfg, trait, surf, G0=G, generations=1)
        G += 1
        conn.send(time.perf_counter() - t0)
    conn.close()


def run_reference(args):
    """The oracle as the reference arm: one replica of the workload per host
    core (spawned processes, own seeds); a step advances every replica by one
    generation of the full grid (a bounded sample of the workload)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import multiprocessing as mp
    import oracle
    oracle.build()
    cores = host_cores()
    ctx = mp.get_context("spawn")
    pipes, procs = [], []
    for i in range(cores):
        a, b = ctx.Pipe()
        pr = ctx.Process(target=_oracle_replica_server, args=(b, 1 + i), daemon=True)
        pr.start()
        pipes.append(a)
        procs.append(pr)

    def step():
        for c in pipes:
            c.send(1)
        for c in pipes:
            c.recv()

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    for c in pipes:
        c.send(None)
    for pr in procs:
        pr.join(timeout=30)
    value = AGENTS * cores * args.steps / dt
    sample = (f"{args.steps} timed steps; a step = one generation of the full grid on each of "
              f"{cores} replicas (one per host core, seeds 1..{cores})")
    line = {"impl": "reference", "metric": "agent replications/sec", "value": value,
            "unit": "agent replications/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": config_json(),
            "step": {"generations": 1, "replicas": cores, "sample_genomes": 0,
                     "engine": "CPU oracle (plain C, one single-threaded process per core)"},
            "cpu_baseline": {"value": value, "unit": "agent replications/s", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "agent replications/s",
                    "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def philox_peak(stream) -> dict:
    """Measured ceiling of the integer-issue bound: Philox4x32-10 blocks per
    second drawn by hsga_philox_throughput (the generation kernels' form of
    the generator) over every SM at full occupancy, timed with CUDA events on
    its stream.  Every replication draws one block, so replications/s can
    not exceed this."""
    import torch
    from paper_2404_10861_gb300 import binding as hb
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    threads, m = sms * 2048, 2048
    out = torch.empty(threads, dtype=torch.int32, device="cuda")
    for _ in range(3):
        hb.hsga_philox_throughput(7, threads, m, 0, 1, out, stream.cuda_stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 10
    e0.record(stream)
    for _ in range(reps):
        hb.hsga_philox_throughput(7, threads, m, 0, 1, out, stream.cuda_stream)
    e1.record(stream)
    e1.synchronize()
    sec = e0.elapsed_time(e1) / 1e3
    return {"blocks_per_s": threads * m * reps / sec, "kernel": "philox_throughput_kernel",
            "launch": f"{threads} threads x {m} blocks, {reps} launches",
            "ms_per_launch": sec * 1e3 / reps}


def alu_roofline(reps_per_s: float, peak: dict) -> dict:
    return {"bound": "alu", "achieved": reps_per_s, "peak": peak["blocks_per_s"],
            "unit": "replications/s (one Philox4x32-10 block each)",
            "frac": reps_per_s / peak["blocks_per_s"],
            "peak_kind": "measured in this run: Philox blocks/s of hsga_philox_throughput",
            "peak_ms_per_launch": peak["ms_per_launch"]}


def run_ours(args):
    import torch
    from paper_2404_10861_gb300 import _build, binding as hb
    from paper_2404_10861_gb300 import inputs

    _build.build()
    rank, world, local = dist_setup(args.gpus)
    hb.use_torch_allocator()
    stream = torch.cuda.Stream()
    seed = 1 + rank
    grid = hb.Grid(stream=stream.cuda_stream, kernel=hb.KERNEL_STREAMED, seed=seed, **WORKLOAD)
    words = torch.zeros((SAMPLE_K, 4), dtype=torch.int32, device="cuda")
    where = torch.zeros((SAMPLE_K, 2), dtype=torch.int32, device="cuda")

    def step():
        hb.hsga_run_generations(grid.handle, GENS_PER_STEP)
        hb.hsga_sample_surfaces(grid.handle, SAMPLE_K, words, where)

    for _ in range(args.warmup):
        step()
    hb.hsga_synchronize(grid.handle)
    launches0 = grid.stats()["kernel_launches"]

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for i in range(args.steps):
            ev[i][0].record(stream)
            hb.hsga_run_generations(grid.handle, GENS_PER_STEP)
            ev[i][1].record(stream)
            hb.hsga_sample_surfaces(grid.handle, SAMPLE_K, words, where)
            ev[i][2].record(stream)
        t_end.record(stream)
        torch.cuda.synchronize()
    hb.hsga_synchronize(grid.handle)
    barrier(world)
    elapsed_ms = t_start.elapsed_time(t_end)
    gen_ms = sum(a.elapsed_time(b) for a, b, _ in ev)
    sample_ms = sum(b.elapsed_time(c) for _, b, c in ev)
    launches = grid.stats()["kernel_launches"] - launches0
    elapsed_ms = max_over_ranks(elapsed_ms, world)
    reps = AGENTS * GENS_PER_STEP * args.steps * world
    value = reps / (elapsed_ms / 1e3)

    # roofline of the dominant kernel (the staged generation kernel)
    per_launch_s = gen_ms / 1e3 / (GENS_PER_STEP * args.steps)
    alu_peak = philox_peak(stream)
    achieved = BYTES_PER_LAUNCH / per_launch_s / 1e9
    peak, peak_kind = measured_peaks()
    traffic = profiled_traffic()

    # end to end through the C-ABI with host buffers: every step copies a
    # population in from pinned host memory, runs the generations and reads
    # the sample back to the host.  Two grids take turns, so that the next
    # step's host->device copy (on its own grid's stream) runs while the
    # current step's generations do; the generations themselves run one step
    # at a time.
    e2e = None
    if args.e2e_steps > 0:
        ht, hs = inputs.founders(AGENTS)
        pin_t = torch.from_numpy(ht.view(np.int32)).pin_memory()
        pin_s = torch.from_numpy(hs.view(np.int64)).pin_memory()
        hw = np.zeros((SAMPLE_K, 4), dtype=np.uint32)
        hwhere = np.zeros((SAMPLE_K, 2), dtype=np.uint32)
        pin_w = torch.from_numpy(hw.view(np.int32)).pin_memory()
        pin_where = torch.from_numpy(hwhere.view(np.int32)).pin_memory()
        stream2 = torch.cuda.Stream()
        grid2 = hb.Grid(stream=stream2.cuda_stream, kernel=hb.KERNEL_STREAMED, seed=seed,
                        **WORKLOAD)
        grids = (grid, grid2)
        e2e_steps = args.e2e_steps
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hb.hsga_set_population(grids[0].handle, pin_t, pin_s, 0)
        for i in range(e2e_steps):
            cur, nxt = grids[i % 2], grids[(i + 1) % 2]
            hb.hsga_run_generations(cur.handle, GENS_PER_STEP)
            if i + 1 < e2e_steps:
                hb.hsga_set_population(nxt.handle, pin_t, pin_s, 0)
            hb.hsga_sample_surfaces(cur.handle, SAMPLE_K, pin_w, pin_where)
        for g in grids:
            hb.hsga_synchronize(g.handle)
        dt = time.perf_counter() - t0
        dt = max_over_ranks(dt, world)
        grid2.close()
        e2e = {"value": AGENTS * GENS_PER_STEP * e2e_steps * world / dt,
               "unit": "agent replications/s", "h2d_bytes_per_step": AGENTS * 12,
               "d2h_bytes_per_step": SAMPLE_K * 24}
    grid.close()

    if rank == 0:
        cpu = cpu_baseline_oracle() if (world == 1 and not args.no_cpu_baseline) else None
        line = {"metric": "agent replications/sec", "value": value,
                "unit": "agent replications/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "u32", "data": "synthetic",
                "config": config_json(world),
                "step": {"generations": GENS_PER_STEP, "sample_genomes": SAMPLE_K,
                         "kernel": "step_staged_kernel (one generation per launch)"},
                "e2e": e2e,
                "gpu_launches": int(launches),
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak,
                             "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                             "kernel": "step_staged_kernel", "peak_kind": peak_kind,
                             "algorithmic_bytes_per_launch": BYTES_PER_LAUNCH,
                             "avg_launch_us": per_launch_s * 1e6},
                "alu": alu_roofline(value / world, alu_peak),
                "sample_ms_per_step": sample_ms / args.steps,
                "clocks": clk.summary(),
                "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


SECONDARY = {
    # the 4x4-island tiny workload (whole 2,000-generation run per step) and the
    # 64x64-island mid-grid workload (1,000 generations per step); both run on
    # the default kernel choice (resident: genomes stay in registers)
    "tiny": (dict(rows=4, cols=4, n=32, tournament=2, policy="steady", bits=1, W=2,
                  interval=1, p_ben=0.0, p_del=0.0), 2000),
    "mid": (dict(rows=64, cols=64, n=32, tournament=2, policy="tilted", bits=2, W=2,
                 interval=1, p_ben=1e-3, p_del=0.0), 1000),
}


def run_secondary(args):
    """Informational lines for the smaller workloads (not the headline)."""
    import torch
    from paper_2404_10861_gb300 import _build, binding as hb
    _build.build()
    torch.cuda.set_device(0)
    kw, gens = SECONDARY[args.workload]
    agents = kw["rows"] * kw["cols"] * kw["n"]
    out = []
    for kernel in (hb.KERNEL_RESIDENT, hb.KERNEL_RESIDENT_GRID, hb.KERNEL_STREAMED):
        stream = torch.cuda.Stream()
        with hb.Grid(stream=stream.cuda_stream, kernel=kernel, seed=1, **kw) as g:
            for _ in range(args.warmup):
                g.run(gens)
            g.sync()
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            for _ in range(args.steps):
                g.run(gens)
            s1.record(stream)
            g.sync()
            ms = s0.elapsed_time(s1)
            st = g.stats()
        out.append({"kernel": {hb.KERNEL_RESIDENT: "resident", hb.KERNEL_RESIDENT_GRID:
                               "resident_grid", hb.KERNEL_STREAMED: "streamed"}[kernel],
                    "value": agents * gens * args.steps / (ms / 1e3),
                    "ms_per_step": ms / args.steps, "us_per_generation": ms * 1e3 / (gens * args.steps),
                    "islands_per_warp": st["islands_per_warp"], "blocks": st["blocks"]})
    # the resident path's roofline is integer issue: every replication draws
    # one Philox block, against the measured block rate of the generator
    best = max(out, key=lambda r: r["value"])
    alu = dict(alu_roofline(best["value"], philox_peak(torch.cuda.Stream())),
               kernel=best["kernel"])
    print(json.dumps({"metric": "agent replications/sec", "unit": "agent replications/s",
                      "workload": args.workload, "config": dict(kw, generations_per_step=gens),
                      "steps": args.steps, "warmup": args.warmup, "dtype": "u32",
                      "data": "synthetic", "kernels": out, "alu": alu}), flush=True)


def splitmix64(x: int) -> int:
    """Seed derivation hash(master, index) (SplitMix64 finaliser, Steele et al. 2014)."""
    x = (x + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
    x = ((x ^ (x >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
    x = ((x ^ (x >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
    return x ^ (x >> 31)


def batched_runs(gen_scale: int, count: int = 256, master: int = 4):
    """The batched-replicates workload: grid side uniform over
    {8,16,32,64,128,256}, square or 2:1 (coin flip), 16-64 agents per island,
    steady / tilted / stretched, adaptation on (p_ben 1e-3) or off, budgets
    uniform over [10,000, 200,000] generations divided by gen_scale."""
    rng = np.random.default_rng(master)
    runs = []
    for i in range(count):
        side = int(rng.choice([8, 16, 32, 64, 128, 256]))
        rows, cols = (side, side) if rng.random() < 0.5 else (side, 2 * side)
        n = int(rng.integers(16, 65))
        policy = str(rng.choice(["steady", "tilted", "stretched"]))
        p_ben = 1e-3 if rng.random() < 0.5 else 0.0
        gens = int(rng.integers(10_000, 200_001)) // gen_scale
        runs.append((gens, dict(rows=rows, cols=cols, n=n, tournament=2, policy=policy,
                                bits=1, W=2, interval=1, p_ben=p_ben, p_del=0.0,
                                seed=splitmix64((master << 32) | i))))
    return runs


def run_batched(args):
    """Batched replicates in one batch against the same runs launched one
    after another through the plain grid API."""
    import torch
    from paper_2404_10861_gb300 import _build, binding as hb
    _build.build()
    torch.cuda.set_device(0)
    hb.use_torch_allocator()
    if args.gen_scale is None:
        args.gen_scale = 1
    runs = batched_runs(args.gen_scale)
    reps = sum(g * kw["rows"] * kw["cols"] * kw["n"] for g, kw in runs)
    stream = torch.cuda.Stream()
    # batched: all runs admitted at tick 0, run until every budget is spent
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with hb.Batch(stream=stream.cuda_stream) as b:
        for g, kw in runs:
            b.add(g, **kw)
        b.run(10**9)
        torch.cuda.synchronize()
        t_batch = time.perf_counter() - t0
        st = b.stats()
    # plain: one grid per run, one after another
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for g, kw in runs:
        with hb.Grid(stream=stream.cuda_stream, **kw) as grid:
            grid.run(g)
            grid.sync()
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0
    print(json.dumps({
        "metric": "runs/hour and agent replications/sec, batched vs plain",
        "workload": "batched replicates: 256 runs, sides {8..256} square or 2:1, 16-64 agents "
                    "per island, steady/tilted/stretched, adaptive coin flip, master seed 4",
        "generation_budgets": f"uniform [10000, 200000] / {args.gen_scale}",
        "replications": reps,
        "batched": {"seconds": t_batch, "runs_per_hour": len(runs) * 3600 / t_batch,
                    "agent_replications_per_s": reps / t_batch, "phases": st["phases"],
                    "kernel_launches": st["kernel_launches"],
                    "threads_per_block": st["threads_per_block"]},
        "plain_sequential": {"seconds": t_plain, "runs_per_hour": len(runs) * 3600 / t_plain,
                             "agent_replications_per_s": reps / t_plain},
        "speedup": t_plain / t_batch, "dtype": "u32", "data": "synthetic"}), flush=True)


def run_served(args):
    """Served experiments: a Poisson stream of runs served by continuous
    batching against the same stream served one run at a time."""
    import torch
    from paper_2404_10861_gb300 import _build, binding as hb, serve
    _build.build()
    torch.cuda.set_device(0)
    hb.use_torch_allocator()
    if args.gen_scale is None:
        args.gen_scale = 1
    rate = 20.0 * args.gen_scale      # keeps the offered load of the full-size stream
    reqs = serve.poisson_requests(args.requests, rate, seed=5, gen_scale=args.gen_scale)
    offered = sum(r.agents * r.generations for r in reqs) / reqs[-1].arrival
    stream = torch.cuda.Stream()
    large_stream = torch.cuda.Stream()     # large runs' own grids, beside the batch
    # the device's own memory is the cap unless one is given
    cap = (args.memory_cap_mb * 2**20 if args.memory_cap_mb
           else int(0.9 * torch.cuda.mem_get_info()[0]))
    res_b, st_b = serve.serve(reqs, memory_cap=cap, stream=stream.cuda_stream,
                              large_stream=large_stream.cuda_stream)
    res_a, st_a = serve.serve_alone(reqs, stream=stream.cuda_stream)
    same = sum(int(np.array_equal(a.words, b.words) and np.array_equal(a.where, b.where))
               for a, b in zip(sorted(res_a, key=lambda r: r.rid),
                               sorted(res_b, key=lambda r: r.rid)))
    print(json.dumps({
        "metric": "runs/hour and p50/p99 completion latency, continuous batching vs alone",
        "workload": f"{args.requests} requests, Poisson {rate:g}/s, agents log-uniform "
                    f"[1024, 4194304] (32 per island, near-square torus), generations "
                    f"log-uniform [1000, 100000] / {args.gen_scale}, random policy and "
                    f"adaptive flag, seed 5, 10,000-genome samples",
        "admission": "size-aware: runs of >= 2^20 agents one at a time (first come, first "
                     "served among them) on their own grid beside the batch, smaller runs "
                     "first come, first served into the batch as they fit",
        "offered_agent_replications_per_s": offered,
        "memory_cap_bytes": cap,
        "served": serve.summarize(res_b, st_b), "alone": serve.summarize(res_a, st_a),
        "results_identical_alone_and_in_the_mix": f"{same}/{len(reqs)}",
        "dtype": "u32", "data": "synthetic"}), flush=True)


def run_async_wafer(args, mode="async"):
    """Free-running migration on the wafer-shaped grid, K generations per
    persistent launch (every warp stays resident and streams its islands
    through HBM each generation; islands never wait for one another).  mode
    "async": latest-emigrant records; "buffered": the per-neighbour send and
    receive buffers."""
    import torch
    from paper_2404_10861_gb300 import _build, binding as hb
    _build.build()
    torch.cuda.set_device(0)
    hb.use_torch_allocator()
    stream = torch.cuda.Stream()
    out = []
    for octet_slice in args.octet_slices:
        for K in args.slices:
            with hb.Grid(stream=stream.cuda_stream, mode=mode, seed=1, **WORKLOAD) as g:
                hb.hsga_set_octet_slice(g.handle, octet_slice)
                for _ in range(args.warmup):
                    g.run(K)
                g.sync()
                steps = max(1, args.async_gens // K)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(steps):
                    g.run(K)
                e1.record(stream)
                g.sync()
                ms = e0.elapsed_time(e1)
            gens = steps * K
            out.append({"generations_per_launch": K, "generations_per_octet_visit": octet_slice,
                        "generations": gens, "value": AGENTS * gens / (ms / 1e3),
                        "us_per_generation": ms * 1e3 / gens})
    # Every genome streams through HBM each generation (the grid is far larger
    # than what stays on chip).  Algorithmic bytes per agent-generation: the
    # 16-byte genome (trait, 64-bit surface, counter) read and written = 32 B,
    # plus the exchange state of its island spread over the island's 32
    # agents.  Latest-emigrant records: a 32-byte record written and read and
    # 16 B of seen-stamps read and written per island = 96 B / 32 = 3 B, for
    # 35 B.  Per-neighbour buffers: the island's lane state, channel words
    # and acknowledgements add 13 B per agent, for 45 B.  The ALU view: every replication draws one Philox block, against the
    # measured block rate of the generator.
    # the roofline line is the best whole-grid-together schedule (one
    # generation per octet visit); octet slices are reported beside it
    best = max((r for r in out if r["generations_per_octet_visit"] == 1),
               key=lambda r: r["value"], default=max(out, key=lambda r: r["value"]))
    bytes_per_agent = {"async": 35.0, "buffered": 45.0}[mode]
    peak, peak_kind = measured_peaks()
    gbs = best["value"] * bytes_per_agent / 1e9
    alu = alu_roofline(best["value"], philox_peak(stream))
    label = {"async": "free-running migration, latest-emigrant records",
             "buffered": "free-running migration, per-neighbour buffers"}[mode]
    # DRAM traffic from the committed ncu capture (bytes per generation; a
    # launch of K generations streams the grid K times)
    per_gen = profiled_traffic(f"{mode}_dram_bytes_per_generation", FREE_RUNNING_PROFILE,
                               FREE_RUNNING_SOURCES)
    traffic = per_gen * best["generations_per_launch"] if per_gen is not None else None
    print(json.dumps({"metric": "agent replications/sec", "unit": "agent replications/s",
                      "workload": f"wafer-shaped island GA, {label} "
                                  "(512x1024 islands x 32 agents)",
                      "config": dict(WORKLOAD, mode=mode), "slices": out,
                      "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                                   "frac": gbs / peak, "traffic": traffic,
                                   "traffic_per_generation": per_gen, "peak_kind": peak_kind,
                                   "generations_per_launch": best["generations_per_launch"],
                                   "algorithmic_bytes_per_agent_generation": bytes_per_agent},
                      "alu": alu,
                      "dtype": "u32",
                      "data": "synthetic"}), flush=True)


def run_wafer_full(args, mode):
    """The wafer-shaped workload as the paper runs it: free-running migration
    on the full 512 x 1024-island grid for args.full_gens generations
    (1,000,000 by default) from founders, then a 10,000-genome sample and its
    phylogeny reconstructed on the GPU (hsga_reconstruct) among the sampled
    genomes that share the modal deposition counter (free-running genomes
    carry their own counters).  The paper's own figure for this regime (a
    different machine, workload and genome) is context only."""
    import torch
    from paper_2404_10861_gb300 import _build, binding as hb
    _build.build()
    torch.cuda.set_device(0)
    hb.use_torch_allocator()
    stream = torch.cuda.Stream()
    K = 512
    total = args.full_gens
    with hb.Grid(stream=stream.cuda_stream, mode=mode, seed=1, **WORKLOAD) as g:
        g.run(K)                                   # warm-up launch (counted in the run)
        g.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        with ClockSampler(0) as clk:
            e0.record(stream)
            done = K
            while done < total:
                m = min(K, total - done)
                g.run(m)
                done += m
            e1.record(stream)
            e1.synchronize()
        wall = time.perf_counter() - t0
        gpu_s = e0.elapsed_time(e1) / 1e3
        timed = total - K
        words, where = g.sample(SAMPLE_K)
        trait, _ = g.population()
    T = words[:, 3].astype(np.int64)
    vals, counts = np.unique(T, return_counts=True)
    Tm = int(vals[np.argmax(counts)])
    pick = T == Tm
    surf = words[pick, 1].astype(np.uint64) | (words[pick, 2].astype(np.uint64) << np.uint64(32))
    t1 = time.perf_counter()
    parent, tm, leaf = hb.hsga_reconstruct(surf, "tilted", 1, 2, Tm, stream=stream.cuda_stream)
    rec_s = time.perf_counter() - t1
    root = parent < 0
    sbl = int((tm[~root] - tm[parent[~root]]).sum())
    print(json.dumps({
        "metric": "agent replications/sec", "unit": "agent replications/s",
        "workload": f"wafer-shaped island GA, free-running migration ({mode}), "
                    f"512x1024 islands x 32 agents, {total} generations from founders",
        "config": dict(WORKLOAD, mode=mode, generations=total, generations_per_launch=K),
        "value": AGENTS * timed / gpu_s, "generations_per_s": timed / gpu_s,
        "seconds_for_1M_generations": 1e6 * gpu_s / timed, "wall_s": wall,
        "clocks": clk.summary(),
        "sample": {"genomes": SAMPLE_K, "counter_min": int(T.min()), "counter_max": int(T.max()),
                   "counter_modal": Tm, "genomes_at_modal_counter": int(pick.sum()),
                   "distinct_counters": int(len(vals))},
        "reconstruction": {"genomes": int(pick.sum()), "nodes": int(len(parent)),
                           "sum_branch_length": sbl, "seconds": rec_s,
                           "engine": "hsga_reconstruct (GPU trie)"},
        "mean_trait": float(trait.mean()),
        "paper_context": "Cerebras CS-2, 750x750 PEs x 32 agents (18.0M), tournament 5, float "
                         "fitness: 1M generations in slightly under a minute (17,688 "
                         "generations/s); a different machine and workload",
        "dtype": "u32", "data": "synthetic"}), flush=True)


def run_reconstruct(args):
    """Phylogeny reconstruction from sampled surfaces of the wafer-shaped grid
    after 1,000 generations: the GPU trie (hsga_reconstruct, inputs and
    outputs resident on the device) for 10,000 genomes (the paper's sample
    size), 1M genomes and the whole 16.8M-agent population, beside the
    oracle's reconstruction of the 10,000-genome sample on one host core."""
    import time as _time
    import torch
    import oracle
    from oracle import phylo
    from paper_2404_10861_gb300 import _build, binding as hb
    _build.build()
    oracle.build()
    torch.cuda.set_device(0)
    hb.use_torch_allocator()
    stream = torch.cuda.Stream()
    G = 1000
    with hb.Grid(stream=stream.cuda_stream, seed=1, **WORKLOAD) as g:
        g.run(G)
        _, surf = g.population()
    rng = np.random.default_rng(0)
    out = []
    for k in (10_000, 1_000_000, AGENTS):
        pick = rng.choice(AGENTS, size=k, replace=False) if k < AGENTS else np.arange(AGENTS)
        s_dev = torch.from_numpy(surf[pick].view(np.int64)).cuda()
        cap = 2 * k + 1
        parent = torch.empty(cap, dtype=torch.int64, device="cuda")
        tm = torch.empty(cap, dtype=torch.int64, device="cuda")
        leaf = torch.empty(k, dtype=torch.int32, device="cuda")
        nodes = ctypes.c_uint32(0)

        def call():
            hb._check(hb.lib().hsga_reconstruct(
                s_dev.data_ptr(), k, 1, 1, 1, 2, G, 1, parent.data_ptr(), tm.data_ptr(),
                leaf.data_ptr(), cap, ctypes.byref(nodes), ctypes.c_void_p(stream.cuda_stream)),
                "hsga_reconstruct")
        for _ in range(args.warmup):
            call()
        reps = max(1, args.steps // 10)
        t0 = _time.perf_counter()
        for _ in range(reps):
            call()
        dt = (_time.perf_counter() - t0) / reps
        out.append({"genomes": k, "ms": dt * 1e3, "genomes_per_s": k / dt,
                    "nodes": nodes.value})
    k = 10_000
    pick = rng.choice(AGENTS, size=k, replace=False)
    t0 = _time.perf_counter()
    tree = phylo.reconstruct(surf[pick], 1, 1, 2, G)
    cpu = _time.perf_counter() - t0
    print(json.dumps({"metric": "genomes reconstructed/sec", "unit": "genomes/s",
                      "workload": "trie reconstruction of sampled surfaces, wafer-shaped grid "
                                  "(512x1024 islands x 32 agents) after 1,000 generations, "
                                  "64-bit tilted surface, 1-bit differentiae",
                      "gpu": out,
                      "cpu_baseline": {"value": k / cpu, "unit": "genomes/s", "cores": 1,
                                       "kind": "oracle", "sample": f"{k} genomes, "
                                       f"{tree.n_nodes} nodes, {cpu:.2f} s"},
                      "dtype": "u64", "data": "synthetic"}), flush=True)


def run_profile(gens: int):
    """Workload only, for profilers: founders, `gens` generations, one sample."""
    import torch
    from paper_2404_10861_gb300 import _build, binding as hb
    _build.build()
    torch.cuda.set_device(0)
    with hb.Grid(kernel=hb.KERNEL_STREAMED, seed=1, **WORKLOAD) as grid:
        grid.run(gens)
        grid.sample(SAMPLE_K)
        grid.sync()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=5,
                    help="steps of the end-to-end (host buffers) measurement")
    ap.add_argument("--profile-gens", type=int, default=0,
                    help="profiling mode: only run this many generations of the workload "
                         "(no timing); used for ncu captures")
    ap.add_argument("--workload", default="wafer",
                    choices=["wafer", "tiny", "mid", "batched", "served", "async", "buffered",
                             "reconstruct", "async-full", "buffered-full"],
                    help="wafer: the benchmark line; the others: informational lines")
    ap.add_argument("--requests", type=int, default=2000, help="served workload: requests")
    ap.add_argument("--memory-cap-mb", type=int, default=0,
                    help="served workload: device memory cap for admission (default: 90%% of "
                         "the device's free memory)")
    ap.add_argument("--gen-scale", type=int, default=None,
                    help="batched / served workloads: divide the generation budgets by this "
                         "(default 1: the stated budgets)")
    ap.add_argument("--slices", type=int, nargs="+", default=[1, 8, 64, 512],
                    help="async workload: generations per launch to measure")
    ap.add_argument("--full-gens", type=int, default=1_000_000,
                    help="async-full / buffered-full workloads: generations from founders")
    ap.add_argument("--octet-slices", type=int, nargs="+", default=[1],
                    help="async / buffered workloads: generations per octet visit to measure "
                         "(hsga_set_octet_slice; 1 = the whole grid one generation at a time)")
    ap.add_argument("--async-gens", type=int, default=2048,
                    help="async workload: timed generations per slice length")
    args = ap.parse_args()
    if args.workload in ("async", "buffered"):
        run_async_wafer(args, args.workload)
        return
    if args.workload == "reconstruct":
        run_reconstruct(args)
        return
    if args.workload in ("async-full", "buffered-full"):
        run_wafer_full(args, args.workload.split("-")[0])
        return
    if args.workload == "batched":
        run_batched(args)
        return
    if args.workload == "served":
        run_served(args)
        return
    if args.workload != "wafer":
        if args.warmup < 3:
            args.warmup = 3
        run_secondary(args)
        return
    if args.profile_gens:
        run_profile(args.profile_gens)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
