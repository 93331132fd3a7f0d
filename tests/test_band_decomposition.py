"""Multi-rank decomposition of the island grid, on CPU ranks (gloo, world
sizes 2 and 3): the torus split into row bands, each rank advancing its band
with the oracle's step functions and exchanging only the emigrant records of
its first and last rows with the two neighbouring bands every generation
(point-to-point sends and receives, no collective), must equal the
single-domain run bit-exactly.  This is the exchange a multi-GPU run would
perform (one 16-byte record per boundary island per generation, to the band
above and the band below).
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def band_rows(R, world, rank):
    base, extra = divmod(R, world)
    r0 = rank * base + min(rank, extra)
    return r0, r0 + base + (1 if rank < extra else 0)


def worker(rank, world, port, kw, G, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    oracle.build()
    cfg = oracle.Config(**kw)
    R, C, n = cfg.rows, cfg.cols, cfg.n
    r0, r1 = band_rows(R, world, rank)
    B = r1 - r0
    band_gid = np.array([r * C + c for r in range(r0, r1) for c in range(C)], dtype=np.uint32)
    top = (r0 - 1) % R
    bot = r1 % R
    halo_gid = np.array([top * C + c for c in range(C)] + [bot * C + c for c in range(C)],
                        dtype=np.uint32)
    gid = np.concatenate([band_gid, halo_gid])
    L = len(gid)
    nbr = np.zeros((L, 4), dtype=np.int32)
    for li in range(B * C):
        r, c = divmod(li, C)
        nbr[li, 0] = B * C + c if r == 0 else li - C                       # N
        nbr[li, 2] = B * C + C + c if r == B - 1 else li + C               # S
        nbr[li, 1] = r * C + (c + 1) % C                                   # E
        nbr[li, 3] = r * C + (c - 1) % C                                   # W
    active = np.zeros(L, dtype=np.uint8)
    active[:B * C] = 1
    trait = np.zeros(L * n, dtype=np.uint32)
    surf = np.zeros(L * n, dtype=np.uint64)
    up, down = (rank - 1) % world, (rank + 1) % world   # owners of rows top and bot
    FIRST, LAST = 1, 2                                   # message tags: which row is sent
    for G_ in range(G):
        rec = oracle.emigrate(cfg, band_gid, trait[:B * C * n], surf[:B * C * n], G_)
        # my first row is the bottom halo of the band above, my last row the
        # top halo of the band below; receive theirs in turn
        first = torch.from_numpy(rec[:C].astype(np.int64))
        last = torch.from_numpy(rec[-C:].astype(np.int64))
        top_halo = torch.zeros_like(first)
        bot_halo = torch.zeros_like(last)
        reqs = [dist.isend(first, up, tag=FIRST), dist.isend(last, down, tag=LAST),
                dist.irecv(top_halo, up, tag=LAST), dist.irecv(bot_halo, down, tag=FIRST)]
        for q in reqs:
            q.wait()
        rec_local = np.concatenate([rec, top_halo.numpy().astype(np.uint32),
                                    bot_halo.numpy().astype(np.uint32)])
        t2, s2 = oracle.immigrate_select(cfg, gid, nbr.reshape(-1), active, trait, surf,
                                         rec_local, G_)
        trait[:B * C * n] = t2[:B * C * n]
        surf[:B * C * n] = s2[:B * C * n]
    np.savez(out_path + f".{rank}.npz", trait=trait[:B * C * n], surf=surf[:B * C * n])
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,rows,cols,G", [(2, 6, 5, 40), (2, 5, 4, 25), (2, 3, 7, 30),
                                               (3, 7, 4, 30), (3, 3, 5, 20)])
def test_row_bands_equal_single_domain(orc, tmp_path, world, rows, cols, G):
    kw = dict(rows=rows, cols=cols, n=8, tournament=2, policy=orc.TILTED, bits=2, W=2,
              interval=1, p_ben=0.02, p_del=0.01, seed=31)
    out = str(tmp_path / "band")
    mp.start_processes(worker, args=(world, free_port(), kw, G, out), nprocs=world,
                       join=True, start_method="spawn")
    parts = [np.load(out + f".{r}.npz") for r in range(world)]
    trait = np.concatenate([p["trait"] for p in parts])
    surf = np.concatenate([p["surf"] for p in parts])
    want_t, want_s, _ = orc.run(orc.Config(**kw), generations=G)
    assert np.array_equal(trait, want_t)
    assert np.array_equal(surf, want_s)
