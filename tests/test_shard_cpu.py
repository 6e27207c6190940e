"""The sharded step's plan and halo exchange on CPU: 2 and 3 gloo ranks, one
shard each.  Every rank fills its own tiles from the oracle's state, runs the
exchange (torch.distributed point-to-point calls, the same code the GPU path
uses), and checks against the oracle that

* the shards' own tiles partition the instance in omega order;
* every received halo tile holds the oracle's cells of that tile;
* for every own tile and Moore direction, the buffer slot the shard's
  neighbour table names holds the oracle's neighbouring tile (found
  independently with the oracle's lambda and nu one level of tiles up), and
  the slot is -1 exactly where the oracle finds no neighbour.

Nothing here needs a GPU: the plan is computed by the library on the host."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2110_12952_gb300 import workloads as W

CASES = [("triangle", 8, 3), ("carpet", 4, 1), ("vicsek", 5, 2), ("menger", 3, 1)]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _check_rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2110_12952_gb300.shard import ShardPlan, exchange_dist
        res = []
        for name, r, L in CASES:
            fam = W.FAMILIES[name]
            o = oracle.Fractal(fam.k, fam.s, r, fam.dim, fam.table())
            state = o.init_bernoulli(55 + r, 0.5)
            kl = fam.k ** L
            p = ShardPlan.from_family(fam, r, L, world, rank)
            buf = torch.zeros(p.buffer_cells, dtype=torch.uint8)
            own = slice(p.first_cell, p.first_cell + p.local_cells)
            buf[: p.local_cells] = torch.from_numpy(state[own].copy())
            exchange_dist(p, buf, dist)
            b = buf.numpy()
            ok_recv = True
            for peer in range(world):
                if peer == rank:
                    continue
                tiles, dst = p.recvs(peer)
                got = b[dst: dst + len(tiles) * kl].reshape(-1, kl)
                want = np.stack([state[t * kl:(t + 1) * kl] for t in tiles]) if len(tiles) else got
                ok_recv &= bool(np.array_equal(got, want))
            # neighbours of every own tile, from the oracle one level of tiles up
            coarse = oracle.Fractal(fam.k, fam.s, r - L, fam.dim, fam.table())
            table = p.neighbours()
            t0 = p.first_cell // kl
            ntl = p.local_cells // kl
            c = coarse.lam(np.arange(t0, t0 + ntl))
            ok_nb = True
            d = 0
            for q in range(3 ** fam.dim):
                dd = [q % 3 - 1, (q // 3) % 3 - 1, q // 9 - 1][: fam.dim]
                if not any(dd):
                    continue
                tn = coarse.nu(c + np.asarray(dd)[None, :])
                slot = table[:, d]
                ok_nb &= bool(np.array_equal(slot < 0, tn < 0))
                for i in np.nonzero(tn >= 0)[0]:
                    ok_nb &= bool(np.array_equal(b[slot[i] * kl:(slot[i] + 1) * kl],
                                                 state[tn[i] * kl:(tn[i] + 1) * kl]))
                d += 1
            res.append((name, p.first_cell, p.local_cells, ok_recv, ok_nb))
            p.close()
        out[rank] = res
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_shard_exchange_matches_oracle(world):
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_check_rank, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
        results = [out[r] for r in range(world)]
    for ci, (name, r, L) in enumerate(CASES):
        fam = W.FAMILIES[name]
        spans = sorted((res[ci][1], res[ci][2]) for res in results)
        # own tiles partition the instance in omega order
        pos = 0
        for first, n in spans:
            assert first == pos
            pos += n
        assert pos == fam.k ** r
        for res in results:
            assert res[ci][3], f"{name}: received halo differs from the oracle's tiles"
            assert res[ci][4], f"{name}: neighbour slots differ from the oracle's neighbours"


def test_shard_plan_rejects_bad_arguments():
    from paper_2110_12952_gb300.capi import FractalError
    from paper_2110_12952_gb300.shard import ShardPlan
    with pytest.raises(FractalError, match="EINVAL"):
        ShardPlan.from_family(W.TRIANGLE, 4, 4, 2, 0)       # one tile, two shards
    with pytest.raises(FractalError, match="EINVAL"):
        ShardPlan.from_family(W.TRIANGLE, 4, 2, 2, 2)       # shard index out of range
    p = ShardPlan.from_family(W.TRIANGLE, 6, 2, 1, 0)       # one shard: no halo
    assert p.local_cells == p.buffer_cells == 3 ** 6 and p.first_cell == 0
    p.close()
