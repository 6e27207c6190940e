"""Python binding of the sharded step (``fractal_shard_*`` in
``include/fractal.h``): one instance split into contiguous tile ranges, one
per shard, with a halo of neighbouring tiles exchanged every generation.

``ShardPlan`` marshals arguments only: the plan is computed by the library on
the host, the gathers and the step run in its CUDA kernels.  Moving the send
buffers is plain data movement: ``exchange_dist`` uses torch.distributed
point-to-point calls (NCCL between GPUs, gloo on CPU tensors) and
``exchange_local`` device copies when several shards share one GPU.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import capi


class ShardPlan:
    """Shard ``shard`` of ``nshards`` of the level-``r`` fractal with tile depth
    ``tile_levels`` (``fractal_shard_plan``; host only, no GPU needed)."""

    def __init__(self, k, s, r, dim, offsets, tile_levels, nshards, shard):
        self._lib = capi.load()
        off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32).reshape(k * dim))
        h = capi.c_vp()
        capi.check(self._lib.fractal_shard_plan(k, s, r, dim, off.ctypes.data_as(capi.c_i32p), tile_levels,
                                                nshards, shard, ctypes.byref(h)), self._lib)
        self._h = h
        self.k, self.s, self.r, self.dim = k, s, r, dim
        self.tile_levels, self.nshards, self.shard = tile_levels, nshards, shard
        self.tile_cells = k ** tile_levels
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        capi.check(self._lib.fractal_shard_info(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), self._lib)
        self.first_cell, self.local_cells, self.buffer_cells = a.value, b.value, c.value
        self._fr = None

    @classmethod
    def from_family(cls, fam, r, tile_levels, nshards, shard):
        return cls(fam.k, fam.s, r, fam.dim, fam.table(), tile_levels, nshards, shard)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.fractal_shard_destroy(self._h)
            self._h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def _list(self, fn, peer):
        n, dst = ctypes.c_int64(), ctypes.c_int64()
        capi.check(fn(self._h, peer, None, 0, ctypes.byref(n), ctypes.byref(dst)), self._lib)
        tiles = np.zeros(n.value, dtype=np.int64)
        capi.check(fn(self._h, peer, tiles.ctypes.data_as(capi.c_i64p), n.value, ctypes.byref(n),
                      ctypes.byref(dst)), self._lib)
        return tiles, dst.value

    def sends(self, peer):
        """(global tiles sent to ``peer``, first cell of their block in the peer's buffer)."""
        return self._list(self._lib.fractal_shard_sends, peer)

    def recvs(self, peer):
        """(global tiles received from ``peer``, first cell of their block in this buffer)."""
        return self._list(self._lib.fractal_shard_recvs, peer)

    def neighbours(self) -> np.ndarray:
        """(own tiles, 3^dim - 1) table of buffer tile slots, -1 = none."""
        ndir = 3 ** self.dim - 1
        n = self.local_cells // self.tile_cells
        t = np.zeros((n, ndir), dtype=np.int32)
        capi.check(self._lib.fractal_shard_neighbours(self._h, t.ctypes.data_as(capi.c_i32p), t.size), self._lib)
        return t

    # ------------------------------------------------------------ device
    def attach(self, fr):
        """Bind to a ``Fractal`` handle of the same fractal (sets its tile depth)."""
        capi.check(self._lib.fractal_shard_attach(self._h, fr._h), self._lib)
        self._fr = fr

    def pack(self, peer, buffer, send=None, stream=None):
        import torch
        tiles, _ = self.sends(peer)
        n = len(tiles) * self.tile_cells
        if send is None:
            send = torch.empty(n, dtype=torch.uint8, device=buffer.device)
        s = stream if stream is not None else torch.cuda.current_stream()
        capi.check(self._lib.fractal_shard_pack(self._h, peer, buffer.data_ptr(), send.data_ptr() if n else None,
                                                s.cuda_stream), self._lib)
        return send

    def step(self, buf_in, buf_out, rule=None, stream=None):
        import torch
        from .workloads import Family, default_rule
        if rule is None:
            rule = default_rule(Family("", self.k, self.s, self.dim, ()))
        s = stream if stream is not None else torch.cuda.current_stream()
        capi.check(self._lib.fractal_shard_step(self._h, buf_in.data_ptr(), buf_out.data_ptr(), rule[0], rule[1],
                                                s.cuda_stream), self._lib)


def exchange_local(plans, buffers):
    """Halo exchange between shards that share one GPU: each shard's gathered
    tiles are copied into each peer's buffer at the offset the plan gives."""
    for g, p in enumerate(plans):
        for h in range(len(plans)):
            if h == g:
                continue
            tiles, dst = p.sends(h)
            if len(tiles) == 0:
                continue
            send = p.pack(h, buffers[g])
            buffers[h][dst:dst + send.numel()].copy_(send)


def exchange_dist(plan, buffer, dist, group=None):
    """Halo exchange of this rank's shard with torch.distributed
    point-to-point calls: gathered tiles to every peer that needs some, and
    the peers' tiles straight into this rank's buffer."""
    ops, keep = [], []
    for peer in range(plan.nshards):
        if peer == plan.shard:
            continue
        tiles, _ = plan.sends(peer)
        if len(tiles):
            send = plan.pack(peer, buffer) if buffer.is_cuda else pack_host(plan, peer, buffer)
            keep.append(send)
            ops.append(dist.P2POp(dist.isend, send, peer, group))
        rtiles, rdst = plan.recvs(peer)
        if len(rtiles):
            ops.append(dist.P2POp(dist.irecv, buffer[rdst:rdst + len(rtiles) * plan.tile_cells], peer, group))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()


def pack_host(plan, peer, buffer):
    """The gather of ``fractal_shard_pack`` for a CPU tensor (data movement
    only; used by CPU runs of the exchange)."""
    import torch
    tiles, _ = plan.sends(peer)
    local = (tiles - plan.first_cell // plan.tile_cells).astype(np.int64)
    kl = plan.tile_cells
    idx = (local[:, None] * kl + np.arange(kl, dtype=np.int64)[None, :]).reshape(-1)
    return buffer[torch.from_numpy(idx)].contiguous()
