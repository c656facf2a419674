"""Window-sharded REWL: the windows of one run split over several handles (one per GPU).

Sec. 2: walkers of different energy windows meet only in the exchange of Eq. (1) between
neighbouring windows, so a run shards into consecutive window ranges with one exchange per
round across each shard boundary.  Each shard is a handle with `rewl_set_shard`; after every
round the pair across a boundary trades bins, halves of ln P and accepted lattices through the
library's boundary calls.  This module only sequences those calls and moves their buffers
through a transport the caller picks (in-process copies, or torch.distributed point-to-point).
"""
from __future__ import annotations

import numpy as np
import torch

from . import rewl as R


def split_windows(h: int, parts: int):
    """Consecutive window ranges [(w_begin, count), ...] of nearly equal size."""
    if parts < 1 or parts > h // 2:
        raise ValueError("every shard needs at least two windows")
    base, extra = divmod(h, parts)
    out, w = [], 0
    for p in range(parts):
        n = base + (1 if p < extra else 0)
        out.append((w, n))
        w += n
    return out


class Boundary:
    """Device buffers of one side of a shard boundary (side 1: the shard's last window, side 0:
    its first)."""

    def __init__(self, handle: R.REWL, side: int, device):
        m, N = handle.m, handle.N
        self.side = side
        self.bins = torch.zeros(m, dtype=torch.int32, device=device)
        self.pbins = torch.zeros_like(self.bins)
        self.half = torch.zeros(m, dtype=torch.float64, device=device)
        self.phalf = torch.zeros_like(self.half)
        self.acc = torch.zeros(m, dtype=torch.uint8, device=device)
        self.lat = torch.zeros((m, N), dtype=torch.int8, device=device)
        self.plat = torch.zeros_like(self.lat)


def make_shard(model, L, lo, hi, w_begin, count, walkers, lnf_final, flatness, seed, **params):
    """A handle for windows w_begin .. w_begin + count - 1 of the global layout (lo, hi)."""
    r = R.REWL(model, L, count, 0.75, walkers, lnf_final, flatness, seed=seed, **params)
    r.set_shard(np.asarray(lo, np.int32), np.asarray(hi, np.int32), w_begin)
    return r


def exchange(shards, transfer):
    """The boundary exchange after a round.  `shards` is a list of (handle, [Boundary, ...]);
    `transfer(field)` must fill every boundary's partner buffer p<field> with the partner's
    <field> (bins, half, lat) before the next call runs on the handles' streams."""
    for h, bs in shards:
        for b in bs:
            h.boundary_bins(b.side, b.bins)
    transfer("bins")
    for h, bs in shards:
        for b in bs:
            h.boundary_half(b.side, b.pbins, b.half)
    transfer("half")
    for h, bs in shards:
        for b in bs:
            h.boundary_decide(b.side, b.half, b.phalf, b.acc, b.lat)
    transfer("lat")
    for h, bs in shards:
        for b in bs:
            h.boundary_import(b.side, b.pbins, b.acc, b.plat)


class LocalShards:
    """Several shards of one run in one process (one device): the transport is a device copy
    between neighbouring shards' buffers."""

    def __init__(self, handles, device="cuda"):
        self.handles = handles
        self.bounds = []
        for i, h in enumerate(handles):
            bs = []
            if i > 0:
                bs.append(Boundary(h, 0, device))
            if i + 1 < len(handles):
                bs.append(Boundary(h, 1, device))
            self.bounds.append(bs)

    def _transfer(self, field):
        for i in range(len(self.handles) - 1):
            up = [b for b in self.bounds[i] if b.side == 1][0]
            down = [b for b in self.bounds[i + 1] if b.side == 0][0]
            getattr(up, "p" + field).copy_(getattr(down, field))
            getattr(down, "p" + field).copy_(getattr(up, field))

    def step(self, rounds: int = 1):
        for _ in range(rounds):
            for h in self.handles:
                h.step(1)
            exchange(list(zip(self.handles, self.bounds)), self._transfer)

    def finished(self) -> bool:
        return all(h.stats()["windows_finished"] == h.h for h in self.handles)

    def run(self, max_rounds: int):
        """Rounds until every window of every shard finished (or max_rounds); returns rounds."""
        n = 0
        while n < max_rounds and not self.finished():
            self.step(1)
            n += 1
        return n


class DistShard:
    """One shard per rank of a torch.distributed group; neighbouring ranks hold neighbouring
    window ranges.  With the gloo backend the buffers travel through host memory."""

    def __init__(self, handle, rank: int, world: int, device):
        import torch.distributed as dist
        self.dist = dist
        self.handle, self.rank, self.world = handle, rank, world
        self.bounds = []
        if rank > 0:
            self.bounds.append(Boundary(handle, 0, device))
        if rank + 1 < world:
            self.bounds.append(Boundary(handle, 1, device))
        self.host = dist.get_backend() == "gloo"

    def _transfer(self, field):
        ops, copies = [], []
        for b in self.bounds:
            peer = self.rank - 1 if b.side == 0 else self.rank + 1
            send, recv = getattr(b, field), getattr(b, "p" + field)
            if self.host:
                s_h, r_h = send.cpu(), torch.empty_like(recv, device="cpu")
                copies.append((recv, r_h))
                send, recv = s_h, r_h
            ops.append(self.dist.P2POp(self.dist.isend, send, peer))
            ops.append(self.dist.P2POp(self.dist.irecv, recv, peer))
        if ops:
            for w in self.dist.batch_isend_irecv(ops):
                w.wait()
        for dev, h in copies:
            dev.copy_(h)

    def step(self, rounds: int = 1):
        for _ in range(rounds):
            self.handle.step(1)
            exchange([(self.handle, self.bounds)], self._transfer)

    def finished(self) -> bool:
        """All windows of all ranks finished (one all-reduce)."""
        mine = int(self.handle.stats()["windows_finished"] == self.handle.h)
        t = torch.tensor([mine], dtype=torch.int32,
                         device="cpu" if self.host else torch.device("cuda", torch.cuda.current_device()))
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MIN)
        return bool(t.item())
