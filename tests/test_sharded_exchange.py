"""The window-sharded exchange on CPU ranks (gloo, world size 2).

Rank 0 owns windows [0, h/2), rank 1 owns [h/2, h).  The exchange of the boundary pair
(w, w+1) = (h/2-1, h/2) (Sec. 2, Eq. 1) runs as messages: the partners' bins k_X / k_Y go both
ways, each rank computes its own half of ln P from its own ln g rows, rank 1 sends its halves,
rank 0 draws the permutation and the acceptance words, decides, and the accepted lattices and
bins are exchanged.  Both ranks' rows must equal the single-process exchange bit for bit.
"""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as tmp

import oracle as O

H, M, L = 4, 3, 6
SEED, INST = 0xBEEF, 0


ROUNDS = (9, 13, 17, 21, 25, 29)  # states the exchange is tried on (odd: pair (1, 2))


def _state(n):
    r = O.REWL(0, L, H, 0.75, M, 1e-3, 0.8, seed=SEED, instance=INST, interval=150)
    assert r.init() == 0
    r.run(n)
    return r


def _philox(c0, c1, c2, tag):
    return O.philox([c0 & 0xFFFFFFFF, c1 & 0xFFFFFFFF, c2, tag], [SEED & 0xFFFFFFFF, SEED >> 32])


def _mulhi(a, b):
    return (int(a) * int(b)) >> 32


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"], os.environ["MASTER_PORT"] = "127.0.0.1", str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    for n in ROUNDS:
        out[(rank, n)] = _exchange(rank, n)
    dist.destroy_process_group()


def _exchange(rank, n):
    import torch
    r = _state(n)
    st = r.state()
    rd = int(st["round"]) | 1  # an odd round pairs (1, 2): the boundary pair for h = 4
    w = H // 2 - 1
    lo, hi = r.lo, r.hi
    mine = w if rank == 0 else w + 1
    rows = slice(mine * M, (mine + 1) * M)
    k = st["k"][rows].astype(np.int64).copy()
    lng = st["lng"][rows].copy()
    spins = st["spins"][rows].copy()
    # 1. bins both ways
    other = torch.zeros(M, dtype=torch.int64)
    sendk = torch.from_numpy(k)
    if rank == 0:
        dist.send(sendk, 1); dist.recv(other, 1)
    else:
        dist.recv(other, 0); dist.send(sendk, 0)
    kX = k if rank == 0 else other.numpy()      # bins of window w's walkers
    kY = other.numpy() if rank == 0 else k      # bins of window w+1's walkers
    tag = (INST << 8) | 3
    # 2. permutation (Fisher-Yates from the swap stream), computed by both ranks
    perm = list(range(M))
    for i in range(M - 1, 0, -1):
        j = _mulhi(_philox(i, rd, w, tag)[0], i + 1)
        perm[i], perm[j] = perm[j], perm[i]
    lo_a, hi_a, lo_b, hi_b = lo[w], hi[w], lo[w + 1], hi[w + 1]
    ok = [lo_b <= kX[i] <= hi_b and lo_a <= kY[perm[i]] <= hi_a for i in range(M)]
    # 3. each rank's half of ln P from its own rows
    half = np.zeros(M)
    for i in range(M):
        if not ok[i]:
            continue
        if rank == 0:   # lg_i[kX] - lg_i[kY] of walker i of window w
            half[i] = lng[i, kX[i] - lo_a] - lng[i, kY[perm[i]] - lo_a]
        else:           # lg_j[kY] - lg_j[kX] of walker perm[i] of window w+1
            j = perm[i]
            half[i] = lng[j, kY[j] - lo_b] - lng[j, kX[i] - lo_b]
    t_half = torch.from_numpy(half)
    acc = torch.zeros(M, dtype=torch.int64)
    if rank == 1:
        dist.send(t_half, 0)
        dist.recv(acc, 0)
    else:
        other_half = torch.zeros(M, dtype=torch.float64)
        dist.recv(other_half, 1)
        for i in range(M):
            if not ok[i]:
                continue
            lnP = half[i] + float(other_half[i])
            a = lnP >= 0.0 or O.lnu(int(_philox(M + i, rd, w, tag)[0])) < lnP
            acc[i] = int(a)
        dist.send(acc, 1)
    # 4. accepted pairs swap lattice and bin
    for i in range(M):
        if not acc[i]:
            continue
        mine_i = i if rank == 0 else perm[i]
        buf = torch.from_numpy(spins[mine_i].copy())
        got = torch.zeros_like(buf)
        if rank == 0:
            dist.send(buf, 1); dist.recv(got, 1)
        else:
            dist.recv(got, 0); dist.send(buf, 0)
        spins[mine_i] = got.numpy()
        k[mine_i] = kY[perm[i]] if rank == 0 else kX[i]
    return (k.copy(), spins.copy(), int(acc.sum()), rd)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_rank_exchange_equals_single_process():
    mgr = tmp.Manager()
    out = mgr.dict()
    port = _free_port()
    tmp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
    w = H // 2 - 1
    accepted = attempted = 0
    for n in ROUNDS:
        rd = out[(0, n)][3]
        ref = _state(n)
        before = ref.state()
        ref.swap(w, rd)
        after = ref.state()
        for rank, win in ((0, w), (1, w + 1)):
            k, spins, nacc, _ = out[(rank, n)]
            rows = slice(win * M, (win + 1) * M)
            assert np.array_equal(k, after["k"][rows])
            assert np.array_equal(spins, after["spins"][rows])
        assert out[(0, n)][2] == out[(1, n)][2] == int(after["swap_acc"][w] - before["swap_acc"][w])
        accepted += out[(0, n)][2]
        attempted += int(after["swap_att"][w] - before["swap_att"][w])
    assert 0 < accepted < attempted  # both outcomes occurred
