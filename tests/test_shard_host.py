"""Host side of window-sharded runs (no device): the split of a layout into consecutive
shards, and the transport bookkeeping of DistShard over two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def test_split_windows_consecutive_and_balanced():
    from paper_1402_2328_gb300 import shard as S
    for h in (4, 6, 7, 32, 64):
        for parts in range(1, h // 2 + 1):
            sp = S.split_windows(h, parts)
            assert len(sp) == parts
            assert sp[0][0] == 0 and sum(n for _, n in sp) == h
            assert all(b == a + n for (a, n), (b, _) in zip(sp, sp[1:]))
            assert max(n for _, n in sp) - min(n for _, n in sp) <= 1
            assert min(n for _, n in sp) >= 2
    for h, parts in ((5, 3), (4, 3), (8, 0)):
        with pytest.raises(ValueError):
            S.split_windows(h, parts)


class _FakeHandle:
    m, N, h = 3, 4, 2


def _rank(rank, port, out):
    import torch.distributed as dist
    from paper_1402_2328_gb300 import shard as S
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=2)
    d = S.DistShard(_FakeHandle(), rank, 2, "cpu")
    assert [b.side for b in d.bounds] == ([1] if rank == 0 else [0])
    b = d.bounds[0]
    b.bins.fill_(10 + rank)
    b.half.fill_(0.5 + rank)
    b.lat.fill_(rank + 1)
    for f in ("bins", "half", "lat"):
        d._transfer(f)
    other = 1 - rank
    ok = (bool((b.pbins == 10 + other).all()) and bool((b.phalf == 0.5 + other).all()) and
          bool((b.plat == other + 1).all()))
    open(os.path.join(out, f"r{rank}"), "w").write("ok" if ok else "bad")
    dist.destroy_process_group()


def test_dist_transfer_two_gloo_ranks(tmp_path):
    """Each side's buffers arrive in the partner's p-buffers (the three transfers of a round)."""
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.start_processes(_rank, args=(port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    assert [open(tmp_path / f"r{r}").read() for r in range(2)] == ["ok", "ok"]
