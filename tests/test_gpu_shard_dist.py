"""Window-sharded run over two torch.distributed ranks (gloo transport through host memory),
against the single-handle run, bit for bit.  Both ranks share the one GPU of the test box; their
kernels never wait on each other (the exchange goes through the host between rounds)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ARGS = dict(model=0, L=8, h=6, m=2, lnf_final=1e-3, interval=500, seed=83)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, lo, hi, out_dir):
    import torch
    import torch.distributed as dist
    from paper_1402_2328_gb300 import shard as S
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    a = ARGS
    wb, n = S.split_windows(a["h"], world)[rank]
    h = S.make_shard(a["model"], a["L"], lo, hi, wb, n, a["m"], a["lnf_final"], 0.8, a["seed"],
                     interval=a["interval"])
    h.init()
    d = S.DistShard(h, rank, world, "cuda")
    rounds = 0
    while rounds < 100_000 and not d.finished():
        d.step(1)
        rounds += 1
    st = h.state()
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), rounds=rounds,
             **{k: np.asarray(v) for k, v in st.items()})
    h.close()
    dist.destroy_process_group()


def test_two_ranks_gloo_equal_single_run(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_2328_gb300 import build as B
    B.build()
    import torch.multiprocessing as mp
    import paper_1402_2328_gb300.rewl as R
    a = ARGS
    full = R.REWL(a["model"], a["L"], a["h"], 0.75, a["m"], a["lnf_final"], 0.8, seed=a["seed"],
                  interval=a["interval"])
    full.init()
    lo, hi = full.get_state("lo"), full.get_state("hi")
    assert full.run() == "done"
    fs = full.state()
    mp.start_processes(_rank_main, args=(2, _free_port(), lo, hi, str(tmp_path)), nprocs=2,
                       join=True, start_method="spawn")
    parts = [np.load(tmp_path / f"rank{r}.npz") for r in range(2)]
    assert all(int(p["rounds"]) == fs["round"] for p in parts)
    w = 0
    for p in parts:
        nwin = p["lnf"].shape[0]
        for lw in range(nwin):
            nb = int(hi[w] - lo[w] + 1)
            for f in ("lnf", "iter", "finished", "swap_att", "swap_acc"):
                assert np.array_equal(np.asarray(fs[f])[w], p[f][lw]), (f, w)
            for i in range(a["m"]):
                g, l_ = w * a["m"] + i, lw * a["m"] + i
                for f in ("spins", "k", "step", "acc"):
                    assert np.array_equal(np.asarray(fs[f])[g], p[f][l_]), (f, w, i)
                for f in ("lng", "H"):
                    x, y = np.asarray(fs[f])[g][:nb], p[f][l_][:nb]
                    assert np.array_equal(x.view(np.uint64) if x.dtype == np.float64 else x,
                                          y.view(np.uint64) if y.dtype == np.float64 else y), f
            w += 1
    assert w == a["h"]
    full.close()
