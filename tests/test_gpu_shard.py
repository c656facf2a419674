"""Window-sharded runs against the single-handle run, bit for bit (Sec. 2, Eq. 1 across shards).

Several shards of consecutive windows (rewl_set_shard) advance round by round; after every
round the pair across each shard boundary exchanges through the library's boundary calls.
The shards' state, put side by side, must equal one handle's state over all windows.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PER_SLOT = ["spins", "k", "lng", "H", "step", "acc", "flat", "frag"]
PER_WIN = ["lnf", "iter", "finished", "mask", "swap_att", "swap_acc", "first_iter_round", "mode"]


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_2328_gb300 import build as B
    B.build()
    import paper_1402_2328_gb300.rewl as R
    return R


def _bits(a):
    a = np.asarray(a)
    return a.view(np.uint64) if a.dtype == np.float64 else a


def _compare(full, shards):
    fs = full.state()
    lo, hi = full.get_state("lo"), full.get_state("hi")
    m, w = full.m, 0
    for sh in shards:
        ss = sh.state()
        assert ss["round"] == fs["round"]
        for lw in range(sh.h):
            nb = int(hi[w] - lo[w] + 1)
            for f in PER_WIN:
                a, b = np.asarray(fs[f])[w], np.asarray(ss[f])[lw]
                if f == "mask":
                    a, b = a[:nb], b[:nb]
                assert np.array_equal(_bits(a), _bits(b)), (f, w)
            for i in range(m):
                g, l_ = w * m + i, lw * m + i
                for f in PER_SLOT:
                    a, b = np.asarray(fs[f])[g], np.asarray(ss[f])[l_]
                    if f in ("lng", "H", "frag"):
                        a, b = a[:nb], b[:nb]
                    assert np.array_equal(_bits(a), _bits(b)), (f, w, i)
            w += 1
    assert w == full.h


@pytest.mark.parametrize("model,L,h,m,parts,interval,lnf_final", [
    (0, 8, 6, 3, 2, 500, 1e-4), (0, 8, 6, 2, 3, 400, 1e-4), (3, 6, 5, 2, 2, 300, 1e-4),
    (10, 12, 8, 2, 4, 700, 1e-4)])
def test_shards_equal_single_run(R, model, L, h, m, parts, interval, lnf_final):
    from paper_1402_2328_gb300 import shard as S
    seed = 71 + L + model
    full = R.REWL(model, L, h, 0.75, m, lnf_final, 0.8, seed=seed, interval=interval, schedule=1)
    full.init()
    lo, hi = full.get_state("lo"), full.get_state("hi")
    handles = [S.make_shard(model, L, lo, hi, wb, n, m, lnf_final, 0.8, seed, interval=interval,
                            schedule=1)
               for wb, n in S.split_windows(h, parts)]
    for x in handles:
        x.init()
    group = S.LocalShards(handles)
    _compare(full, handles)
    for chunk in (1, 5, 30):
        full.run(max_rounds=chunk)
        group.step(chunk)
        torch.cuda.synchronize()
        _compare(full, handles)
    assert sum(int(x.get_state("swap_acc").sum()) for x in handles) > 0
    full.close()
    for x in handles:
        x.close()


def test_shards_run_to_completion(R):
    from paper_1402_2328_gb300 import shard as S
    model, L, h, m, seed = 0, 6, 4, 2, 5
    full = R.REWL(model, L, h, 0.75, m, 1e-3, 0.8, seed=seed, interval=400)
    full.init()
    lo, hi = full.get_state("lo"), full.get_state("hi")
    handles = [S.make_shard(model, L, lo, hi, wb, n, m, 1e-3, 0.8, seed, interval=400)
               for wb, n in S.split_windows(h, 2)]
    assert full.run() == "done"
    for x in handles:
        x.init()
    rounds = S.LocalShards(handles).run(10 ** 6)
    assert rounds == full.get_state("round")[0]
    _compare(full, handles)
    full.close()
    for x in handles:
        x.close()


def test_shard_refusals(R):
    from paper_1402_2328_gb300 import shard as S
    full = R.REWL(0, 8, 6, 0.75, 1, 1e-3, 0.8)
    full.init()
    lo, hi = full.get_state("lo"), full.get_state("hi")
    x = R.REWL(0, 8, 3, 0.75, 1, 1e-3, 0.8)
    with pytest.raises(R.REWLError):
        x.set_shard(lo, hi, 4)              # windows 4..6 do not exist
    bad = hi.copy()
    bad[-1] -= 1
    with pytest.raises(R.REWLError):
        x.set_shard(lo, bad, 0)             # the layout must end at B
    x.set_shard(lo, hi, 0)
    with pytest.raises(R.REWLError):
        x.set_param("production", 0)        # a shard never ends a run by itself
    b = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(R.REWLError):
        x.boundary_bins(1, b)               # before rewl_init
    x.init()
    with pytest.raises(R.REWLError):
        x.boundary_bins(0, b)               # no shard below window 0
    x.boundary_bins(1, b)
    with pytest.raises(ValueError):
        S.split_windows(5, 3)
    full.close(); x.close()
