"""Batched uneven instances: every instance evolves bit for bit as it does alone.

The batch advances many REWL instances (mixed models, lattice sizes, window counts and
walkers per window) with one move-kernel launch per round; its results may not depend on
the batching, the walkers-per-CTA bound or the autotuner's trial rounds.
"""
import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FIELDS = ["spins", "k", "lng", "H", "step", "acc", "flat", "lnf", "iter", "finished", "mask",
          "swap_att", "swap_acc", "pstep", "prep_restarts", "round", "first_iter_round", "mode", "frag"]


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_2328_gb300 import build as B
    B.build()
    import paper_1402_2328_gb300.rewl as R
    return R


def _same(a, b):
    for f in FIELDS:
        x, y = np.asarray(a[f]), np.asarray(b[f])
        if x.dtype.kind == "f":
            assert np.array_equal(x.view(np.uint64), y.view(np.uint64)), f
        else:
            assert np.array_equal(x, y), f


def config4_descs(lnf_final=1e-8):
    """24 instances: (model, L) cycles Ising 16/32/64, Potts q=10 20/40; windows 8..64;
    4..16 walkers per window; one seed each."""
    out = []
    for i in range(24):
        model, L = [(0, 16), (0, 32), (0, 64), (10, 20), (10, 40)][i % 5]
        out.append(dict(model=model, L=L, windows=[8, 16, 32, 64][i % 4],
                        walkers=[4, 8, 16][(i // 4) % 3], lnf_final=lnf_final,
                        seed=0x5EED201400000000 + 4 * 1000 + i, instance=i))
    return out


def _solo(R, d, interval, rounds):
    g = R.REWL(d["model"], d["L"], d["windows"], d.get("overlap", 0.75), d["walkers"],
               d["lnf_final"], d.get("flatness", 0.8), seed=d["seed"], interval=interval,
               instance=d.get("instance", 0))
    g.run(max_rounds=rounds)
    st = g.state()
    g.close()
    return st


@pytest.mark.parametrize("wpb,tsites", [(0, 0), (1, 0), (16, 0), (4, 100), (1, 256)])
def test_small_batch_equals_solo_and_oracle(R, wpb, tsites):
    descs = [dict(model=0, L=8, windows=4, walkers=2, lnf_final=1e-4, seed=11, instance=0),
             dict(model=3, L=6, windows=3, walkers=3, lnf_final=1e-4, seed=12, instance=1),
             dict(model=0, L=16, windows=8, walkers=4, lnf_final=1e-4, seed=13, instance=2),
             dict(model=10, L=12, windows=8, walkers=2, lnf_final=1e-4, seed=14, instance=3),
             dict(model=0, L=5, windows=1, walkers=1, lnf_final=1e-4, seed=15, instance=4)]
    b = R.REWLBatch(descs, interval=700, walkers_per_block=wpb, thread_layout_max_sites=tsites)
    b.init()
    b.run(max_rounds=40)
    for i, d in enumerate(descs):
        got = b.instance(i).state()
        _same(got, _solo(R, d, 700, 40))
        o = O.REWL(d["model"], d["L"], d["windows"], 0.75, d["walkers"], d["lnf_final"], 0.8,
                   seed=d["seed"], instance=d["instance"], interval=700)
        assert o.init() == 0
        o.run(40)
        _same(got, o.state())
    b.close()


def test_batch_to_completion_equals_solo(R):
    descs = [dict(model=0, L=6, windows=3, walkers=2, lnf_final=1e-5, seed=21, instance=0),
             dict(model=2, L=6, windows=2, walkers=2, lnf_final=1e-5, seed=22, instance=1),
             dict(model=3, L=4, windows=2, walkers=1, lnf_final=1e-5, seed=23, instance=2)]
    b = R.REWLBatch(descs, interval=500)
    assert b.run() == "done"
    for i, d in enumerate(descs):
        g = R.REWL(d["model"], d["L"], d["windows"], 0.75, d["walkers"], d["lnf_final"], 0.8,
                   seed=d["seed"], interval=500, instance=d["instance"])
        assert g.run() == "done"
        _same(b.instance(i).state(), g.state())
        a, ja = b.instance(i).stitch(0)
        c, jc = g.stitch(0)
        assert np.array_equal(ja, jc) and np.array_equal(a.view(np.uint64), c.view(np.uint64))
        g.close()
    b.close()


def test_batch_instance_with_caller_windows(R):
    """Windows replaced on a batch instance before init: the instance equals the oracle."""
    descs = [dict(model=0, L=16, windows=5, walkers=2, lnf_final=1e-4, seed=31, instance=0),
             dict(model=10, L=8, windows=4, walkers=2, lnf_final=1e-4, seed=32, instance=1)]
    cost = np.ones(257)
    cost[200:] = 6.0
    lo, hi = R.windows_balanced(cost, 5, 0.75)
    b = R.REWLBatch(descs, interval=600)
    b.instance(0).set_windows(lo, hi)
    b.init()
    b.run(max_rounds=25)
    for i, d in enumerate(descs):
        o = O.REWL(d["model"], d["L"], d["windows"], 0.75, d["walkers"], d["lnf_final"], 0.8,
                   seed=d["seed"], instance=d["instance"], interval=600,
                   lo_hi=(lo, hi) if i == 0 else None)
        assert o.init() == 0
        o.run(25)
        _same(b.instance(i).state(), o.state())
    b.close()


def test_config4_batch_autotuned_equals_solo(R):
    descs = config4_descs()
    b = R.REWLBatch(descs, interval=10_000)
    b.init()
    best, ms = b.autotune(rounds=1)  # trial rounds of the simulation itself
    assert best["walkers_per_block"] in (2, 4, 8, 16) and best["graph_rounds"] in (8, 32, 128)
    assert best["thread_layout_max_sites"] in (0, 400, 1024, 1600)
    assert all(v > 0 for v in ms.values())  # every site limit applies to some instance here
    b.run(max_rounds=1)
    info = b.info()
    assert info["instances"] == 24 and info["walkers"] == 6720
    assert info["thread_layout_max_sites"] == best["thread_layout_max_sites"]
    rounds = int(b.instance(0).get_state("round")[0])
    assert rounds == 16 + 8 + 32 + 128 + 1
    for i in (0, 2, 3, 7, 12, 17, 23):
        _same(b.instance(i).state(), _solo(R, descs[i], 10_000, rounds))
    # the first instances of each model against the oracle, the same rounds (the autotuner's
    # trial rounds are ordinary rounds, whatever layout ran them)
    for i in (0, 3):
        d = descs[i]
        o = O.REWL(d["model"], d["L"], d["windows"], 0.75, d["walkers"], d["lnf_final"], 0.8,
                   seed=d["seed"], instance=d["instance"], interval=10_000)
        assert o.init() == 0
        o.run(rounds)
        _same(b.instance(i).state(), o.state())
    b.close()
