"""Late-stage parity at full size: a state planted deep into a run (|ln g| in the thousands,
ln f near 1e-8, dyadic in halving mode and non-dyadic in 1/t mode, finished windows, 64-bit
step counters, near-flat histograms) advanced two rounds on the GPU and in the oracle.

These are the conditions of every full run's last hours, where the float32 screen of the move
kernel has its smallest margin (Sec. 2 decision rule, exact by construction): every field must
be bit-identical, and with every decision also taken in float64 no screen decision may
disagree with it.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from tests import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FIELDS = ["spins", "k", "lng", "H", "step", "acc", "flat", "lnf", "iter", "finished", "mask",
          "swap_att", "swap_acc", "round", "first_iter_round", "mode", "frag"]
PLANT = ["lng", "H", "step", "flat", "lnf", "iter", "finished", "mask", "mode"]


@pytest.fixture(scope="module", autouse=True)
def cuda_lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_2328_gb300 import build as B
    B.build()


def _golden_ising_lng(L):
    path = os.path.join(os.path.dirname(__file__), "golden", f"ising_L{L}_lng.txt")
    vals = [float(line.split()[1]) for line in open(path) if not line.startswith("#")]
    return np.array(vals)


def _bins(model, L):
    N = L * L
    if model == 0:
        ex = _golden_ising_lng(L)
        return np.where(np.isfinite(ex), ex, 0.0), np.isfinite(ex)
    B = 2 * N
    valid = np.ones(B + 1, bool)
    valid[1:4] = False  # one changed site leaves 4 bonds unsatisfied: k = 1..3 cannot occur
    lng = I.smooth_concave_lng(B, int(1.8 * N), N * math.log(model))
    return np.where(valid, lng, 0.0), valid


# rounds done so far: visited bins / moves (the 1/t value) lands just below 1e-8 for the
# widest windows and above it for narrower ones
@pytest.mark.parametrize("model,L,h,m,cfg,rounds_done", [(0, 64, 32, 16, 2, 4_700_001),
                                                         (10, 80, 64, 16, 5, 7_700_001)])
@pytest.mark.parametrize("check_all", [0, 1])
def test_late_stage_rounds_bit_exact(model, L, h, m, cfg, rounds_done, check_all):
    import paper_1402_2328_gb300.rewl as R
    seed, interval, lnf_final = I.seed_for(cfg, 77), 10_000, 1e-8
    g = R.REWL(model, L, h, 0.75, m, lnf_final, 0.8, seed=seed, interval=interval, schedule=1,
               check_all=check_all)
    o = O.REWL(model, L, h, 0.75, m, lnf_final, 0.8, seed=seed, interval=interval, schedule=1)
    g.init()
    assert o.init() == 0
    lng_bins, valid = _bins(model, L)
    st = I.late_stage_state(np.random.default_rng(cfg), o.lo, o.hi, o.W, m, lng_bins, valid,
                            rounds_done * interval, lnf_final)
    for f in PLANT:
        g.set_state(f, st[f])
    g.set_state("round", [rounds_done])
    o.put(lng=st["lng"], H=st["H"], step=st["step"])
    o.put_window(lnf=st["lnf"], iter=st["iter"], flat=st["flat"], finished=st["finished"],
                 mask=st["mask"], mode=st["mode"], round=rounds_done)
    assert np.max(np.abs(st["lng"])) > 1000
    g.run(max_rounds=2)
    o.run(2)
    gs, os_ = g.state(), o.state()
    for f in FIELDS:
        a, b = np.asarray(gs[f]), np.asarray(os_[f])
        if a.dtype.kind == "f":
            assert np.array_equal(a.view(np.uint64), b.view(np.uint64)), f
        else:
            assert np.array_equal(a, b), (f, np.argwhere(a != b)[:5])
    # the planted windows took every branch: advances in both modes, finishing, frozen windows
    assert gs["iter"].sum() > st["iter"].sum() and gs["finished"].sum() > st["finished"].sum()
    assert gs["acc"].sum() > 0
    if check_all:
        assert int(g.get_state("n_mismatch")[0]) == 0
    g.close()
