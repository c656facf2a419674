"""The learned warm start end to end at small scale: plain REWL on Ising L = 8..16 trains the
MLP on the GPU; the predicted ln g of L = 24 seeds a run from ln f = 1e-3.  What the network
gains: from the same small starting ln f, the method without it (flat ln g) needs far more
rounds than with the prediction.  The cold start (ln f = 1) is run for context: WL's late
iterations dominate, so the warm start does not beat it here (recorded, not asserted)."""
import math

import numpy as np
import pytest

from oracle import exact_dos as X

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_warm_start_gains_over_cold_start():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_2328_gb300 import build as B
    B.build()
    import paper_1402_2328_gb300.rewl as R
    from paper_1402_2328_gb300 import warm as WM

    descs = [dict(model=0, L=L, windows=2, walkers=2, lnf_final=1e-5, seed=70 + L, instance=L)
             for L in (8, 10, 12, 14, 16)]
    b = R.REWLBatch(descs, interval=2000)
    assert b.run(max_seconds=300) == "done"
    runs = [(0, d["L"], b.instance(i).stitch(0)[0]) for i, d in enumerate(descs)]
    b.close()
    Xd, Td = WM.training_set(runs)
    P, hist = WM.train(Xd, Td, steps=3000, lr=3e-3, seed=1)
    assert hist[-1][1] < 0.01 * hist[0][1] + 1e-4
    pred = WM.predict_lng(P, 0, 24)
    ex = X.normalise_lng(np.array(X.exact_lng(0, 24)), 576 * math.log(2))
    fin = np.isfinite(ex)

    def run(kind, max_rounds=-1):
        if kind == "warm":
            r = WM.warm_handle(0, 24, 4, 4, 1e-5, 99, pred, lnf_init=1e-3, interval=2000)
        elif kind == "flat":
            r = WM.warm_handle(0, 24, 4, 4, 1e-5, 99, np.zeros(577), lnf_init=1e-3, interval=2000)
        else:
            r = R.REWL(0, 24, 4, 0.75, 4, 1e-5, 0.8, seed=99, interval=2000)
        status = r.run(max_seconds=300, max_rounds=max_rounds)
        out = r.stitch(0)[0] if status == "done" else None
        rounds = r.stats()["rounds"]
        r.close()
        err = None if out is None else float(np.max(np.abs(out[fin] - ex[fin])))
        return status, rounds, err

    sw, rw, ew = run("warm")
    assert sw == "done" and ew < 1.0
    sf, rf, _ = run("flat", max_rounds=3 * rw)
    sc, rc, ec = run("cold")
    print(f"warm: {rw} rounds err {ew:.3f}; flat ln g from the same ln f: {sf} after {rf} "
          f"rounds; cold start: {rc} rounds err {ec:.3f}")
    assert sf == "budget" or rf > 2 * rw
