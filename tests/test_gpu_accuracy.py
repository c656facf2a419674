"""Accuracy against the exact density of states (the run's error, not its parity).

The GPU run is bit-identical to the oracle for a given seed, so these bounds are properties of
the method at these settings: Ising L = 8 (the config-1 lattice, 4 windows at 75 % overlap),
ln f halved to 1e-8 with 128 walkers per window reaches max |d ln g| <= 1e-2 against the exact
g(E) (Kaufman/Beale, tests/golden), and 16 walkers per window to 1e-6 stay within 0.06.
"""
import math
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _exact_L8():
    path = os.path.join(os.path.dirname(__file__), "golden", "ising_L8_counts.txt")
    lng = []
    for line in open(path):
        if line.startswith("#"):
            continue
        c = int(line.split()[1])
        lng.append(math.log(c) if c > 0 else -math.inf)
    ex = np.array(lng)
    fin = np.isfinite(ex)
    mx = ex[fin].max()
    return ex - (mx + math.log(np.exp(ex[fin] - mx).sum()) - 64 * math.log(2)), fin


@pytest.mark.parametrize("m,lnf_final,bound", [(128, 1e-8, 1e-2), (16, 1e-6, 0.06)])
def test_ising_L8_error_against_exact(m, lnf_final, bound):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_2328_gb300 import build as B
    B.build()
    import paper_1402_2328_gb300.rewl as R
    r = R.REWL(0, 8, 4, 0.75, m, lnf_final, 0.8, seed=0x5EED201400000000 + 1000 + 108,
               interval=10_000)
    assert r.run(max_seconds=120) == "done"
    lng, _ = r.stitch(0)
    ex, fin = _exact_L8()
    assert np.array_equal(np.isfinite(lng), fin)
    err = np.abs(lng[fin] - ex[fin])
    assert err.max() <= bound, err.max()
    r.close()
