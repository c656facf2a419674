"""Run-time balanced windows (Fig. 1b): host logic of the library, no GPU needed."""
import numpy as np
import pytest

import oracle as O


@pytest.fixture(scope="module")
def R():
    from paper_1402_2328_gb300 import build as B
    B.build()
    import paper_1402_2328_gb300.rewl as R
    return R


@pytest.mark.parametrize("B,h", [(64, 4), (4096, 32), (3200, 64), (500, 7)])
def test_uniform_cost_gives_equal_windows(R, B, h):
    lo, hi = R.windows_balanced(np.ones(B + 1), h, 0.75)
    elo, ehi = O.windows(B, h, 0.75)
    assert np.all(np.abs(lo - elo) <= 1) and np.all(np.abs(hi - ehi) <= 1)


def test_windows_follow_the_cost(R):
    B, h = 1000, 8
    cost = np.ones(B + 1)
    cost[:200] = 20.0  # expensive low-energy region
    lo, hi = R.windows_balanced(cost, h, 0.75)
    assert lo[0] == 0 and hi[-1] == B
    width = hi - lo
    assert width[0] < width[-1] / 3  # narrow where the work is
    share = [cost[a:b + 1].sum() for a, b in zip(lo, hi)]
    inner = np.array(share[1:-1])
    assert inner.max() / inner.min() < 1.6  # roughly equal work per window
    assert np.all(lo[1:] <= hi[:-1]) and np.all(np.diff(lo) > 0)  # overlapping, ordered


def test_rejects_bad_cost(R):
    with pytest.raises(R.REWLError):
        R.windows_balanced(np.array([1.0, -1.0, 1.0]), 1)
