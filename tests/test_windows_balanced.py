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


def test_late_balanced_layout_properties():
    """Windows balanced by later-iteration cost (host call): a valid layout; equal cost keeps
    equal-size windows; a window that takes 16x longer per iteration becomes ~4x narrower."""
    import numpy as np
    import paper_1402_2328_gb300.rewl as R
    B, h = 4096, 16
    lo, hi = R.windows_layout(B, h, 0.75)
    for per in (np.full(h, 1000.0), np.r_[16000.0, np.full(h - 1, 1000.0)],
                np.r_[np.full(h - 1, 1000.0), -1.0]):
        nlo, nhi = R.windows_late_balanced(lo, hi, per, B, h, 0.75)
        assert nlo[0] == 0 and nhi[-1] == B
        assert np.all(np.diff(nlo) > 0) and np.all(np.diff(nhi) > 0)
        assert np.all(nlo[1:] <= nhi[:-1])           # neighbours overlap
    w_eq = (hi - lo + 1).astype(float)
    nlo, nhi = R.windows_late_balanced(lo, hi, np.full(h, 1000.0), B, h, 0.75)
    assert np.max(np.abs((nhi - nlo + 1) - w_eq)) <= 2
    nlo, nhi = R.windows_late_balanced(lo, hi, np.r_[16000.0, np.full(h - 1, 1000.0)], B, h, 0.75)
    ratio = (nhi[0] - nlo[0] + 1) / w_eq[0]
    assert 0.15 < ratio < 0.45, ratio
    with pytest.raises(R.REWLError):
        R.windows_late_balanced(lo, hi, np.full(h, -1.0), B, h, 0.75)


class _FakePre:
    """A pre-run whose window w completes an iteration every (w + 1) * 10 rounds."""
    h, B = 4, 64

    def __init__(self):
        self.rd = 0
        import numpy as np
        import paper_1402_2328_gb300.rewl as R
        self.lo, self.hi = R.windows_layout(self.B, self.h, 0.75)
        self.np = np

    def run(self, max_rounds=-1, **kw):
        self.rd += max(0, max_rounds)
        return "budget"

    def get_state(self, f):
        np = self.np
        if f == "iter":
            return np.array([self.rd // (10 * (w + 1)) for w in range(self.h)], np.int32)
        if f == "round":
            return np.array([self.rd], np.int64)
        return {"lo": self.lo, "hi": self.hi}[f]


def test_late_balance_helper_reads_iteration_times():
    """balance.late_balanced_windows: iteration completion rounds polled between chunks give
    the rounds per iteration of each window; the slowest window comes out narrowest."""
    from paper_1402_2328_gb300 import balance as BL
    pre = _FakePre()
    lo, hi, info = BL.late_balanced_windows(pre, 4, it_from=2, it_to=4, chunk=5, max_seconds=30)
    assert info["complete"]
    assert info["rounds_per_iter"] == [10.0, 20.0, 30.0, 40.0]
    widths = hi - lo + 1
    assert widths[3] < widths[0] and lo[0] == 0 and hi[-1] == 64
    with pytest.raises(ValueError):
        BL.late_balanced_windows(pre, 4, it_from=3, it_to=3)
