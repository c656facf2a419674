"""Window layouts from a pre-run (Fig. 1b): sequencing of library calls only.

`late_balanced_windows` runs a pre-run on the target lattice with its current layout, notes the
round at which every window completes each WL iteration (polling the iteration counters between
chunks of rounds), and hands the rounds per iteration between two later iterations to
rewl_windows_late_balanced, which computes the layout.
"""
from __future__ import annotations

import time

import numpy as np

from . import rewl as R


def late_balanced_windows(pre: R.REWL, h_new: int, it_from: int = 3, it_to: int = 6,
                          overlap: float = 0.75, chunk: int = 256, max_seconds: float = 600.0):
    """(lo, hi, info): run `pre` (initialised or not) until every window completed iteration
    `it_to` or max_seconds, then the layout balanced by the later iterations' cost."""
    if not 1 <= it_from < it_to:
        raise ValueError("need 1 <= it_from < it_to")
    reached = np.full((pre.h, it_to + 1), -1, np.int64)
    t0 = time.perf_counter()
    pre.run(max_rounds=0)  # initialises if needed
    while time.perf_counter() - t0 < max_seconds:
        pre.run(max_rounds=chunk)
        it = pre.get_state("iter")
        rd = int(pre.get_state("round")[0])
        for w in range(pre.h):
            for i in range(1, min(int(it[w]), it_to) + 1):
                if reached[w, i] < 0:
                    reached[w, i] = rd
        if np.all(it >= it_to):
            break
    ok = (reached[:, it_from] >= 0) & (reached[:, it_to] >= 0)
    per = np.where(ok, (reached[:, it_to] - reached[:, it_from]) / float(it_to - it_from), -1.0)
    lo, hi = pre.get_state("lo"), pre.get_state("hi")
    nlo, nhi = R.windows_late_balanced(lo, hi, per, pre.B, h_new, overlap)
    info = dict(seconds=time.perf_counter() - t0, rounds=int(pre.get_state("round")[0]),
                rounds_per_iter=per.tolist(), complete=bool(ok.all()))
    return nlo, nhi, info
