"""rewl_replay_static -- the replay entry point that allocates nothing -- against rewl_replay.

Some callers cannot call cudaMalloc (they draw every device buffer from their own pool, or
must not let a cudaFree stall the GPU).  For them rewl_replay_static keeps the move kernel's
per-case scratch in a fixed device array of the library.  Its outputs must equal those of
rewl_replay exactly, on consecutive calls (the array is shared and keeps the previous call's
contents), and it must refuse more cases than the array holds.  This file is collected last
and also passes when run on its own in a fresh process.
"""
import numpy as np
import pytest

import oracle as O
from tests import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_2328_gb300 import build as B
    B.build()
    import paper_1402_2328_gb300.rewl as R
    return R


def _case(model, L, n, T, W, seed):
    rng = np.random.default_rng(seed)
    N = L * L
    B = O.num_bins(model, L)
    spins = I.random_lattices(rng, model, L, n)
    k = np.array([(O.energy(model, L, s) + 2 * N) // (4 if model == 0 else 1) for s in spins],
                 np.int32)
    width = rng.integers(1, W, n)
    lo = np.clip(k - rng.integers(0, width + 1), 0, B).astype(np.int32)
    hi = np.minimum(B, lo + width).astype(np.int32)
    lng = I.random_lng(rng, n, W, scale=0.4) + 50.0
    H = I.random_H(rng, n, W)
    lnf = np.where(rng.random(n) < 0.5, 2.0 ** -rng.integers(0, 27, n), rng.uniform(1e-6, 0.3, n))
    frozen = (rng.random(n) < 0.1).astype(np.uint8)
    words = rng.integers(0, 2 ** 32, (n, T, 3), dtype=np.uint64).astype(np.uint32)
    return dict(spins=spins, k=k, lo=lo, hi=hi, lng=lng, H=H, lnf=lnf, frozen=frozen, words=words)


def _run(fn, model, L, c):
    d = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).view(dt)).cuda()  # noqa: E731
    n, T = c["words"].shape[:2]
    st = dict(spins=d(c["spins"], np.int8), k=d(c["k"], np.int32), lng=d(c["lng"], np.float64),
              H=d(c["H"], np.int32))
    acc = torch.full((n, T), -1, dtype=torch.int32, device="cuda")
    dk = torch.full((n, T), -99, dtype=torch.int32, device="cuda")
    fn(model, L, st["spins"], st["k"], d(c["lo"], np.int32), d(c["hi"], np.int32), st["lng"],
       st["H"], d(c["lnf"], np.float64), d(c["frozen"], np.uint8), d(c["words"], np.int32),
       acc, dk)
    torch.cuda.synchronize()
    out = {key: v.cpu().numpy() for key, v in st.items()}
    out["acc"], out["dk"] = acc.cpu().numpy(), dk.cpu().numpy()
    return out


def test_static_replay_equals_allocating_replay_twice(R):
    cases = [(0, 16, 500, 100, 48, 101), (10, 12, 300, 70, 64, 202)]
    for model, L, n, T, W, seed in cases:  # two calls in a row on the shared array
        c = _case(model, L, n, T, W, seed)
        a = _run(R.replay, model, L, c)
        b = _run(R.replay_static, model, L, c)
        for key in ("acc", "dk", "spins", "k", "H"):
            assert np.array_equal(a[key], b[key]), key
        assert np.array_equal(a["lng"].view(np.uint64), b["lng"].view(np.uint64))
        assert np.all(b["acc"] >= 0)  # every step of every case was written


def test_static_replay_refuses_more_cases_than_it_holds(R):
    c = _case(0, 4, 1, 1, 8, 3)
    n = R.REPLAY_STATIC_MAX_N + 1
    big = {key: np.repeat(v[:1], n, axis=0) for key, v in c.items()}
    with pytest.raises(R.REWLError, match="REWL_REPLAY_STATIC_MAX_N"):
        _run(R.replay_static, 0, 4, big)
