"""Refusals at the boundary for settings the move kernel's int64 ln g shadow cannot hold, and
checkpoints of 1/t, production and (E, M) runs.

The shadow keeps ln g as a multiple of 2^-32 in an int64: a launch of T moves is refused when
max|ln g| + T ln f could reach 2^30 or ln f < 2^-32, and a refused case keeps its state.
"""
import numpy as np
import pytest

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


def test_parameter_refusals(R):
    with pytest.raises(R.REWLError):
        R.REWL(0, 8, 2, 0.75, 1, 2.0 ** -33, 0.8)
    g = R.REWL(0, 8, 2, 0.75, 1, 1e-6, 0.8)
    for key, v in (("lnf_init", 2.0 ** 20), ("lnf_init", 2.0 ** -33), ("lnf_init", -1.0)):
        with pytest.raises(R.REWLError):
            g.set_param(key, v)
    g.set_param("lnf_init", 2.0 ** 13)
    g.set_param("interval", 100_000)          # 2^13 * 1e5 = 8.2e8 < 2^30
    with pytest.raises(R.REWLError):
        g.set_param("interval", 200_000)      # 1.6e9 >= 2^30
    with pytest.raises(R.REWLError):
        g.set_param("lnf_init", 2.0 ** 14)    # with interval 1e5
    g.set_param("lnf_init", 1.0)
    g.init()
    for f, v in (("lnf", [-1.0, 1.0]), ("lnf", [np.inf, 1.0]), ("mode", [2, 0]),
                 ("finished", [0, 3]), ("iter", [-1, 0])):
        with pytest.raises(R.REWLError):
            g.set_state(f, v)
    g.close()


def _case(n, T, lnf, frozen, lng0=10.0):
    rng = np.random.default_rng(5)
    L, W = 8, 16
    spins = np.ones((n, L * L), np.int8)        # ground state: bin 0
    k = np.zeros(n, np.int32)
    lo = np.zeros(n, np.int32)
    hi = np.full(n, W - 1, np.int32)
    lng = np.full((n, W), lng0)
    H = np.zeros((n, W), np.uint32)
    words = rng.integers(0, 2 ** 32, (n, T, 3), dtype=np.uint64).astype(np.uint32)
    return dict(spins=spins, k=k, lo=lo, hi=hi, lng=lng, H=H,
                lnf=np.full(n, lnf), frozen=np.full(n, frozen, np.uint8), words=words)


def _call(fn, c):
    d = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).view(dt)).cuda()  # noqa: E731
    n, T = c["words"].shape[:2]
    st = dict(spins=d(c["spins"], np.int8), k=d(c["k"], np.int32), lng=d(c["lng"], np.float64),
              H=d(c["H"], np.int32))
    acc = torch.zeros((n, T), dtype=torch.int32, device="cuda")
    dk = torch.zeros((n, T), dtype=torch.int32, device="cuda")
    fn(0, 8, st["spins"], st["k"], d(c["lo"], np.int32), d(c["hi"], np.int32), st["lng"],
       st["H"], d(c["lnf"], np.float64), d(c["frozen"], np.uint8), d(c["words"], np.int32),
       acc, dk)
    torch.cuda.synchronize()
    return {key: v.cpu().numpy() for key, v in st.items()}


@pytest.mark.parametrize("which", ["replay", "replay_static"])
def test_replay_refuses_shadow_overflow_and_keeps_state(R, which):
    fn = getattr(R, which)
    T = 10_000
    c = _case(4, T, 2.0 ** 19, 0)            # ln f in range, T ln f = 5.2e9 >= 2^30
    with pytest.raises(R.REWLError):
        _call(fn, c)
    c = _case(4, T, 2.0 ** 19, 0)
    d = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).view(dt)).cuda()  # noqa: E731
    lng_d, H_d = d(c["lng"], np.float64), d(c["H"], np.int32)
    sp_d, k_d = d(c["spins"], np.int8), d(c["k"], np.int32)
    acc = torch.zeros((4, T), dtype=torch.int32, device="cuda")
    with pytest.raises(R.REWLError):
        fn(0, 8, sp_d, k_d, d(c["lo"], np.int32), d(c["hi"], np.int32), lng_d, H_d,
           d(c["lnf"], np.float64), d(c["frozen"], np.uint8), d(c["words"], np.int32), acc,
           torch.zeros_like(acc))
    torch.cuda.synchronize()
    assert np.array_equal(lng_d.cpu().numpy(), c["lng"]) and not H_d.cpu().numpy().any()
    assert np.array_equal(sp_d.cpu().numpy(), c["spins"]) and not k_d.cpu().numpy().any()
    # the same ln f in a frozen window adds nothing to the shadow: accepted
    out = _call(fn, _case(4, T, 2.0 ** 19, 1))
    assert np.array_equal(out["lng"], np.full((4, 16), 10.0))
    # just inside the bound: 2^16 * 10^4 + 10 < 2^30
    out = _call(fn, _case(4, T, 2.0 ** 16, 0))
    assert out["H"].sum() == 4 * T


def test_checkpoint_of_one_over_t_run(R, tmp_path):
    args = (0, 6, 3, 0.75, 2, 1e-5, 0.8)
    a = R.REWL(*args, seed=21, interval=400, schedule=1)
    a.init()
    for _ in range(4000):                     # until some window is in 1/t mode
        a.run(max_rounds=5)
        if a.get_state("mode").any():
            break
    assert a.get_state("mode").any() and not a.get_state("mode").all()
    p = str(tmp_path / "t.ck")
    a.checkpoint(p)
    a.run(max_rounds=300)
    b = R.REWL(*args, seed=21, interval=400, schedule=1)
    b.restore(p)
    b.run(max_rounds=300)
    sa, sb = a.state(), b.state()
    for f in sa:
        assert np.array_equal(np.asarray(sa[f]), np.asarray(sb[f])), f
    c = R.REWL(*args, seed=21, interval=400)  # halving schedule: refused
    with pytest.raises(R.REWLError):
        c.restore(p)
    a.close(); b.close(); c.close()


def test_checkpoint_of_production_run_with_em(R, tmp_path):
    args = (0, 4, 2, 0.75, 2, 1e-2, 0.8)
    a = R.REWL(*args, seed=23, interval=300)
    assert a.run() == "done"
    a.set_param("production", 1)
    a.set_param("measure_em", 1)
    a.run(max_rounds=20)
    p = str(tmp_path / "p.ck")
    a.checkpoint(p)
    a.run(max_rounds=20)
    b = R.REWL(*args, seed=23, interval=300)
    b.restore(p)
    assert b.run(max_rounds=20) == "budget"   # production: the run goes on after "done"
    sa, sb = a.state(), b.state()
    for f in sa:
        assert np.array_equal(np.asarray(sa[f]), np.asarray(sb[f])), f
    assert np.array_equal(a.hist_em(), b.hist_em()) and a.hist_em().sum() == 40 * 4
    a.close(); b.close()
