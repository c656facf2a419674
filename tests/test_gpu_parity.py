"""CUDA path versus the CPU oracle, element by element, through the C ABI.

Integer state (lattices, bins, histograms, counters, flags) and the float64 ln g must be
bit-identical: the move kernel's decisions are exact by construction (float64 fallback
inside the screening band), so any difference is a bug.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import exact_dos as X
from tests import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FIELDS = ["spins", "k", "lng", "H", "step", "acc", "flat", "lnf", "iter", "finished", "mask",
          "swap_att", "swap_acc", "pstep", "prep_restarts", "round", "first_iter_round", "mode", "frag"]


@pytest.fixture(scope="module", autouse=True)
def cuda_lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_2328_gb300 import build as B
    B.build()
    import paper_1402_2328_gb300.rewl as R
    return R


def _pair(model, L, h, m, lnf_final=1e-6, flat=0.8, seed=1, interval=1000, **kw):
    import paper_1402_2328_gb300.rewl as R
    g = R.REWL(model, L, h, 0.75, m, lnf_final, flat, seed=seed, interval=interval, **kw)
    o = O.REWL(model, L, h, 0.75, m, lnf_final, flat, seed=seed, interval=interval,
               lnf_init=kw.get("lnf_init", 1.0), schedule=kw.get("schedule", 0))
    return g, o


def _same(gs, os_, fields=FIELDS):
    for f in fields:
        a, b = np.asarray(gs[f]), np.asarray(os_[f])
        assert a.shape == b.shape, (f, a.shape, b.shape)
        if a.dtype.kind == "f":
            assert np.array_equal(a.view(np.uint64), b.view(np.uint64)), f
        else:
            assert np.array_equal(a, b), (f, np.argwhere(a != b)[:5])


# ------------------------------------------------------------------ arithmetic
def test_philox_device_equals_oracle(cuda_lib):
    rng = np.random.default_rng(0)
    n = 4096
    ctr = rng.integers(0, 2 ** 32, (n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, (n, 2), dtype=np.uint64).astype(np.uint32)
    ctr[:3] = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344]]
    key[:3] = [[0, 0], [0xFFFFFFFF] * 2, [0xA4093822, 0x299F31D0]]
    c_d, k_d = torch.from_numpy(ctr.view(np.int32)).cuda(), torch.from_numpy(key.view(np.int32)).cuda()
    out = torch.zeros((n, 4), dtype=torch.int32, device="cuda")
    cuda_lib.philox(c_d, k_d, out)
    got = out.cpu().numpy().view(np.uint32)
    for i in range(n):
        assert np.array_equal(got[i], O.philox(ctr[i], key[i])), i


def test_lnu_device_bit_equals_oracle(cuda_lib):
    rng = np.random.default_rng(1)
    w = np.concatenate([rng.integers(0, 2 ** 32, 200000, dtype=np.uint64),
                        np.arange(0, 1000), 2 ** 32 - 1 - np.arange(0, 1000),
                        (2 ** np.arange(32)).astype(np.uint64)]).astype(np.uint32)
    wd = torch.from_numpy(w.view(np.int32)).cuda()
    out = torch.zeros(len(w), dtype=torch.float64, device="cuda")
    cuda_lib.lnu(wd, out)
    got = out.cpu().numpy()
    lib = O.lib()
    want = np.array([lib.or_lnu(int(x)) for x in w])
    assert np.array_equal(got.view(np.uint64), want.view(np.uint64))


def test_lnu_screen_bound_all_words(cuda_lib):
    """max over all 2^32 words of |float32 screen - float64 ln u| stays below the
    tolerance the move kernel assumes, and ln u < 0 for every word."""
    mx = torch.zeros(1, dtype=torch.float64, device="cuda")
    bad = torch.zeros(1, dtype=torch.int64, device="cuda")
    cuda_lib.lnu_bound(0, 2 ** 32, mx, bad)
    torch.cuda.synchronize()
    assert int(bad.item()) == 0
    assert 0.0 < mx.item() < cuda_lib.lnu_eps(), (mx.item(), cuda_lib.lnu_eps())


def test_seqadd_equals_sequential_float64_loop(cuda_lib):
    """x + f + ... + f (c additions) as the kernels rebuild ln g: dyadic and non-dyadic f (the 1/t
    schedule), negative x (warm starts), x at binade edges, and ties (f = (a + 1/2) ulp(x))."""
    rng = np.random.default_rng(2)
    n = 3000
    k = n // 5
    x = np.concatenate([rng.uniform(0, 5000, k), rng.uniform(-50, 50, k),
                        2.0 ** rng.integers(-5, 12, k) - rng.uniform(0, 1e-3, k),
                        (2.0 ** rng.integers(-8, 14, k)) * rng.choice([-1.0, 1.0], k),
                        rng.uniform(-3e4, 3e4, n - 4 * k)])
    f = np.where(rng.random(n) < 0.4, 2.0 ** -rng.integers(0, 27, n),
                 np.where(rng.random(n) < 0.5, rng.uniform(1e-9, 1e-2, n),
                          rng.integers(1, 10 ** 4, n) / rng.integers(10 ** 6, 10 ** 11, n)))
    ties = rng.random(n) < 0.1
    ulp = np.spacing(np.abs(x))
    f = np.where(ties & (x != 0), (rng.integers(0, 300, n) + 0.5) * ulp, f)
    c = rng.integers(0, 20000, n).astype(np.uint32)
    x[:4] = [0.0, -0.0, 2047.9999999999998, -1e-12]
    want = x.copy()  # the additions one at a time, all cases in step
    for step in range(int(c.max())):
        live = step < c
        want[live] = want[live] + f[live]
    xd, fd = torch.from_numpy(x).cuda(), torch.from_numpy(f).cuda()
    cd = torch.from_numpy(c.view(np.int32)).cuda()
    out = torch.zeros(n, dtype=torch.float64, device="cuda")
    cuda_lib.seqadd(xd, fd, cd, out)
    got = out.cpu().numpy()
    assert np.array_equal(got.view(np.uint64), want.view(np.uint64)), np.flatnonzero(got != want)[:10]


# ------------------------------------------------------------------ replay (one kernel, given words)
def _replay_inputs(model, L, n, T, W, seed, scale):
    rng = np.random.default_rng(seed)
    N = L * L
    B = O.num_bins(model, L)
    spins = I.random_lattices(rng, model, L, n)
    if n > 4:
        spins[: n // 8] = 1 if model == 0 else 0  # some ordered lattices (low-energy edge)
    k = np.array([(O.energy(model, L, s) + 2 * N) // (4 if model == 0 else 1) for s in spins], np.int32)
    width = rng.integers(1, W, n)
    lo = np.clip(k - rng.integers(0, width + 1), 0, B).astype(np.int32)  # lo <= k
    hi = np.minimum(B, lo + width).astype(np.int32)  # k <= hi, hi - lo + 1 <= W
    lng = I.random_lng(rng, n, W, scale=scale)
    lng += rng.choice([-50.0, 0.0, 100.0, 3000.0], size=(n, 1))
    if scale >= 5.0:  # steep rows with spikes: many cached bins beyond the float32 cap
        lng += np.where(rng.random((n, W)) < 0.1, 500.0, 0.0)
    H = I.random_H(rng, n, W)
    lnf = np.where(rng.random(n) < 0.6, 2.0 ** -rng.integers(0, 27, n), rng.uniform(1e-6, 0.5, n))
    frozen = (rng.random(n) < 0.1).astype(np.uint8)
    words = rng.integers(0, 2 ** 32, (n, T, 3), dtype=np.uint64).astype(np.uint32)
    return spins, k, lo, hi, lng, H, lnf, frozen, words


@pytest.mark.parametrize("model,L,n,T,W,scale", [
    (0, 4, 300, 1, 12, 0.8), (0, 8, 300, 64, 40, 0.5), (0, 7, 200, 45, 40, 0.5),
    (0, 64, 128, 200, 64, 0.3), (3, 5, 300, 33, 40, 0.5), (10, 12, 200, 100, 80, 0.4),
    (2, 6, 100, 70, 60, 0.5), (10, 40, 64, 300, 64, 0.2), (0, 16, 200, 150, 60, 6.0),
    (10, 12, 200, 150, 80, 8.0)])
def test_replay_bit_exact(cuda_lib, model, L, n, T, W, scale):
    spins, k, lo, hi, lng, H, lnf, frozen, words = _replay_inputs(model, L, n, T, W, 7 + L + model, scale)
    q = 2 if model == 0 else model
    # oracle: T single attempts in sequence
    st = dict(spins=spins.copy(), k=k.copy(), lng=lng.copy(), H=H.copy())
    acc_o = np.zeros((n, T), np.int32)
    dk_o = np.zeros((n, T), np.int32)
    for t in range(T):
        r = O.replay_batch(model, q, L, st["spins"], st["k"], lo, hi, st["lng"], st["H"], lnf,
                           frozen, words[:, t, :])
        st = dict(spins=r["spins"], k=r["k"], lng=r["lng"], H=r["H"])
        acc_o[:, t], dk_o[:, t] = r["acc"], r["dk"]
    d = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).view(dt)).cuda()  # noqa: E731
    sp_d, k_d = d(spins, np.int8), d(k, np.int32)
    lng_d, H_d = d(lng, np.float64), d(H, np.int32)
    acc_d = torch.zeros((n, T), dtype=torch.int32, device="cuda")
    dk_d = torch.zeros((n, T), dtype=torch.int32, device="cuda")
    cuda_lib.replay(model, L, sp_d, k_d, d(lo, np.int32), d(hi, np.int32), lng_d, H_d,
                    d(lnf, np.float64), d(frozen, np.uint8), d(words, np.int32), acc_d, dk_d)
    torch.cuda.synchronize()
    assert np.array_equal(acc_d.cpu().numpy(), acc_o)
    assert np.array_equal(dk_d.cpu().numpy(), dk_o)
    assert np.array_equal(sp_d.cpu().numpy(), st["spins"])
    assert np.array_equal(k_d.cpu().numpy(), st["k"])
    assert np.array_equal(H_d.cpu().numpy().view(np.uint32), st["H"])
    assert np.array_equal(lng_d.cpu().numpy().view(np.uint64), st["lng"].view(np.uint64))


# ------------------------------------------------------------------ whole runs
@pytest.mark.parametrize("check", [0, 1])
@pytest.mark.parametrize("model,L,h,m,rounds,interval", [
    (0, 8, 4, 2, 60, 1000), (3, 6, 3, 3, 60, 700), (0, 16, 8, 4, 25, 2000),
    (10, 12, 8, 2, 25, 1500), (0, 5, 2, 3, 80, 333), (0, 8, 1, 1, 50, 1000)])
def test_rounds_bit_exact(model, L, h, m, rounds, interval, check):
    g, o = _pair(model, L, h, m, seed=11 + L, interval=interval, check_all=check)
    g.init()
    assert o.init() == 0
    _same(g.state(), o.state())
    for chunk in (1, 7, rounds - 8):
        g.run(max_rounds=chunk)
        o.run(chunk)
        _same(g.state(), o.state())
    assert int(g.get_state("n_mismatch")[0]) == 0
    g.close()


def test_config1_to_completion_bit_exact_and_accuracy():
    seed = I.seed_for(1)
    g, o = _pair(0, 8, 4, 1, lnf_final=1e-6, seed=seed, interval=10_000)
    assert g.run() == "done"
    o.init()
    o.run(10 ** 7)
    _same(g.state(), o.state())
    out_g, joins_g = g.stitch(0)
    out_o, joins_o = o.stitch(0)
    assert np.array_equal(joins_g, joins_o)
    fin = np.isfinite(out_o)
    assert np.array_equal(np.isfinite(out_g), fin)
    assert np.max(np.abs(out_g[fin] - out_o[fin])) < 1e-12
    ex = X.normalise_lng(np.array(X.exact_lng(0, 8)), 64 * math.log(2))
    err = np.max(np.abs(out_g[fin] - ex[fin]))
    print(f"config 1: max |d ln g| vs exact = {err:.4f} (one walker per window)")
    assert err < 0.5
    g.close()


def test_potts_q3_3x3_against_enumeration():
    """The small Potts check of the q = 10 workload: q = 3 on 3x3 (3^9 states enumerated),
    two windows x four walkers, ln f to 1e-6, three seeds; each run equals the oracle's."""
    ex = X.normalise_lng(np.array(X.exact_lng(3, 3, 3)), 9 * math.log(3))
    fin = np.isfinite(ex)
    errs = []
    for seed in range(3):
        g, o = _pair(3, 3, 2, 4, lnf_final=1e-6, seed=900 + seed, interval=500)
        assert g.run() == "done"
        o.init()
        o.run(10 ** 7)
        _same(g.state(), o.state())
        out, _ = g.stitch(0)
        assert np.array_equal(np.isfinite(out), fin)
        errs.append(np.max(np.abs(out[fin] - ex[fin])))
        g.close()
    print(f"Potts q=3 3x3: max |d ln g| vs enumeration per seed = {np.round(errs, 4)}")
    assert max(errs) < 0.25


@pytest.mark.parametrize("model,L,h,m,rounds,cfg", [(0, 64, 32, 16, 2, 2), (10, 40, 64, 16, 2, 3),
                                                   (10, 80, 64, 16, 2, 5)])
def test_full_size_rounds_bit_exact(model, L, h, m, rounds, cfg):
    """The workloads of the benchmark (Ising L = 64, Potts q = 10 L = 40 and L = 80), in the
    benchmark's launch configuration."""
    g, o = _pair(model, L, h, m, lnf_final=1e-8, seed=I.seed_for(cfg), interval=10_000)
    g.init()
    assert o.init() == 0
    g.run(max_rounds=rounds)
    o.run(rounds)
    _same(g.state(), o.state())
    g.close()


@pytest.mark.parametrize("model,L,h,m,interval", [(0, 6, 2, 2, 400), (3, 5, 2, 2, 300)])
def test_one_over_t_schedule_to_completion_bit_exact(model, L, h, m, interval):
    """The 1/t schedule: ln f = visited bins / moves after the switch, averaged every check."""
    g, o = _pair(model, L, h, m, lnf_final=1e-5, seed=31 + L, interval=interval, schedule=1)
    assert g.run() == "done"
    o.init()
    o.run(10 ** 7)
    st = g.state()
    _same(st, o.state())
    assert np.all(st["mode"] == 1) and np.all(st["first_iter_round"] > 0)
    g.close()


def test_jackknife_gpu_equals_oracle():
    g, o = _pair(0, 6, 3, 4, lnf_final=1e-5, seed=41, interval=500)
    assert g.run() == "done"
    o.init()
    o.run(10 ** 7)
    _same(g.state(), o.state(), FIELDS + ["frag"])
    eg, eo = g.jackknife(0), o.jackknife(0)
    fin = np.isfinite(eo)
    assert np.array_equal(np.isfinite(eg), fin) and fin.sum() > 10
    assert np.max(np.abs(eg[fin] - eo[fin])) < 1e-9
    assert np.all(eg[fin] >= 0) and np.max(eg[fin]) < 1.0
    g.close()


def test_balanced_windows_pipeline():
    """Pre-run with equal windows until every first iteration ended, then balanced windows."""
    import paper_1402_2328_gb300.rewl as R
    pre = R.REWL(0, 16, 8, 0.75, 2, 1e-3, 0.8, seed=5, interval=2000)
    pre.init()
    for _ in range(200):
        pre.run(max_rounds=5)
        if np.all(pre.get_state("first_iter_round") > 0):
            break
    t1 = pre.get_state("first_iter_round")
    assert np.all(t1 > 0)
    lo, hi = pre.balanced_windows(8, 0.75)
    assert lo[0] == 0 and hi[-1] == 256 and np.all(lo[1:] <= hi[:-1])
    # carried to a lattice by energy per site: the same lattice gives the same layout, a
    # larger one a valid layout of its own bins that a run accepts
    lo2, hi2 = pre.balanced_windows_for(16, 8, 0.75)
    assert np.array_equal(lo2, lo) and np.array_equal(hi2, hi)
    lo3, hi3 = pre.balanced_windows_for(32, 8, 0.75)
    assert lo3[0] == 0 and hi3[-1] == 1024 and np.all(np.diff(lo3) > 0)
    assert np.all(lo3[1:] <= hi3[:-1]) and np.all(np.diff(hi3) > 0)
    big = R.REWL(0, 32, 8, 0.75, 1, 1e-3, 0.8, seed=7, interval=500)
    big.set_windows(lo3, hi3)
    big.init()
    assert big.run(max_rounds=2) == "budget"
    big.close()
    r = R.REWL(0, 16, 8, 0.75, 2, 1e-4, 0.8, seed=6, interval=2000)
    r.set_windows(lo, hi)
    assert r.run() == "done"
    out, joins = r.stitch(0)
    ex = X.normalise_lng(np.array(X.exact_lng(0, 16)), 256 * math.log(2))
    fin = np.isfinite(ex)
    assert np.array_equal(np.isfinite(out), fin)
    assert np.max(np.abs(out[fin] - ex[fin])) < 1.0
    pre.close()
    r.close()


def test_caller_windows_bit_exact():
    """Uneven caller windows (balanced layouts): GPU rounds equal the oracle's bit for bit."""
    import paper_1402_2328_gb300.rewl as R
    cost = np.ones(257)
    cost[:60] = 8.0
    top = (np.array([0, 200, 240, 250]), np.array([210, 245, 252, 256]))  # prep restarts
    for model, L, h, m, lohi in [(0, 16, 6, 2, R.windows_balanced(cost, 6, 0.75)),
                                 (3, 8, 4, 3, R.windows_balanced(np.linspace(4, 1, 129), 4, 0.75)),
                                 (0, 16, 4, 3, top)]:
        lo, hi = lohi
        pb = 2 if lohi is top else 100
        g = R.REWL(model, L, h, 0.75, m, 1e-4, 0.8, seed=9 + model, interval=700, prep_budget=pb)
        g.set_windows(lo, hi)
        o = O.REWL(model, L, h, 0.75, m, 1e-4, 0.8, seed=9 + model, interval=700, lo_hi=(lo, hi),
                   prep_budget=pb)
        g.init()
        assert o.init() == 0
        g.run(max_rounds=30)
        o.run(30)
        _same(g.state(), o.state())
        g.close()


def test_stitch_gpu_equals_oracle_partial_run():
    g, o = _pair(3, 6, 4, 2, seed=5, interval=800)
    g.init()
    o.init()
    g.run(max_rounds=40)
    o.run(40)
    for norm in (0, 1):
        a, ja = g.stitch(norm)
        b, jb = o.stitch(norm)
        assert np.array_equal(ja, jb)
        fin = np.isfinite(b)
        assert np.array_equal(np.isfinite(a), fin)
        assert np.max(np.abs(a[fin] - b[fin])) < 1e-11
    g.close()


def test_checkpoint_restore_bit_exact(tmp_path):
    import paper_1402_2328_gb300.rewl as R
    args = (0, 8, 4, 0.75, 2, 1e-6, 0.8)
    a = R.REWL(*args, seed=9, interval=1000)
    a.init()
    a.run(max_rounds=20)
    p = str(tmp_path / "ck.bin")
    a.checkpoint(p)
    a.run(max_rounds=15)
    sa = a.state()
    b = R.REWL(*args, seed=9, interval=1000)
    b.restore(p)
    b.run(max_rounds=15)
    _same(b.state(), sa)
    c = R.REWL(0, 8, 4, 0.75, 2, 1e-6, 0.8, seed=10, interval=1000)
    with pytest.raises(R.REWLError):
        c.restore(p)
    a.close(); b.close(); c.close()


def test_edge_cases():
    import paper_1402_2328_gb300.rewl as R
    # ln f_init below ln f_final: finished before the first round
    g = R.REWL(0, 4, 2, 0.75, 1, 1e-3, 0.8, seed=1, lnf_init=1e-4, interval=100)
    assert g.run() == "done"
    assert g.get_state("round")[0] == 0
    g.close()
    with pytest.raises(R.REWLError):
        R.REWL(0, 4, 40, 0.75, 1, 1e-3, 0.8)  # windows cannot overlap
    with pytest.raises(R.REWLError):
        R.REWL(1, 4, 2, 0.75, 1, 1e-3, 0.8)  # model 1 is not a model
    g = R.REWL(0, 4, 2, 0.75, 1, 1e-3, 0.8)
    with pytest.raises(R.REWLError):
        g.set_param("no_such_key", 1)
    g.close()
    with pytest.raises(R.REWLError):
        R.REWL(0, 256, 64, 0.75, 1, 1e-3, 0.8)  # lattices up to L = 255
    with pytest.raises(R.REWLError):
        R.REWL(0, 255, 2, 0.75, 1, 1e-3, 0.8)  # window too wide for shared memory


@pytest.mark.parametrize("model,L,h,m", [(0, 2, 1, 2), (3, 2, 2, 1), (0, 255, 64, 1)])
def test_smallest_and_largest_lattices_bit_exact(model, L, h, m):
    """L = 2 (4 sites) and L = 255 (65,025 sites, 226 KB of shared memory per walker)."""
    g, o = _pair(model, L, h, m, lnf_final=1e-3, seed=17, interval=200)
    g.init()
    assert o.init() == 0
    g.run(max_rounds=3)
    o.run(3)
    _same(g.state(), o.state())
    g.close()


# ------------------------------------------------------------------ one thread per walker
@pytest.mark.parametrize("check", [0, 1])
@pytest.mark.parametrize("model,L,h,m,rounds,interval,sched", [
    (0, 8, 4, 8, 60, 1000, 0), (3, 6, 3, 16, 60, 700, 1), (0, 16, 8, 40, 25, 2000, 0),
    (10, 12, 8, 33, 25, 1500, 1), (0, 5, 2, 3, 80, 333, 0), (0, 32, 16, 70, 10, 3000, 1)])
def test_thread_layout_rounds_bit_exact(model, L, h, m, rounds, interval, sched, check):
    """The thread-per-walker move kernel (layout 1) against the oracle, round by round."""
    g, o = _pair(model, L, h, m, seed=13 + L, interval=interval, check_all=check, layout=1,
                 schedule=sched)
    g.init()
    assert o.init() == 0
    assert rounds > 8
    for chunk in (1, 7, rounds - 8):
        g.run(max_rounds=chunk)
        o.run(chunk)
        _same(g.state(), o.state())
    assert int(g.get_state("n_mismatch")[0]) == 0
    g.close()


def test_thread_layout_to_completion_bit_exact():
    """Frozen windows, the 1/t switch and the last fragments, one thread per walker."""
    g, o = _pair(0, 6, 3, 4, lnf_final=1e-5, seed=43, interval=500, layout=1, schedule=1)
    assert g.run() == "done"
    o.init()
    o.run(10 ** 7)
    _same(g.state(), o.state())
    g.close()


def test_late_balanced_windows_pipeline():
    """Pre-run to the 4th iteration of every window, windows balanced by the 2nd-4th
    iterations' cost (paper_1402_2328_gb300.balance); the layout runs bit-exactly against the
    oracle with the same windows."""
    import paper_1402_2328_gb300.rewl as R
    from paper_1402_2328_gb300 import balance as BL
    pre = R.REWL(0, 16, 8, 0.75, 2, 1e-4, 0.8, seed=15, interval=2000)
    lo, hi, info = BL.late_balanced_windows(pre, 8, it_from=2, it_to=4, chunk=16, max_seconds=120)
    assert info["complete"] and lo[0] == 0 and hi[-1] == 256
    assert np.all(lo[1:] <= hi[:-1]) and np.all(np.diff(lo) > 0)
    pre.close()
    g = R.REWL(0, 16, 8, 0.75, 2, 1e-4, 0.8, seed=16, interval=900)
    g.set_windows(lo, hi)
    o = O.REWL(0, 16, 8, 0.75, 2, 1e-4, 0.8, seed=16, interval=900, lo_hi=(lo, hi))
    g.init()
    assert o.init() == 0
    g.run(max_rounds=20)
    o.run(20)
    _same(g.state(), o.state())
    g.close()
