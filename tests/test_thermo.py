"""Canonical averages from g(E) (Eqs. 6-7): the oracle pinned by direct Boltzmann enumeration,
the CUDA kernel checked against the oracle."""
import numpy as np
import pytest

from oracle import exact_dos as X
from oracle import thermo as TH

TS = np.array([0.5, 1.0, 2.0, 2.269, 3.0, 10.0, 100.0])


def _enumerate_4x4(T):
    L, N = 4, 16
    idx = np.arange(1 << N)
    s = (((idx[:, None] >> np.arange(N)) & 1) * 2 - 1).reshape(-1, L, L)
    E = -(s * np.roll(s, 1, 1)).sum(axis=(1, 2)) - (s * np.roll(s, 1, 2)).sum(axis=(1, 2))
    E = E.astype(np.float64)
    u, c = [], []
    for t in T:
        w = np.exp(-(E - E.min()) / t)
        Z = w.sum()
        e1 = (w * E).sum() / Z
        u.append(e1 / N)
        c.append(((w * (E - e1) ** 2).sum() / Z) / (N * t * t))
    return np.array(u), np.array(c)


def test_oracle_thermo_equals_boltzmann_enumeration():
    lng = np.array(X.exact_lng(0, 4))
    u, c = TH.canonical(lng, 0, 4, TS)
    ue, ce = _enumerate_4x4(TS)
    assert np.allclose(u, ue, rtol=0, atol=1e-12) and np.allclose(c, ce, rtol=1e-10, atol=1e-14)


def test_oracle_thermo_limits():
    lng = np.array(X.exact_lng(0, 16))
    u, c = TH.canonical(lng, 0, 16, [0.05, 1e6])
    assert u[0] == pytest.approx(-2.0, abs=1e-12) and abs(u[1]) < 1e-5
    assert np.all(c >= 0) and c[0] < 1e-12
    # q = 3 Potts 3x3: u -> -2 at low T and -> -2/q at infinite T (each bond satisfied w.p. 1/q)
    lngp = np.array(X.exact_lng(3, 3, 3))
    u, _ = TH.canonical(lngp, 3, 3, [0.02, 1e9])
    assert u[0] == pytest.approx(-2.0, abs=1e-9) and u[1] == pytest.approx(-2.0 / 3, abs=1e-6)


@pytest.mark.gpu
def test_cuda_thermo_matches_oracle():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1402_2328_gb300.rewl as R
    for model, L, lng in [(0, 16, np.array(X.exact_lng(0, 16))),
                          (3, 3, np.array(X.exact_lng(3, 3, 3)))]:
        T = torch.tensor(TS, dtype=torch.float64, device="cuda")
        U = torch.zeros_like(T)
        C = torch.zeros_like(T)
        R.thermo(torch.from_numpy(lng).cuda(), model, L, T, U, C)
        u, c = TH.canonical(lng, model, L, TS)
        assert np.allclose(U.cpu().numpy(), u, rtol=1e-12, atol=1e-14)
        assert np.allclose(C.cpu().numpy(), c, rtol=1e-11, atol=1e-14)
