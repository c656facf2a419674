"""Warm-start MLP: the float64 oracle pinned by central differences and closed forms; the CUDA
forward, gradient, Adam and sample extraction checked against it."""
import math

import numpy as np
import pytest

from oracle import mlp as M
from tests import inputs as I


def test_oracle_gradient_matches_central_differences():
    p = I.mlp_params(1, scale=0.2)
    X, T = I.mlp_data(2, 40)
    loss, g = M.loss_and_grad(p, X, T)
    rng = np.random.default_rng(3)
    idx = np.concatenate([rng.choice(M.NPARAM, 60, replace=False), [0, 191, 192, 255, 256,
                                                                       4351, 4352, 4415, 4416, 4480]])
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        num = (M.loss_and_grad(pp, X, T)[0] - M.loss_and_grad(pm, X, T)[0]) / (2 * h)
        assert abs(num - g[i]) <= 1e-6 * max(1.0, abs(num)), (i, num, g[i])


def test_oracle_closed_forms():
    # all weights zero: the output is b3 for every input, only b3 has a gradient
    p = np.zeros(M.NPARAM)
    p[-1] = 0.7
    X, T = I.mlp_data(4, 17)
    y, _ = M.forward(p, X)
    assert np.allclose(y, 0.7)
    loss, g = M.loss_and_grad(p, X, T)
    assert loss == pytest.approx(np.mean((0.7 - T.astype(np.float64)) ** 2))
    assert g[-1] == pytest.approx(2 * np.mean(0.7 - T.astype(np.float64)))
    assert np.count_nonzero(g[:-1]) == 0
    # Adam's first step moves every parameter with a nonzero gradient by lr (bias correction)
    m = np.zeros(M.NPARAM)
    v = np.zeros(M.NPARAM)
    p2, _, _ = M.adam(p, g, m, v, 1, 1e-2)
    assert p2[-1] == pytest.approx(0.7 - 1e-2 * math.copysign(1, g[-1]), abs=1e-9)


def test_features_map_ising_onto_q2_potts():
    # Ising bin k has E_P = (E_I - 2N)/2 = -2N + 2k: the same e as q=2 Potts bin 2k
    L = 8
    fi = M.features(0, L, np.arange(0, 65))
    fp = M.features(2, L, 2 * np.arange(0, 65))
    assert np.allclose(fi, fp)
    assert fi[0, 0] == -2.0 and fi[-1, 0] == 0.0


# ---------------------------------------------------------------- CUDA side
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_2328_gb300 import build as B
    B.build()
    import paper_1402_2328_gb300.rewl as R
    return R


@pytest.mark.gpu
def test_cuda_forward_and_gradient_match_oracle(R):
    p = I.mlp_params(5, scale=0.15)
    X, T = I.mlp_data(6, 1000)  # 8 tiles with a ragged tail
    P = torch.tensor(p, dtype=torch.float32, device="cuda")
    Xd = torch.from_numpy(X).cuda()
    Td = torch.from_numpy(T).cuda()
    Y = torch.zeros(len(T), dtype=torch.float32, device="cuda")
    R.mlp_forward(P, Xd, Y)
    y_ref, _ = M.forward(p, X)
    assert np.max(np.abs(Y.cpu().numpy() - y_ref)) < 2e-5
    grad = torch.zeros(M.NPARAM, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    work = torch.zeros(R.mlp_workspace_floats(len(T)), dtype=torch.float32, device="cuda")
    R.mlp_grad(P, Xd, Td, grad, loss, work)
    l_ref, g_ref = M.loss_and_grad(p, X, T)
    g = grad.cpu().numpy().astype(np.float64)
    assert loss.item() == pytest.approx(l_ref, rel=1e-4)
    scale = np.max(np.abs(g_ref))
    assert np.max(np.abs(g - g_ref)) < 1e-4 * scale
    # deterministic: a second evaluation gives the same bits
    grad2 = torch.zeros_like(grad)
    R.mlp_grad(P, Xd, Td, grad2, loss, work)
    assert torch.equal(grad, grad2)


@pytest.mark.gpu
def test_cuda_adam_steps_match_oracle(R):
    # the update rule alone, fed the same gradients (Adam divides by sqrt(v), so comparing
    # whole training runs would amplify float32 gradient noise of near-zero components)
    rng = np.random.default_rng(7)
    p = I.mlp_params(7, scale=0.15)
    P = torch.tensor(p, dtype=torch.float32, device="cuda")
    m = torch.zeros(M.NPARAM, dtype=torch.float32, device="cuda")
    v = torch.zeros_like(m)
    pr, mr, vr = p.copy(), np.zeros(M.NPARAM), np.zeros(M.NPARAM)
    for t in range(1, 6):
        g = rng.normal(0, 1e-2, M.NPARAM).astype(np.float32)
        R.mlp_adam(P, torch.from_numpy(g).cuda(), m, v, t, 1e-3)
        pr, mr, vr = M.adam(pr, g.astype(np.float64), mr, vr, t, 1e-3)
    assert np.max(np.abs(P.cpu().numpy() - pr)) < 1e-6
    assert np.max(np.abs(v.cpu().numpy() - vr)) < 1e-9


@pytest.mark.gpu
def test_cuda_training_reduces_loss_and_samples_follow_bins(R):
    X, T = I.mlp_data(9, 4000)
    P = torch.zeros(M.NPARAM, dtype=torch.float32, device="cuda")
    R.mlp_init(P, 123)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    m, v, grad = (torch.zeros(M.NPARAM, dtype=torch.float32, device="cuda") for _ in range(3))
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    work = torch.zeros(R.mlp_workspace_floats(len(T)), dtype=torch.float32, device="cuda")
    R.mlp_train(P, Xd, Td, 1, 3e-3, 0, m, v, grad, work, loss)
    l0 = loss.item()
    R.mlp_train(P, Xd, Td, 400, 3e-3, 1, m, v, grad, work, loss)
    assert loss.item() < 0.05 * l0
    # samples: visited bins in bin order with Potts-convention features
    lng = np.array([0.7, -np.inf, 2.0, 3.5, 4.0], dtype=np.float64)  # model 0, L=2: B=4
    out_X = torch.zeros((5, 3), dtype=torch.float32, device="cuda")
    out_T = torch.zeros(5, dtype=torch.float32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    R.mlp_samples(torch.from_numpy(lng).cuda(), 0, 2, out_X, out_T, cnt)
    assert cnt.item() == 4
    ref = M.features(0, 2, [0, 2, 3, 4])
    assert np.allclose(out_X.cpu().numpy()[:4], ref)
    assert np.allclose(out_T.cpu().numpy()[:4], np.array([0.7, 2.0, 3.5, 4.0]) / 4)
    pred = torch.zeros(5, dtype=torch.float64, device="cuda")
    R.mlp_predict(P, 0, 2, pred)
    Y = torch.zeros(5, dtype=torch.float32, device="cuda")
    R.mlp_forward(P, torch.from_numpy(M.features(0, 2, np.arange(5)).astype(np.float32)).cuda(), Y)
    assert np.allclose(pred.cpu().numpy(), 4 * Y.cpu().numpy().astype(np.float64), rtol=1e-6)
