"""Learned warm start: orchestration of library calls (no arithmetic here).

1. plain cold-start REWL runs on small lattices (`converged_lng`, CUDA: move / flatness /
   exchange / joining kernels);
2. their joined ln g become training samples (`training_set`, CUDA: rewl_mlp_samples);
3. the 3 -> 64 -> 64 -> 1 MLP is trained with the library's forward/backward/Adam kernels
   (`train`);
4. it predicts ln g of a larger lattice (`predict_lng`, CUDA: rewl_mlp_predict), which
   seeds a REWL run starting from a small ln f (`warm_handle`).
Plain cold-start REWL stays the fallback: the predicted ln g only changes the starting
point of Wang-Landau sampling, which converges from any start.
"""
from __future__ import annotations

import numpy as np

from . import rewl as R

# Lattices whose converged ln g trains the network: Ising and q=10 Potts, L = 8 ... 32.
TRAIN_LATTICES = [(model, L) for model in (0, 10) for L in (8, 12, 16, 20, 24, 28, 32)]


def converged_lng(model, L, windows, walkers, lnf_final, seed, interval=10_000, overlap=0.75,
                  flatness=0.8, max_seconds=0.0, stream=None):
    """Joined, normalised ln g (B+1 values, -inf where unvisited) of a cold-start run."""
    r = R.REWL(model, L, windows, overlap, walkers, lnf_final, flatness, seed=seed,
               interval=interval, stream=stream)
    try:
        status = r.run(max_seconds=max_seconds)
        if status != "done":
            raise R.REWLError(f"training run model={model} L={L} did not finish ({status})")
        lng, _ = r.stitch(0)
        return lng, r.stats()
    finally:
        r.close()


def training_set(runs):
    """runs: iterable of (model, L, lng). Returns device tensors X (n x 3) and T (n)."""
    import torch
    Xs, Ts = [], []
    for model, L, lng in runs:
        B = len(lng) - 1
        X = torch.zeros((B + 1, 3), dtype=torch.float32, device="cuda")
        T = torch.zeros(B + 1, dtype=torch.float32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
        R.mlp_samples(torch.from_numpy(np.ascontiguousarray(lng, np.float64)).cuda(), model, L,
                      X, T, cnt)
        n = int(cnt.item())
        Xs.append(X[:n])
        Ts.append(T[:n])
    return torch.cat(Xs).contiguous(), torch.cat(Ts).contiguous()


def train(X, T, steps=3000, lr=3e-3, seed=0, chunk=500):
    """Full-batch Adam on the GPU; returns (parameters, loss history)."""
    import torch
    P = torch.zeros(R.MLP_NPARAM, dtype=torch.float32, device="cuda")
    R.mlp_init(P, seed)
    m, v, grad = (torch.zeros(R.MLP_NPARAM, dtype=torch.float32, device="cuda") for _ in range(3))
    work = torch.zeros(R.mlp_workspace_floats(X.shape[0]), dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    hist, done = [], 0
    while done < steps:
        k = min(chunk, steps - done)
        R.mlp_train(P, X, T, k, lr, done, m, v, grad, work, loss)
        done += k
        hist.append((done, float(loss.item())))
    return P, hist


def predict_lng(P, model, L):
    """N * net(e, q, 1/L) for the B+1 bins of the lattice (host float64 array)."""
    import torch
    B = L * L if model == 0 else 2 * L * L
    out = torch.zeros(B + 1, dtype=torch.float64, device="cuda")
    R.mlp_predict(P, model, L, out)
    return out.cpu().numpy()


def warm_handle(model, L, windows, walkers, lnf_final, seed, lng_init, lnf_init=1e-3,
                interval=10_000, overlap=0.75, flatness=0.8, stream=None):
    """A REWL handle seeded with the predicted ln g and a small starting ln f."""
    r = R.REWL(model, L, windows, overlap, walkers, lnf_final, flatness, seed=seed,
               interval=interval, lnf_init=lnf_init, stream=stream)
    r.set_lng_init(lng_init)
    return r
