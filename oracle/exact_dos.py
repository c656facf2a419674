"""Exact densities of states g(E) for the 2D Ising and q-state Potts models.

TEST INFRASTRUCTURE ONLY (part of the oracle): the tests, the golden-file script and
the smoke check use these functions to pin the REWL oracle; the CUDA library never
imports them.

Bins follow the same convention as the oracle: k counts unsatisfied bonds
(Ising k = n_u / 2, E = -2N + 4k; Potts k = n_u, E = -2N + k).

Three independent routes:

* ``brute_force_*``  -- enumerate every configuration (4x4 Ising, 3x3 q=3 Potts).
* ``transfer_matrix_ising`` -- row-to-row transfer matrix, exact counts modulo a
  few primes (exact float64 BLAS products of residues < 2^20), CRT-combined.
* ``kaufman_ising`` -- Kaufman's closed-form partition function for the periodic
  m x n lattice (Phys. Rev. 76, 1232 (1949)), expanded into the polynomial
  G(y) = sum_k g_k y^k as Beale did (Phys. Rev. Lett. 76, 78 (1996)): the product of
  each pair gamma_l = gamma_{2n-l} becomes 2 +- 2 T_m(cosh gamma_l) (T = Chebyshev),
  so the square roots disappear; with x = e^{-2K} every factor is a polynomial in x
  over Z[cos(pi/n)].  We evaluate it modulo primes p = 1 (mod 2n), where cos(pi l/n)
  is an element of F_p, and rebuild the integers by CRT.
"""
from __future__ import annotations

import math
from functools import lru_cache

import numpy as np


# --------------------------------------------------------------------------- helpers
def ln_of_counts(g) -> np.ndarray:
    """ln g_k as float64 (-inf where g_k == 0); exact for arbitrarily large ints."""
    out = np.full(len(g), -np.inf)
    for i, v in enumerate(g):
        v = int(v)
        if v > 0:
            nb = v.bit_length()
            if nb <= 900:
                out[i] = math.log(v)
            else:
                sh = nb - 64
                out[i] = math.log(v >> sh) + sh * math.log(2.0)
    return out


def _primes_1_mod(mod: int, below: int, count: int) -> list[int]:
    """Largest `count` primes p < below with p = 1 (mod `mod`)."""
    out = []
    p = (below - 1) // mod * mod + 1
    while len(out) < count:
        if p < 3:
            raise ValueError("ran out of primes")
        if _is_prime(p):
            out.append(p)
        p -= mod
    return out


def _is_prime(n: int) -> bool:
    if n < 2:
        return False
    small = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)
    for s in small:
        if n % s == 0:
            return n == s
    d, r = n - 1, 0
    while d % 2 == 0:
        d //= 2
        r += 1
    for a in small:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(r - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def _crt(residues: list[np.ndarray], primes: list[int]) -> list[int]:
    """Garner/CRT: non-negative integers below prod(primes) from their residues."""
    n = len(residues[0])
    vals = [int(v) for v in residues[0]]
    M = primes[0]
    for res, p in zip(residues[1:], primes[1:]):
        inv = pow(M % p, -1, p)
        for i in range(n):
            t = ((int(res[i]) - vals[i]) % p) * inv % p
            vals[i] += M * t
        M *= p
    return vals


# --------------------------------------------------------------------------- brute force
def brute_force_ising(L: int) -> list[int]:
    """g_k, k = 0..N, by enumerating all 2^N configurations (L <= 5)."""
    N = L * L
    if N > 25:
        raise ValueError("brute force only for N <= 25")
    idx = np.arange(1 << N, dtype=np.int64)
    spins = ((idx[:, None] >> np.arange(N)) & 1).astype(np.int8)  # bit=1 -> spin +1
    s = 2 * spins - 1
    s = s.reshape(-1, L, L)
    nu = (s != np.roll(s, 1, axis=2)).sum(axis=(1, 2)) + (s != np.roll(s, 1, axis=1)).sum(axis=(1, 2))
    assert np.all(nu % 2 == 0)
    k = nu // 2
    return [int(c) for c in np.bincount(k, minlength=N + 1)]


def brute_force_potts(L: int, q: int) -> list[int]:
    """g_k, k = 0..2N, by enumerating all q^N configurations."""
    N = L * L
    if q ** N > 5_000_000:
        raise ValueError("brute force too large")
    idx = np.arange(q ** N, dtype=np.int64)
    digits = np.empty((q ** N, N), dtype=np.int8)
    t = idx.copy()
    for j in range(N):
        digits[:, j] = t % q
        t //= q
    s = digits.reshape(-1, L, L)
    nu = (s != np.roll(s, 1, axis=2)).sum(axis=(1, 2)) + (s != np.roll(s, 1, axis=1)).sum(axis=(1, 2))
    return [int(c) for c in np.bincount(nu, minlength=2 * N + 1)]


# --------------------------------------------------------------------------- transfer matrix
def _tm_mod_p(L: int, p: int) -> np.ndarray:
    """Counts of configurations by n_u (unsatisfied bonds), modulo p (p < 2^20)."""
    S = 1 << L
    rows = np.arange(S)
    rot = ((rows << 1) | (rows >> (L - 1))) & (S - 1)
    hor = np.array([bin(v).count("1") for v in (rows ^ rot)])
    vert = np.array([[bin(a ^ b).count("1") for b in range(S)] for a in range(S)])
    E = 2 * L * L + 1
    # V[s0, s, e]: first row s0, current row s, unsatisfied bonds so far e
    V = np.zeros((S, S, E), dtype=np.float64)
    V[rows, rows, hor] = 1.0
    for _ in range(L - 1):
        Vt = V.transpose(1, 0, 2).reshape(S, S * E)  # [s, (s0,e)]
        acc = np.zeros((S, S, E), dtype=np.float64)  # [t, s0, e]
        for c in range(L + 1):
            Mc = (vert == c).astype(np.float64)
            if not Mc.any():
                continue
            prod = (Mc.T @ Vt).reshape(S, S, E)  # exact: < 2^20 * 2^L
            if c:
                acc[:, :, c:] += prod[:, :, :-c]
            else:
                acc += prod
        acc = np.fmod(acc, p)
        # horizontal bonds of the new row t
        out = np.zeros_like(acc)
        for hv in np.unique(hor):
            sel = hor == hv
            if hv:
                out[sel, :, hv:] = acc[sel, :, :-hv]
            else:
                out[sel] = acc[sel]
        V = np.fmod(out.transpose(1, 0, 2), p)  # [s0, t, e]
    total = np.zeros(E, dtype=np.float64)
    for s0 in range(S):
        for c in range(L + 1):
            sel = vert[:, s0] == c
            if not sel.any():
                continue
            part = V[s0, sel, :].sum(axis=0)
            if c:
                total[c:] += part[:-c]
            else:
                total += part
        total = np.fmod(total, p)
    return total.astype(np.int64)


def transfer_matrix_ising(L: int) -> list[int]:
    """g_k, k = 0..N, exact, for L <= 8 (periodic L x L)."""
    if L > 8:
        raise ValueError("transfer matrix limited to L <= 8")
    N = L * L
    nprimes = (N + 2) // 19 + 1
    primes = _primes_1_mod(2, 1 << 20, nprimes)
    res = [_tm_mod_p(L, p) for p in primes]
    nu_counts = _crt(res, primes)
    assert all(nu_counts[i] == 0 for i in range(1, len(nu_counts), 2))
    return nu_counts[0::2][: N + 1]


# --------------------------------------------------------------------------- Kaufman / Beale
def _pmul(a: np.ndarray, b: np.ndarray, p: int) -> np.ndarray:
    # residues < 2^26 -> products < 2^52; min(len) <= 2^11 terms keeps sums < 2^63
    if min(len(a), len(b)) > 2048:
        raise ValueError("polynomial too long for exact int64 convolution")
    return np.convolve(a, b) % p


def _padd(a: np.ndarray, b: np.ndarray, p: int, sb: int = 1) -> np.ndarray:
    n = max(len(a), len(b))
    out = np.zeros(n, dtype=np.int64)
    out[: len(a)] += a
    out[: len(b)] += sb * b
    return out % p


def _ppow(a: np.ndarray, e: int, p: int) -> np.ndarray:
    out = np.array([1], dtype=np.int64)
    for _ in range(e):
        out = _pmul(out, a, p)
    return out


def _kaufman_mod_p(m: int, n: int, p: int) -> np.ndarray:
    """G(y) mod p for the periodic m x n Ising lattice (m, n even)."""
    N = m * n
    # primitive 2n-th root of unity
    two_n = 2 * n
    rdiv = [r for r in range(2, two_n + 1) if two_n % r == 0 and _is_prime(r)]
    g = 2
    while True:
        z = pow(g, (p - 1) // two_n, p)
        if all(pow(z, two_n // r, p) != 1 for r in rdiv):  # order exactly 2n
            break
        g += 1
    inv2 = pow(2, -1, p)
    A = lambda v: np.array(v, dtype=np.int64) % p  # noqa: E731
    D = A([0, 2, 0, -2])  # 2x(1-x^2): denominator of cosh2K coth2K
    D2 = _pmul(D, D, p)
    Dm = _ppow(D, m, p)

    def plus_minus(l: int):
        c = (pow(z, l, p) + pow(z, 2 * n - l, p)) * inv2 % p  # cos(pi l / n)
        P = A([1, -2 * c, 2, 2 * c, 1])  # (1+x^2)^2 - 2x(1-x^2) cos  ==  D * cosh(gamma_l)
        u_prev, u = A([1]), P
        for _ in range(m - 1):  # U_j = T_j(P/D) D^j
            u_prev, u = u, _padd(_pmul(A([2]), _pmul(P, u, p), p), _pmul(D2, u_prev, p), p, -1)
        two_u, two_dm = 2 * u % p, 2 * Dm % p
        return _padd(two_dm, two_u, p), _padd(two_u, two_dm, p, -1)

    num = []
    # odd l: pairs (l, 2n-l), l = 1, 3, ..., n-1
    n1, n2 = A([1]), A([1])
    for l in range(1, n, 2):
        pl, mi = plus_minus(l)
        n1, n2 = _pmul(n1, pl, p), _pmul(n2, mi, p)
    num += [n1, n2]
    # even l: pairs l = 2, ..., n-2 plus singles l = 0 and l = n
    n3, n4 = A([1]), A([1])
    for l in range(2, n, 2):
        pl, mi = plus_minus(l)
        n3, n4 = _pmul(n3, pl, p), _pmul(n4, mi, p)
    a, b = A([1, -1]), A([0, 1, 1])  # e^{gamma_0} = (1-x) / (x(1+x))
    c_, d_ = A([1, 1]), A([0, 1, -1])  # e^{gamma_n} = (1+x) / (x(1-x))
    am, bm, cm, dm = (_ppow(v, m, p) for v in (a, b, c_, d_))
    two_m = pow(2, m, p)
    s3 = _pmul(_padd(am, bm, p), _padd(cm, dm, p), p) * two_m % p
    s4 = _pmul(_padd(am, bm, p, -1), _padd(cm, dm, p, -1), p) * two_m % p
    num += [_pmul(n3, s3, p), _pmul(n4, s4, p)]
    tot = np.zeros(2 * N + 1, dtype=np.int64)
    for v in num:
        tot[: len(v)] += v
    tot %= p
    if np.any(tot[1::2]):
        raise AssertionError("odd powers of x must cancel")
    inv = pow(pow(2, N // 2 + 1, p), -1, p)
    return tot[0::2] * inv % p


def kaufman_ising(L: int) -> list[int]:
    """g_k, k = 0..N, exact, periodic L x L Ising, L even (Kaufman/Beale)."""
    if L % 2 or L < 2:
        raise ValueError("even L only")
    N = L * L
    nprimes = (N + 2) // 25 + 2  # product of primes > 2^(N+1) >= 2 * sum g
    primes = _primes_1_mod(2 * L, 1 << 26, nprimes)
    res = [_kaufman_mod_p(L, L, p) for p in primes]
    vals = _crt(res, primes)
    M = math.prod(primes)
    # true values are in [0, 2^N]; anything above M/2 would mean a sign error
    if any(v > M // 2 for v in vals):
        raise AssertionError("negative coefficient: formula error")
    return vals


@lru_cache(maxsize=None)
def brute_force_ising_em(L: int) -> np.ndarray:
    """g[k][j] (int64): configurations with k = n_u / 2 unsatisfied-bond pairs and j spins up
    (magnetisation M = 2j - N), by enumerating all 2^N configurations (N <= 20)."""
    N = L * L
    if N > 20:
        raise ValueError("brute force (E, M) only for N <= 20")
    idx = np.arange(1 << N, dtype=np.int64)
    up = ((idx[:, None] >> np.arange(N)) & 1).astype(np.int8)
    s = (2 * up - 1).reshape(-1, L, L)
    nu = (s != np.roll(s, 1, axis=2)).sum(axis=(1, 2)) + (s != np.roll(s, 1, axis=1)).sum(axis=(1, 2))
    j = up.sum(axis=1)
    g = np.zeros((N + 1, N + 1), dtype=np.int64)
    np.add.at(g, (nu // 2, j), 1)
    return g


def transfer_matrix_ising_em(L: int) -> np.ndarray:
    """g[k][j] (int64) of the periodic L x L Ising model, L <= 6, by a row transfer matrix.

    State: (first row, current row, unsatisfied bonds so far, up spins so far).  Adding row b
    after row a adds the horizontal unsatisfied bonds of b, the vertical ones between a and b
    (popcount(a ^ b)) and popcount(b) up spins; the last row closes onto the first.  Counts stay
    below 2^36, so float64 matrix products over the previous row are exact."""
    if L > 6:
        raise ValueError("(E, M) transfer matrix only for L <= 6")
    N, R = L * L, 1 << L
    U, J = 2 * N + 1, N + 1
    pop = np.array([bin(r).count("1") for r in range(R)])
    rot = np.array([((r >> 1) | ((r & 1) << (L - 1))) for r in range(R)])
    hu = np.array([bin(r ^ rot[r]).count("1") for r in range(R)])
    vd = np.array([[bin(a ^ b).count("1") for b in range(R)] for a in range(R)])
    T = np.zeros((R, R, U, J))
    for r0 in range(R):
        T[r0, r0, hu[r0], pop[r0]] = 1.0
    for _ in range(L - 1):
        Tn = np.zeros_like(T)
        for d in range(L + 1):
            A = (vd == d).astype(np.float64)                     # A[a, b]
            S = np.tensordot(T, A, axes=([1], [0]))              # S[z, u, j, b]
            for b in range(R):
                du, dj = d + hu[b], pop[b]
                if du < U and dj < J:
                    Tn[:, b, du:, dj:] += S[:, :U - du, :J - dj, b]
        T = Tn
    g = np.zeros((N + 1, N + 1), dtype=np.int64)
    for r0 in range(R):
        for a in range(R):
            d = vd[a, r0]
            sub = T[r0, a, :U - d, :]
            us = np.nonzero(sub.any(axis=1))[0]
            for u in us:
                ut = u + d
                assert ut % 2 == 0
                g[ut // 2] += np.rint(sub[u]).astype(np.int64)
    return g


def exact_lng(model: int, L: int, q: int = 2) -> tuple:
    """ln g_k over the oracle's bins (tuple of floats, -inf where g = 0)."""
    if model == 0:
        if L * L <= 16:
            g = brute_force_ising(L)
        elif L % 2 == 0:
            g = kaufman_ising(L)
        else:
            g = transfer_matrix_ising(L)
        return tuple(ln_of_counts(g))
    if q ** (L * L) <= 5_000_000:
        return tuple(ln_of_counts(brute_force_potts(L, q)))
    if q == 2 and L % 2 == 0:
        # q=2 Potts == Ising with k_P = 2 k_I
        gi = kaufman_ising(L)
        g = [0] * (2 * L * L + 1)
        for k, v in enumerate(gi):
            g[2 * k] = v
        return tuple(ln_of_counts(g))
    raise ValueError("no exact DOS for this Potts lattice")


def normalise_lng(lng: np.ndarray, target: float) -> np.ndarray:
    """Shift finite entries so that logsumexp == target."""
    lng = np.asarray(lng, dtype=np.float64).copy()
    fin = np.isfinite(lng)
    mx = lng[fin].max()
    lse = mx + math.log(np.exp(lng[fin] - mx).sum())
    lng[fin] -= lse - target
    return lng
