"""CPU oracle for replica-exchange Wang-Landau sampling (arXiv:1402.2328).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  The CUDA library never imports
it and shares no code with it.

* ``rewl_oracle.c``  -- plain single-threaded C: Philox4x32-10, the deterministic ln u,
  window bounds, one WL move, the full REWL loop (moves, flatness, window advance,
  replica exchange) and the joining of Sec. 3 (Eq. 2).
* ``exact_dos.py``   -- exact g(E): enumeration, transfer matrix, Kaufman/Beale.
* ``mlp.py``         -- float64 MLP forward/backward for the learned warm start.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rewl_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "librewl_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (no fast-math, no FP contraction)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
                               "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        P = C.c_void_p
        L.or_philox.argtypes = [P, P, P]
        L.or_lnu.argtypes = [C.c_uint32]
        L.or_lnu.restype = C.c_double
        L.or_windows.argtypes = [C.c_int, C.c_int, C.c_double, P, P]
        L.or_energy.argtypes = [C.c_int, C.c_int, P]
        L.or_energy.restype = C.c_longlong
        L.or_replay_batch.argtypes = [C.c_int] * 5 + [P] * 11
        L.or_rewl_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_int, C.c_double,
                                     C.c_double, C.c_uint64, C.c_uint32, C.c_longlong,
                                     C.c_longlong, C.c_double]
        L.or_rewl_create.restype = P
        L.or_rewl_create_windows.argtypes = [C.c_int, C.c_int, C.c_int, P, P, C.c_double, C.c_int,
                                             C.c_double, C.c_double, C.c_uint64, C.c_uint32,
                                             C.c_longlong, C.c_longlong, C.c_double]
        L.or_rewl_create_windows.restype = P
        L.or_rewl_destroy.argtypes = [P]
        L.or_rewl_set_lng.argtypes = [P, P]
        L.or_rewl_init.argtypes = [P]
        L.or_rewl_round.argtypes = [P]
        L.or_rewl_run.argtypes = [P, C.c_longlong]
        L.or_rewl_run.restype = C.c_longlong
        L.or_rewl_dims.argtypes = [P, P]
        L.or_rewl_windows_get.argtypes = [P, P, P]
        L.or_rewl_get.argtypes = [P] * 17
        L.or_rewl_put.argtypes = [P] * 6
        L.or_rewl_put_window.argtypes = [P] * 8
        L.or_rewl_check.argtypes = [P, C.c_int]
        L.or_rewl_window_mean.argtypes = [P, C.c_int, P]
        L.or_rewl_set_schedule.argtypes = [P, C.c_int]
        L.or_rewl_get_extra.argtypes = [P, P, P, P]
        L.or_stitch.argtypes = [C.c_int, C.c_int, C.c_int, P, P, P, P, C.c_double, C.c_int,
                                C.c_int, C.c_double, P, P]
        L.or_rewl_swap.argtypes = [P, C.c_int, C.c_longlong]
        L.or_ln.argtypes = [C.c_double]
        L.or_ln.restype = C.c_double
        L.or_rewl_measure_em.argtypes = [P, C.c_int]
        L.or_rewl_set_production.argtypes = [P, C.c_int]
        L.or_rewl_get_hem.argtypes = [P, P]
        L.or_frag_em.argtypes = [C.c_int, C.c_int, C.c_int, P, P, P, P, P, P]
        L.or_join_em.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, P, P, P, C.c_double,
                                 C.c_double, C.c_double, P, P]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox(_p(c), _p(k), _p(out))
    return out


def lnu(w: int) -> float:
    return lib().or_lnu(int(w) & 0xFFFFFFFF)


def windows(B: int, h: int, overlap: float):
    lo = np.zeros(h, dtype=np.int32)
    hi = np.zeros(h, dtype=np.int32)
    rc = lib().or_windows(B, h, overlap, _p(lo), _p(hi))
    if rc != 0:
        raise ValueError(f"invalid window layout (rc={rc})")
    return lo, hi


def energy(model: int, L: int, spins: np.ndarray) -> int:
    s = np.ascontiguousarray(spins, dtype=np.int8)
    return int(lib().or_energy(model, L, _p(s)))


def num_bins(model: int, L: int) -> int:
    return L * L if model == 0 else 2 * L * L


def replay_batch(model, q, L, spins, k, lo, hi, lng, H, lnf, frozen, words):
    """n independent single WL attempts; arrays are updated in place (copies returned)."""
    spins = np.ascontiguousarray(spins, dtype=np.int8).copy()
    k = np.ascontiguousarray(k, dtype=np.int32).copy()
    lng = np.ascontiguousarray(lng, dtype=np.float64).copy()
    H = np.ascontiguousarray(H, dtype=np.uint32).copy()
    n, W = lng.shape
    lo = np.ascontiguousarray(lo, dtype=np.int32)
    hi = np.ascontiguousarray(hi, dtype=np.int32)
    lnf = np.ascontiguousarray(lnf, dtype=np.float64)
    frozen = np.ascontiguousarray(frozen, dtype=np.uint8)
    words = np.ascontiguousarray(words, dtype=np.uint32)
    acc = np.zeros(n, dtype=np.int32)
    dk = np.zeros(n, dtype=np.int32)
    lib().or_replay_batch(model, q, L, n, W, _p(spins), _p(k), _p(lo), _p(hi), _p(lng), _p(H),
                          _p(lnf), _p(frozen), _p(words), _p(acc), _p(dk))
    return dict(spins=spins, k=k, lng=lng, H=H, acc=acc, dk=dk)


class REWL:
    """The whole REWL simulation, one round at a time (plain C, single thread)."""

    def __init__(self, model: int, L: int, windows: int, overlap: float, walkers: int,
                 lnf_final: float, flatness: float, seed: int, instance: int = 0,
                 interval: int = 10_000, prep_budget: int = 100, lnf_init: float = 1.0,
                 lng_init=None, schedule: int = 0, lo_hi=None):
        """lo_hi: optional (lo, hi) window layout; `windows` must then equal len(lo)."""
        self._lib = lib()
        if lo_hi is None:
            self._h = self._lib.or_rewl_create(model, L, windows, overlap, walkers, lnf_final,
                                               flatness, seed, instance, interval, prep_budget,
                                               lnf_init)
        else:
            lo = np.ascontiguousarray(lo_hi[0], dtype=np.int32)
            hi = np.ascontiguousarray(lo_hi[1], dtype=np.int32)
            if len(lo) != windows or len(hi) != windows:
                raise ValueError("oracle: lo_hi does not have `windows` entries")
            self._h = self._lib.or_rewl_create_windows(model, L, windows, _p(lo), _p(hi), overlap,
                                                       walkers, lnf_final, flatness, seed,
                                                       instance, interval, prep_budget, lnf_init)
        if not self._h:
            raise ValueError("oracle: invalid REWL parameters")
        d = np.zeros(5, dtype=np.int32)
        self._lib.or_rewl_dims(self._h, _p(d))
        self.N, self.B, self.h, self.m, self.W = (int(v) for v in d)
        self.model, self.L = model, L
        self.q = 2 if model == 0 else model
        self.lo = np.zeros(self.h, dtype=np.int32)
        self.hi = np.zeros(self.h, dtype=np.int32)
        self._lib.or_rewl_windows_get(self._h, _p(self.lo), _p(self.hi))
        self._lib.or_rewl_set_schedule(self._h, schedule)
        if lng_init is not None:
            g = np.ascontiguousarray(lng_init, dtype=np.float64)
            assert g.shape == (self.B + 1,)
            self._lib.or_rewl_set_lng(self._h, _p(g))
        self.init_rc = None

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.or_rewl_destroy(h)
            self._h = None

    def init(self) -> int:
        self.init_rc = int(self._lib.or_rewl_init(self._h))
        return self.init_rc

    def round(self):
        self._lib.or_rewl_round(self._h)

    def run(self, max_rounds: int) -> int:
        return int(self._lib.or_rewl_run(self._h, max_rounds))

    def state(self) -> dict:
        nw, W, h, N = self.h * self.m, self.W, self.h, self.N
        s = dict(spins=np.zeros((nw, N), np.int8), k=np.zeros(nw, np.int32),
                 lng=np.zeros((nw, W), np.float64), H=np.zeros((nw, W), np.uint32),
                 step=np.zeros(nw, np.uint64), acc=np.zeros(nw, np.uint64),
                 flat=np.zeros(nw, np.uint8), lnf=np.zeros(h, np.float64),
                 iter=np.zeros(h, np.int32), finished=np.zeros(h, np.uint8),
                 mask=np.zeros((h, W), np.uint8), swap_att=np.zeros(h, np.uint64),
                 swap_acc=np.zeros(h, np.uint64), pstep=np.zeros(nw, np.uint64),
                 prep_restarts=np.zeros(nw, np.int32))
        rd = C.c_longlong(0)
        order = ["spins", "k", "lng", "H", "step", "acc", "flat", "lnf", "iter", "finished", "mask",
                 "swap_att", "swap_acc", "pstep", "prep_restarts"]
        self._lib.or_rewl_get(self._h, *[_p(s[o]) for o in order], C.byref(rd))
        s["round"] = rd.value
        s["first_iter_round"] = np.zeros(h, np.int64)
        s["mode"] = np.zeros(h, np.uint8)
        s["frag"] = np.zeros((nw, W), np.float64)
        self._lib.or_rewl_get_extra(self._h, _p(s["first_iter_round"]), _p(s["mode"]),
                                    _p(s["frag"]))
        return s

    def put(self, spins=None, k=None, lng=None, H=None, step=None):
        keep = [np.ascontiguousarray(a, dtype=dt) if a is not None else None
                for a, dt in ((spins, np.int8), (k, np.int32), (lng, np.float64),
                              (H, np.uint32), (step, np.uint64))]
        self._lib.or_rewl_put(self._h, *[(_p(a) if a is not None else None) for a in keep])

    def put_window(self, lnf=None, iter=None, flat=None, finished=None, mask=None, mode=None,
                   round=None):
        """Overwrite window-level fields (lnf [h], iter [h], flat [nw], finished [h],
        mask [h][W], mode [h]) and the round counter; None keeps a field."""
        keep = [np.ascontiguousarray(a, dtype=dt) if a is not None else None
                for a, dt in ((lnf, np.float64), (iter, np.int32), (flat, np.uint8),
                              (finished, np.uint8), (mask, np.uint8), (mode, np.uint8))]
        rd = C.c_longlong(int(round)) if round is not None else None
        self._lib.or_rewl_put_window(self._h, *[(_p(a) if a is not None else None) for a in keep],
                                     C.byref(rd) if rd is not None else None)

    def check(self, w: int):
        """Only the flatness test and window advance of window w (Sec. 2), as a round runs it."""
        self._lib.or_rewl_check(self._h, int(w))

    def window_mean(self, w: int) -> np.ndarray:
        out = np.zeros(int(self.hi[w] - self.lo[w] + 1), dtype=np.float64)
        self._lib.or_rewl_window_mean(self._h, w, _p(out))
        return out

    def jackknife(self, norm: int = 0):
        """Per-bin jackknife error of the joined ln g over the m walker fragments (Sec. 3)."""
        st = self.state()
        return jackknife(self.model, self.L, self.lo, self.hi, st["frag"], st["mask"], self.m,
                         norm)

    def swap(self, w: int, rd: int):
        """Only the exchange of windows (w, w+1) as round rd performs it (Eq. 1)."""
        self._lib.or_rewl_swap(self._h, int(w), int(rd))

    def measure_em(self, on: bool = True):
        """Count every walker's (bin, up spins) after the moves of each round (Ising)."""
        if self._lib.or_rewl_measure_em(self._h, int(on)) != 0:
            raise ValueError("oracle: (E, M) measurement needs the Ising model")

    def set_production(self, on: bool = True):
        """run() keeps going after every window finished (frozen ln g)."""
        self._lib.or_rewl_set_production(self._h, int(on))

    def hist_em(self) -> np.ndarray:
        out = np.zeros((self.h, self.W, self.N + 1), np.uint32)
        if self._lib.or_rewl_get_hem(self._h, _p(out)) != 0:
            raise ValueError("oracle: (E, M) measurement is off")
        return out

    def window_means(self) -> np.ndarray:
        lngw = np.zeros((self.h, self.W), np.float64)
        for w in range(self.h):
            mwin = self.window_mean(w)
            lngw[w, : len(mwin)] = mwin
        return lngw

    def stitch_em(self):
        """Joint ln g(E, M) over (B+1) x (N+1) points (Sec. 3, Eqs. 3-4)."""
        S = frag_em(self.lo, self.hi, self.window_means(), self.state()["mask"], self.hist_em())
        return join_em(self.lo, self.hi, S, self.B, self.N)

    def stitch(self, norm: int = 0):
        """Joined ln g over the B+1 bins (Sec. 3, Eq. 2) from the window means."""
        st = self.state()
        lngw = np.zeros((self.h, self.W), np.float64)
        for w in range(self.h):
            mwin = self.window_mean(w)
            lngw[w, : len(mwin)] = mwin
        return stitch(self.model, self.L, self.lo, self.hi, lngw, st["mask"], norm)


def stitch(model: int, L: int, lo, hi, lngw, valid, norm: int = 0):
    N = L * L
    q = 2 if model == 0 else model
    B = num_bins(model, L)
    h, W = lngw.shape
    de = 4.0 if model == 0 else 1.0
    step = 2 if (model != 0 and q == 2) else 1
    target = N * np.log(q) if norm == 0 else np.log(q)
    out = np.zeros(B + 1, dtype=np.float64)
    joins = np.zeros(max(h - 1, 1), dtype=np.int32)
    lo = np.ascontiguousarray(lo, np.int32)
    hi = np.ascontiguousarray(hi, np.int32)
    lngw = np.ascontiguousarray(lngw, np.float64)
    valid = np.ascontiguousarray(valid, np.uint8)
    rc = lib().or_stitch(h, W, B, _p(lo), _p(hi), _p(lngw), _p(valid), de, step, norm, target,
                         _p(out), _p(joins))
    if rc != 0:
        raise ValueError("oracle stitch: cannot join windows")
    return out, joins[: h - 1]


def ln(x: float) -> float:
    """The oracle's deterministic logarithm (exponent split + atanh series), x > 0 normal."""
    return float(lib().or_ln(float(x)))


def frag_em(lo, hi, mean, valid, hem):
    """Fragments S_w(k, j) = mean ln g_w(k) + ln H_w(k, j) - ln sum_j H_w(k, j) (-inf where
    absent); mean/valid [h][W], hem [h][W][N+1] -> [h][W][N+1]."""
    hem = np.ascontiguousarray(hem, np.uint32)
    h, W, N1 = hem.shape
    S = np.zeros((h, W, N1), np.float64)
    lib().or_frag_em(h, W, N1, _p(np.ascontiguousarray(lo, np.int32)),
                     _p(np.ascontiguousarray(hi, np.int32)),
                     _p(np.ascontiguousarray(mean, np.float64)),
                     _p(np.ascontiguousarray(valid, np.uint8)), _p(hem), _p(S))
    return S


def join_em(lo, hi, S, B: int, N: int):
    """Joint ln g(E, M) from window fragments S [h][W][N+1] (Ising: dE = 4 per bin, dM = 2 per
    up spin), normalised to sum g = 2^N.  Returns ((B+1) x (N+1) array, joins [h-1][2])."""
    S = np.ascontiguousarray(S, np.float64)
    h, W, N1 = S.shape
    out = np.zeros((B + 1, N1), np.float64)
    joins = np.zeros((max(h - 1, 1), 2), np.int32)
    rc = lib().or_join_em(h, W, B, N1, _p(np.ascontiguousarray(lo, np.int32)),
                          _p(np.ascontiguousarray(hi, np.int32)), _p(S), 4.0, 2.0,
                          N * np.log(2.0), _p(out), _p(joins))
    if rc != 0:
        raise ValueError("oracle join_em: adjacent fragments share no point")
    return out, joins[: h - 1]


def jackknife(model: int, L: int, lo, hi, frag, mask, m: int, norm: int = 0):
    """Jackknife error of the joined ln g: frag [h*m][W] holds each walker's window-local ln g
    (walker i of window w at row w*m+i); for j = 1..m the windows' means without walker j are
    joined (Sec. 3, Eq. 2); err = sqrt((m-1)/m sum_j (theta_j - mean)^2), NaN where a
    resample has no value."""
    frag = np.asarray(frag, np.float64)
    lo = np.asarray(lo)
    hi = np.asarray(hi)
    h, W = len(lo), frag.shape[1]
    thetas = []
    for j in range(m):
        lngw = np.zeros((h, W), np.float64)
        for w in range(h):
            nb = int(hi[w] - lo[w] + 1)
            acc = np.zeros(nb)
            for i in range(m):
                if i != j:
                    acc = acc + frag[w * m + i, :nb]
            lngw[w, :nb] = acc / (m - 1)
        thetas.append(stitch(model, L, lo, hi, lngw, mask, norm)[0])
    th = np.array(thetas)
    fin = np.all(np.isfinite(th), axis=0)
    err = np.full(th.shape[1], np.nan)
    mean = th[:, fin].mean(axis=0)
    err[fin] = np.sqrt((m - 1) / m * ((th[:, fin] - mean) ** 2).sum(axis=0))
    return err
