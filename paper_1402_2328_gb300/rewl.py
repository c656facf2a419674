"""ctypes binding of librewl.so (include/rewl.h): argument marshalling only.

Every step of the method runs in the library's CUDA kernels; this module converts numpy
arrays / torch CUDA tensors to pointers and error codes to exceptions.  If the library
is not built, ``lib()`` raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "librewl.so")
_lib = None

STATUS = {0: "running", 1: "done", 2: "budget", 3: "aborted"}


class REWLError(RuntimeError):
    pass


class _Stats(C.Structure):
    _fields_ = [("rounds", C.c_longlong), ("attempts", C.c_longlong), ("accepted", C.c_longlong),
                ("swap_attempts", C.c_longlong), ("swap_accepted", C.c_longlong),
                ("exact_decisions", C.c_longlong), ("prep_restarts", C.c_longlong),
                ("windows_finished", C.c_int), ("min_iteration", C.c_int),
                ("max_lnf", C.c_double), ("seconds", C.c_double)]


def lib():
    """The loaded CUDA library; raises if it was not built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise REWLError(f"CUDA library not built ({LIB_PATH}); run "
                            "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        P, I, D = C.c_void_p, C.c_int, C.c_double
        sig = {
            "rewl_create": ([P, I, I, I, D, I, D, D], I),
            "rewl_set_param": ([P, C.c_char_p, D], I),
            "rewl_set_seed": ([P, C.c_uint64], I),
            "rewl_set_lng_init": ([P, P, I], I),
            "rewl_set_windows": ([P, P, I], I),
            "rewl_set_stream": ([P, P], I),
            "rewl_init": ([P], I),
            "rewl_run": ([P, D, C.c_longlong, P], I),
            "rewl_abort": ([P], I),
            "rewl_step": ([P, I], I),
            "rewl_kernel_time": ([P, P, P, I], I),
            "rewl_get_lng": ([P, I, I, P, I, P, P], I),
            "rewl_stitch": ([P, P, I, I, P], I),
            "rewl_dims": ([P, P], I),
            "rewl_get_state": ([P, C.c_char_p, P, C.c_size_t], I),
            "rewl_set_state": ([P, C.c_char_p, P, C.c_size_t], I),
            "rewl_stats": ([P, P], I),
            "rewl_checkpoint": ([P, C.c_char_p], I),
            "rewl_restore": ([P, C.c_char_p], I),
            "rewl_destroy": ([P], None),
            "rewl_last_error": ([P], C.c_char_p),
            "rewl_replay": ([I, I, I, I, I] + [P] * 12, I),
            "rewl_replay_static": ([I, I, I, I, I] + [P] * 12, I),
            "rewl_philox": ([P, P, P, I, P], I),
            "rewl_lnu": ([P, P, I, P], I),
            "rewl_lnu_bound": ([C.c_uint64, C.c_uint64, P, P, P], I),
            "rewl_lnu_eps": ([], D),
            "rewl_seqadd": ([P, P, P, P, I, P], I),
            "rewl_windows_balanced": ([P, I, I, D, P], I),
            "rewl_windows_equal": ([I, I, D, P], I),
            "rewl_windows_late_balanced": ([P, I, P, I, I, D, P], I),
            "rewl_thermo": ([P, I, I, P, I, P, P, P], I),
            "rewl_jackknife": ([P, P, I, I], I),
            "rewl_get_hist_em": ([P, P, C.c_size_t], I),
            "rewl_stitch_em": ([P, P, C.c_size_t, P], I),
            "rewl_join_em": ([P, I, I, I, I, P, D, D, D, P, P, P], I),
            "rewl_balanced_from_prerun": ([P, I, D, P], I),
            "rewl_set_shard": ([P, P, I, I], I),
            "rewl_boundary_bins": ([P, I, P], I),
            "rewl_boundary_half": ([P, I, P, P], I),
            "rewl_boundary_decide": ([P, I, P, P, P, P], I),
            "rewl_boundary_import": ([P, I, P, P, P], I),
            "rewl_balanced_scaled": ([P, I, I, D, P], I),
            "rewl_mlp_forward": ([P, P, P, I, P], I),
            "rewl_mlp_workspace_floats": ([I], I),
            "rewl_mlp_grad": ([P, P, P, I, P, P, P, P], I),
            "rewl_mlp_adam": ([P, P, P, P, I, D, P], I),
            "rewl_mlp_train": ([P, P, P, I, I, D, I, P, P, P, P, P, P], I),
            "rewl_mlp_init": ([P, C.c_uint64, P], I),
            "rewl_mlp_samples": ([P, I, I, P, P, P, P], I),
            "rewl_mlp_predict": ([P, I, I, P, P], I),
            "rewl_mlp_last_error": ([], C.c_char_p),
            "rewl_batch_create": ([P, P, I, C.c_longlong], I),
            "rewl_batch_set_param": ([P, C.c_char_p, D], I),
            "rewl_batch_set_stream": ([P, P], I),
            "rewl_batch_init": ([P], I),
            "rewl_batch_step": ([P, I], I),
            "rewl_batch_run": ([P, D, C.c_longlong, P], I),
            "rewl_batch_autotune": ([P, I, P, P], I),
            "rewl_batch_instance": ([P, I, P], I),
            "rewl_batch_info": ([P, P], I),
            "rewl_batch_kernel_time": ([P, P, P, I], I),
            "rewl_batch_destroy": ([P], None),
            "rewl_batch_last_error": ([P], C.c_char_p),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def exported_symbols():
    return [n for n in dir(lib()) if n.startswith("rewl_")]


def _check(rc, handle=None):
    if rc != 0:
        msg = lib().rewl_last_error(handle)
        raise REWLError(f"rewl error {rc}: {msg.decode() if msg else ''}")


def _ptr(a):
    """Data pointer of a numpy array or a torch tensor."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


_FIELDS = {
    "spins": (np.int8, "nwN"), "k": (np.int32, "nw"), "lng": (np.float64, "nwW"),
    "H": (np.uint32, "nwW"), "step": (np.uint64, "nw"), "acc": (np.uint64, "nw"),
    "flat": (np.uint8, "nw"), "lnf": (np.float64, "h"), "iter": (np.int32, "h"),
    "finished": (np.uint8, "h"), "mask": (np.uint8, "hW"), "swap_att": (np.uint64, "h"),
    "swap_acc": (np.uint64, "h"), "pstep": (np.uint64, "nw"), "prep_restarts": (np.int32, "nw"),
    "round": (np.int64, "1"), "lo": (np.int32, "h"), "hi": (np.int32, "h"),
    "n_exact": (np.uint64, "1"), "n_mismatch": (np.uint64, "1"), "lng_mean": (np.float64, "hW"),
    "first_iter_round": (np.int64, "h"), "mode": (np.uint8, "h"), "frag": (np.float64, "nwW"),
}


class _Desc(C.Structure):
    _fields_ = [("model", C.c_int), ("L", C.c_int), ("windows", C.c_int),
                ("walkers_per_window", C.c_int), ("overlap", C.c_double),
                ("lnf_final", C.c_double), ("flatness", C.c_double), ("lnf_init", C.c_double),
                ("seed", C.c_uint64), ("instance", C.c_int)]


class REWL:
    """One REWL simulation on the current CUDA device (see include/rewl.h)."""

    def __init__(self, model: int, L: int, windows: int, overlap: float, walkers: int,
                 lnf_final: float, flatness: float, seed: int = 0, stream=None, **params):
        self._lib = lib()
        h = C.c_void_p()
        _check(self._lib.rewl_create(C.byref(h), model, L, windows, overlap, walkers,
                                     lnf_final, flatness))
        self._h = h
        self._update_dims()
        self.set_seed(seed)
        for key, v in params.items():
            self.set_param(key, v)
        self.set_stream(stream)

    @classmethod
    def _view(cls, handle):
        """Non-owning view of a handle owned by a batch."""
        obj = cls.__new__(cls)
        obj._lib = lib()
        obj._h = handle
        obj._owned = False
        obj._update_dims()
        return obj

    def _update_dims(self):
        d = np.zeros(8, np.int32)
        _check(self._lib.rewl_dims(self._h, _ptr(d)), self._h)
        self.N, self.B, self.h, self.m, self.W, self.q, self.L, self.model = (int(v) for v in d)
        self.nw = self.h * self.m

    def close(self):
        if getattr(self, "_h", None) and getattr(self, "_owned", True):
            self._lib.rewl_destroy(self._h)
        self._h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---- configuration
    def set_param(self, key: str, value: float):
        _check(self._lib.rewl_set_param(self._h, key.encode(), float(value)), self._h)

    def set_seed(self, seed: int):
        _check(self._lib.rewl_set_seed(self._h, int(seed) & (2 ** 64 - 1)), self._h)

    def set_lng_init(self, lng_bins):
        a = np.ascontiguousarray(lng_bins, np.float64)
        _check(self._lib.rewl_set_lng_init(self._h, _ptr(a), len(a)), self._h)

    def set_windows(self, lo, hi):
        a = np.ascontiguousarray(np.concatenate([lo, hi]), np.int32)
        _check(self._lib.rewl_set_windows(self._h, _ptr(a), len(lo)), self._h)
        self._update_dims()

    def set_stream(self, stream=None):
        _check(self._lib.rewl_set_stream(self._h, _stream_ptr(stream)), self._h)

    def set_shard(self, lo, hi, w_begin: int):
        """This handle runs windows w_begin .. w_begin + windows - 1 of the global layout."""
        a = np.ascontiguousarray(np.concatenate([lo, hi]), np.int32)
        _check(self._lib.rewl_set_shard(self._h, _ptr(a), len(lo), int(w_begin)), self._h)
        self._update_dims()

    def boundary_bins(self, side: int, bins):
        _check(self._lib.rewl_boundary_bins(self._h, int(side), _ptr(bins)), self._h)

    def boundary_half(self, side: int, partner_bins, half):
        _check(self._lib.rewl_boundary_half(self._h, int(side), _ptr(partner_bins), _ptr(half)),
               self._h)

    def boundary_decide(self, side: int, half, partner_half, accepted, lattices):
        _check(self._lib.rewl_boundary_decide(self._h, int(side), _ptr(half), _ptr(partner_half),
                                              _ptr(accepted), _ptr(lattices)), self._h)

    def boundary_import(self, side: int, partner_bins, accepted, partner_lattices):
        _check(self._lib.rewl_boundary_import(self._h, int(side), _ptr(partner_bins), _ptr(accepted),
                                              _ptr(partner_lattices)), self._h)

    def balanced_windows(self, h: int, overlap: float = 0.75):
        """Windows balanced by this (pre-)run's first-iteration times (Fig. 1b)."""
        a = np.zeros(2 * h, np.int32)
        _check(self._lib.rewl_balanced_from_prerun(self._h, int(h), float(overlap), _ptr(a)),
               self._h)
        return a[:h].copy(), a[h:].copy()

    def balanced_windows_for(self, L: int, h: int, overlap: float = 0.75):
        """This run's first-iteration cost profile carried to an L x L lattice (by E/N)."""
        a = np.zeros(2 * h, np.int32)
        _check(self._lib.rewl_balanced_scaled(self._h, int(L), int(h), float(overlap), _ptr(a)),
               self._h)
        return a[:h].copy(), a[h:].copy()

    # ---- running
    def init(self):
        _check(self._lib.rewl_init(self._h), self._h)

    def run(self, max_seconds: float = 0.0, max_rounds: int = -1) -> str:
        st = C.c_int(0)
        _check(self._lib.rewl_run(self._h, float(max_seconds), int(max_rounds), C.byref(st)),
               self._h)
        return STATUS[st.value]

    def abort(self):
        _check(self._lib.rewl_abort(self._h), self._h)

    def step(self, rounds: int = 1):
        """Enqueue rounds on the handle's stream without waiting."""
        _check(self._lib.rewl_step(self._h, int(rounds)), self._h)

    def kernel_time(self, reset: bool = True):
        ms, n = C.c_double(), C.c_longlong()
        _check(self._lib.rewl_kernel_time(self._h, C.byref(ms), C.byref(n), int(reset)), self._h)
        return ms.value, n.value

    # ---- results
    def get_lng(self, window: int, walker: int = -1):
        out = np.zeros(self.W, np.float64)
        lo, hi = C.c_int(), C.c_int()
        _check(self._lib.rewl_get_lng(self._h, window, walker, _ptr(out), len(out),
                                      C.byref(lo), C.byref(hi)), self._h)
        return out[: hi.value - lo.value + 1], lo.value, hi.value

    def stitch(self, norm: int = 0):
        out = np.zeros(self.B + 1, np.float64)
        joins = np.zeros(max(self.h - 1, 1), np.int32)
        _check(self._lib.rewl_stitch(self._h, _ptr(out), len(out), norm, _ptr(joins)), self._h)
        return out, joins[: self.h - 1]

    def hist_em(self) -> np.ndarray:
        """(E, M) histogram [h][W][N+1] (parameter "measure_em" must be on)."""
        out = np.zeros((self.h, self.W, self.N + 1), np.uint32)
        _check(self._lib.rewl_get_hist_em(self._h, _ptr(out), out.nbytes), self._h)
        return out

    def stitch_em(self):
        """Joint ln g(E, M), (B+1) x (N+1) (-inf where absent), and the join points [h-1][2]."""
        out = np.zeros((self.B + 1, self.N + 1), np.float64)
        joins = np.zeros((max(self.h - 1, 1), 2), np.int32)
        _check(self._lib.rewl_stitch_em(self._h, _ptr(out), out.size, _ptr(joins)), self._h)
        return out, joins[: self.h - 1]

    def jackknife(self, norm: int = 0):
        """Per-bin jackknife error of the joined ln g (NaN where a resample has no value)."""
        out = np.zeros(self.B + 1, np.float64)
        _check(self._lib.rewl_jackknife(self._h, _ptr(out), len(out), int(norm)), self._h)
        return out

    def _shape(self, code):
        return {"nwN": (self.nw, self.N), "nw": (self.nw,), "nwW": (self.nw, self.W),
                "h": (self.h,), "hW": (self.h, self.W), "1": (1,)}[code]

    def get_state(self, field: str) -> np.ndarray:
        dt, code = _FIELDS[field]
        out = np.zeros(self._shape(code), dt)
        _check(self._lib.rewl_get_state(self._h, field.encode(), _ptr(out), out.nbytes), self._h)
        return out

    def state(self) -> dict:
        s = {f: self.get_state(f) for f in _FIELDS}
        s["round"] = int(s["round"][0])
        return s

    def set_state(self, field: str, value):
        dt, code = _FIELDS[field]
        a = np.ascontiguousarray(value, dt).reshape(self._shape(code))
        _check(self._lib.rewl_set_state(self._h, field.encode(), _ptr(a), a.nbytes), self._h)

    def stats(self) -> dict:
        s = _Stats()
        _check(self._lib.rewl_stats(self._h, C.byref(s)), self._h)
        return {n: getattr(s, n) for n, _ in _Stats._fields_}

    def checkpoint(self, path: str):
        _check(self._lib.rewl_checkpoint(self._h, os.fsencode(path)), self._h)

    def restore(self, path: str):
        _check(self._lib.rewl_restore(self._h, os.fsencode(path)), self._h)


class REWLBatch:
    """Many independent REWL instances advanced together (include/rewl.h, batched)."""

    def __init__(self, descs, interval: int = 10_000, stream=None, **params):
        self._lib = lib()
        arr = (_Desc * len(descs))()
        for a, d in zip(arr, descs):
            a.model, a.L, a.windows = d["model"], d["L"], d["windows"]
            a.walkers_per_window = d["walkers"]
            a.overlap, a.lnf_final = d.get("overlap", 0.75), d["lnf_final"]
            a.flatness, a.lnf_init = d.get("flatness", 0.8), d.get("lnf_init", 0.0)
            a.seed, a.instance = int(d["seed"]) & (2 ** 64 - 1), d.get("instance", 0)
        h = C.c_void_p()
        rc = self._lib.rewl_batch_create(C.byref(h), arr, len(descs), int(interval))
        if rc != 0:
            raise REWLError(f"rewl error {rc}: {self._lib.rewl_batch_last_error(None).decode()}")
        self._h = h
        self.n = len(descs)
        for k, v in params.items():
            self.set_param(k, v)
        self._check(self._lib.rewl_batch_set_stream(self._h, _stream_ptr(stream)))

    def _check(self, rc):
        if rc != 0:
            raise REWLError(f"rewl error {rc}: {self._lib.rewl_batch_last_error(self._h).decode()}")

    def set_param(self, key, value):
        self._check(self._lib.rewl_batch_set_param(self._h, key.encode(), float(value)))

    def init(self):
        self._check(self._lib.rewl_batch_init(self._h))

    def step(self, rounds: int = 1):
        self._check(self._lib.rewl_batch_step(self._h, int(rounds)))

    def run(self, max_seconds: float = 0.0, max_rounds: int = -1) -> str:
        st = C.c_int(0)
        self._check(self._lib.rewl_batch_run(self._h, float(max_seconds), int(max_rounds),
                                             C.byref(st)))
        return STATUS[st.value]

    TUNE_WALKERS = (2, 4, 8, 16)
    TUNE_SITES = (0, 400, 1024, 1600)
    TUNE_GRAPH = (8, 32, 128)

    def autotune(self, rounds: int = 2):
        """Choose warps per CTA x thread-per-walker site limit, then rounds per graph replay;
        returns (choice, {candidate: ms per round})."""
        best = (C.c_int * 3)()
        ms = (C.c_double * 19)()
        self._check(self._lib.rewl_batch_autotune(self._h, int(rounds), best, ms))
        keys = [f"w{w}_t{t}" for t in self.TUNE_SITES for w in self.TUNE_WALKERS]
        keys += [f"graph{g}" for g in self.TUNE_GRAPH]
        choice = dict(walkers_per_block=best[0], thread_layout_max_sites=best[1],
                      graph_rounds=best[2])
        return choice, dict(zip(keys, list(ms)))

    def instance(self, i: int) -> REWL:
        h = C.c_void_p()
        self._check(self._lib.rewl_batch_instance(self._h, int(i), C.byref(h)))
        return REWL._view(h)

    def info(self):
        out = np.zeros(6, np.int32)
        self._check(self._lib.rewl_batch_info(self._h, _ptr(out)))
        return dict(instances=int(out[0]), walkers=int(out[1]), ctas=int(out[2]),
                    warps_per_cta=int(out[3]), thread_layout_max_sites=int(out[4]),
                    graph_rounds=int(out[5]))

    def kernel_time(self, reset: bool = True):
        ms, n = C.c_double(), C.c_longlong()
        self._check(self._lib.rewl_batch_kernel_time(self._h, C.byref(ms), C.byref(n), int(reset)))
        return ms.value, n.value

    def close(self):
        if getattr(self, "_h", None):
            self._lib.rewl_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()


# ---- free functions (device tensors in, device tensors out)
def replay(model, L, spins, k, lo, hi, lng, H, lnf, frozen, words, acc, dk, stream=None):
    """In-place replay through the move kernel; all arguments are CUDA tensors."""
    n, T = words.shape[0], words.shape[1]
    W = lng.shape[1]
    _check(lib().rewl_replay(model, L, n, W, T, _ptr(spins), _ptr(k), _ptr(lo), _ptr(hi),
                             _ptr(lng), _ptr(H), _ptr(lnf), _ptr(frozen), _ptr(words), _ptr(acc),
                             _ptr(dk), _stream_ptr(stream)))


def thermo(lng, model, L, T, U, C, stream=None):
    """u(T) = <E>/N and c(T) from ln g (device tensors)."""
    _check(lib().rewl_thermo(_ptr(lng), int(model), int(L), _ptr(T), T.numel(), _ptr(U), _ptr(C),
                             _stream_ptr(stream)))


def join_em(S, lo, hi, B: int, out, de: float = 4.0, dq: float = 2.0, norm_target=None,
            stream=None):
    """Joins 2D fragments S (CUDA float64 [h][W][N1]) into out (CUDA float64 [B+1][N1]);
    norm_target defaults to (N1-1) ln 2.  Returns the join points [h-1][2] (bin, j)."""
    h, W, N1 = S.shape
    lohi = np.ascontiguousarray(np.concatenate([lo, hi]), np.int32)
    joins = np.zeros((max(h - 1, 1), 2), np.int32)
    tgt = (N1 - 1) * math.log(2.0) if norm_target is None else float(norm_target)
    _check(lib().rewl_join_em(_ptr(S), int(h), int(W), int(B), int(N1), _ptr(lohi), float(de),
                              float(dq), tgt, _ptr(out), _ptr(joins), _stream_ptr(stream)))
    return joins[: h - 1]


def num_bins(model: int, L: int) -> int:
    """B: the bins are 0..B (Ising B = N, Potts B = 2N)."""
    return L * L if model == 0 else 2 * L * L


def windows_layout(B: int, h: int, overlap: float = 0.75):
    """The equal-size window layout of Fig. 1a (the one rewl_create uses): (lo, hi)."""
    a = np.zeros(2 * h, np.int32)
    _check(lib().rewl_windows_equal(int(B), int(h), float(overlap), _ptr(a)))
    return a[:h].copy(), a[h:].copy()


def windows_late_balanced(lo, hi, rounds_per_iter, B: int, h_new: int, overlap: float = 0.75):
    """Windows with about equal (rounds per later iteration / width^2) x width^2 (host call)."""
    lh = np.ascontiguousarray(np.concatenate([lo, hi]), np.int32)
    t = np.ascontiguousarray(rounds_per_iter, np.float64)
    out = np.zeros(2 * h_new, np.int32)
    _check(lib().rewl_windows_late_balanced(_ptr(lh), len(lo), _ptr(t), int(B), int(h_new),
                                            float(overlap), _ptr(out)))
    return out[:h_new].copy(), out[h_new:].copy()


def windows_balanced(cost, h: int, overlap: float = 0.75):
    """Run-time balanced windows for a per-bin cost profile (host computation)."""
    c = np.ascontiguousarray(cost, np.float64)
    a = np.zeros(2 * h, np.int32)
    _check(lib().rewl_windows_balanced(_ptr(c), len(c) - 1, int(h), float(overlap), _ptr(a)))
    return a[:h].copy(), a[h:].copy()


MLP_NPARAM = 4481


def _mcheck(rc):
    if rc != 0:
        raise REWLError(f"rewl error {rc}: {lib().rewl_mlp_last_error().decode()}")


def mlp_forward(P, X, Y, stream=None):
    _mcheck(lib().rewl_mlp_forward(_ptr(P), _ptr(X), _ptr(Y), X.shape[0], _stream_ptr(stream)))


def mlp_workspace_floats(n: int) -> int:
    return int(lib().rewl_mlp_workspace_floats(int(n)))


def mlp_grad(P, X, T, grad, loss, work, stream=None):
    _mcheck(lib().rewl_mlp_grad(_ptr(P), _ptr(X), _ptr(T), X.shape[0], _ptr(grad), _ptr(loss),
                                _ptr(work), _stream_ptr(stream)))


def mlp_adam(P, grad, m, v, t, lr, stream=None):
    _mcheck(lib().rewl_mlp_adam(_ptr(P), _ptr(grad), _ptr(m), _ptr(v), int(t), float(lr),
                                _stream_ptr(stream)))


def mlp_train(P, X, T, steps, lr, t0, m, v, grad, work, loss, stream=None):
    _mcheck(lib().rewl_mlp_train(_ptr(P), _ptr(X), _ptr(T), X.shape[0], int(steps), float(lr),
                                 int(t0), _ptr(m), _ptr(v), _ptr(grad), _ptr(work), _ptr(loss),
                                 _stream_ptr(stream)))


def mlp_init(P, seed, stream=None):
    _mcheck(lib().rewl_mlp_init(_ptr(P), int(seed) & (2 ** 64 - 1), _stream_ptr(stream)))


def mlp_samples(lng, model, L, X, T, count, stream=None):
    _mcheck(lib().rewl_mlp_samples(_ptr(lng), int(model), int(L), _ptr(X), _ptr(T), _ptr(count),
                                   _stream_ptr(stream)))


def mlp_predict(P, model, L, out, stream=None):
    _mcheck(lib().rewl_mlp_predict(_ptr(P), int(model), int(L), _ptr(out), _stream_ptr(stream)))


REPLAY_STATIC_MAX_N = 16384


def replay_static(model, L, spins, k, lo, hi, lng, H, lnf, frozen, words, acc, dk, stream=None):
    """replay() without any device allocation (scratch in a fixed library array, at most
    REPLAY_STATIC_MAX_N cases per call; calls overlapping on the GPU race on it)."""
    n, T = words.shape[0], words.shape[1]
    W = lng.shape[1]
    _check(lib().rewl_replay_static(model, L, n, W, T, _ptr(spins), _ptr(k), _ptr(lo), _ptr(hi),
                                    _ptr(lng), _ptr(H), _ptr(lnf), _ptr(frozen), _ptr(words),
                                    _ptr(acc), _ptr(dk), _stream_ptr(stream)))


def philox(ctr, key, out, stream=None):
    _check(lib().rewl_philox(_ptr(ctr), _ptr(key), _ptr(out), ctr.shape[0], _stream_ptr(stream)))


def lnu(words, out, stream=None):
    _check(lib().rewl_lnu(_ptr(words), _ptr(out), words.numel(), _stream_ptr(stream)))


def lnu_bound(begin, end, max_err, n_bad, stream=None):
    _check(lib().rewl_lnu_bound(int(begin), int(end), _ptr(max_err), _ptr(n_bad),
                                _stream_ptr(stream)))


def lnu_eps() -> float:
    return float(lib().rewl_lnu_eps())


def seqadd(x, f, c, out, stream=None):
    _check(lib().rewl_seqadd(_ptr(x), _ptr(f), _ptr(c), _ptr(out), x.numel(), _stream_ptr(stream)))
