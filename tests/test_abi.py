"""CPU-only checks of the boundary: the library builds, loads and exports every symbol
that include/rewl.h declares; the binding fails loudly without it.  No compute calls."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(rewl_\w+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def built():
    from paper_1402_2328_gb300 import build as B
    return B.build()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["rewl_create", "rewl_run", "rewl_get_lng", "rewl_stitch", "rewl_replay",
              "rewl_set_param", "rewl_set_lng_init", "rewl_set_stream", "rewl_stats",
              "rewl_checkpoint", "rewl_restore", "rewl_destroy", "rewl_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(built):
    lib = ctypes.CDLL(built)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_header(built):
    import paper_1402_2328_gb300.rewl as R
    lib = R.lib()
    for n in _declared():
        assert getattr(lib, n).argtypes is not None or n == "rewl_lnu_eps", n


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    import paper_1402_2328_gb300.rewl as R
    monkeypatch.setattr(R, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(R, "_lib", None)
    with pytest.raises(R.REWLError):
        R.lib()


def test_oracle_is_not_imported_by_the_product():
    pkg = os.path.join(ROOT, "paper_1402_2328_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", src, flags=re.M), f
                assert "rewl_oracle" not in src and "librewl_oracle" not in src, f


def test_binding_argument_counts_match_header(built):
    """Every prototype's parameter count equals the ctypes binding's argtypes length."""
    import paper_1402_2328_gb300.rewl as R
    lib = R.lib()
    src = open(os.path.join(ROOT, "include", "rewl.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    protos = re.findall(r"\b(rewl_\w+)\s*\(([^)]*)\)\s*;", src)
    assert len(protos) >= 55
    for name, args in protos:
        a = " ".join(args.split())
        n = 0 if a in ("", "void") else a.count(",") + 1
        assert len(getattr(lib, name).argtypes) == n, (name, n)


def test_no_gpu_is_an_error_not_a_fallback(built):
    """Without a usable CUDA device a handle cannot be created: the call fails with an error
    (there is no CPU path behind the boundary)."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    import paper_1402_2328_gb300.rewl as R
    with pytest.raises(R.REWLError):
        R.REWL(0, 8, 2, 0.75, 1, 1e-3, 0.8)


def test_create_refuses_lnf_final_below_the_shadow_resolution(built):
    """ln f_final < 2^-32 cannot be added to the move kernel's 2^-32 fixed-point ln g: refused
    by the argument check, before any device call."""
    import paper_1402_2328_gb300.rewl as R
    lib = R.lib()
    h = ctypes.c_void_p()
    rc = lib.rewl_create(ctypes.byref(h), 0, 8, 2, 0.75, 1, 2.0 ** -33, 0.8)
    assert rc == -1 and not h.value
    assert b"invalid argument" in lib.rewl_last_error(None)


def test_equal_windows_match_the_oracle(built):
    """The library's Fig. 1a layout (a host call, no device needed) equals the oracle's."""
    import numpy as np
    import oracle as O
    import paper_1402_2328_gb300.rewl as R
    for B, h, o in [(64, 4, 0.75), (4096, 32, 0.75), (12800, 64, 0.75), (3200, 64, 0.75),
                    (1000, 7, 0.5), (257, 3, 0.6)]:
        lo, hi = R.windows_layout(B, h, o)
        olo, ohi = O.windows(B, h, o)
        assert np.array_equal(lo, olo) and np.array_equal(hi, ohi), (B, h, o)
    with pytest.raises(R.REWLError):
        R.windows_layout(16, 40, 0.75)
