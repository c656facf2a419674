"""GB300 (sm_103a) replica-exchange Wang-Landau sampling (arXiv:1402.2328).

The hot path (WL moves, flatness test, window advance, replica exchange, joining) runs
in hand-written CUDA kernels behind the C ABI of include/rewl.h; ``rewl`` is its thin
ctypes binding.
"""
from .rewl import REWL, REWLBatch, REWLError, lib, replay  # noqa: F401
