"""Launch-shape autotuning (binding of ``lbm_autotune`` and
``lbm_batch_autotune``; the timing, candidate lists and the cache live in
the library).

Single lattices: x-dominant thread-block shapes (Sec. 6 of the paper) of the
current kernel variant. Batches: tile size and blocks per SM of the
persistent kernel. Each candidate is timed with CUDA events on the handle's
stream; the winner is applied to the handle and kept in a text cache keyed
by GPU and problem.

Tuning advances the state it runs on: tune before initialising the state
you want to keep (or re-initialise afterwards).
"""

from __future__ import annotations

import ctypes
import os

from . import capi

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "lbm_gb300_autotune.txt")


def _path(cache_path):
    if not cache_path:
        return None
    os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
    return os.fsencode(cache_path)


def tune_lattice(L, steps=20, cache_path=DEFAULT_CACHE):
    """Pick the fastest block shape for lattice ``L``; returns
    (bx, by, ms per step)."""
    a, b, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
    capi.call("lbm_autotune", L.handle, _path(cache_path), int(steps), ctypes.byref(a),
              ctypes.byref(b), ctypes.byref(ms))
    return a.value, b.value, ms.value


def tune_batch(B, steps=50, cache_path=DEFAULT_CACHE):
    """Pick the fastest (threads, blocks_per_sm) for the persistent batched
    kernel; returns (threads, blocks_per_sm, ms per step)."""
    a, b, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
    capi.call("lbm_batch_autotune", B.handle, _path(cache_path), int(steps), ctypes.byref(a),
              ctypes.byref(b), ctypes.byref(ms))
    return a.value, b.value, ms.value
