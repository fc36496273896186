"""Block-shape autotuner with a JSON cache.

Single lattices: thread-block shapes (bx along x, by rows) for the node
kernels, kept x-dominant as in Sec. 6 of the paper, timed with CUDA events
over a few steps. Batches: tile size (threads per block) and blocks per SM
of the persistent kernel, timed over whole persistent launches. The winner
is applied to the handle and stored in the cache keyed by problem and GPU.

Tuning advances the state of the lattice it runs on; tune before
initialising the state you want to keep (or re-initialise afterwards).
"""

from __future__ import annotations

import hashlib
import json
import os
import time

import torch

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "lbm_gb300_autotune.json")


def _load(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except Exception:
        return {}


def _store(path, data):
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = f"{path}.tmp{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump(data, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass


def _gpu_name(device):
    return torch.cuda.get_device_name(device).replace(" ", "_")


def lattice_candidates(nx):
    out = []
    for bx in (32, 64, 128, 256):
        if bx > max(32, -(-nx // 32) * 32):
            continue
        for by in (1, 2, 4, 8):
            if bx * by <= 256 and bx * by >= 64:
                out.append((bx, by))
    return out or [(32, 1)]


def tune_lattice(L, steps=20, cache_path=DEFAULT_CACHE, candidates=None, use_cache=True):
    """Pick the fastest (bx, by) for lattice ``L``; returns (bx, by, ms)."""
    key = (f"lattice:{_gpu_name(L.device)}:{L.nx}x{L.ny}x{L.nz}:{L.storage}:"
           f"flags{L.flags}")
    cache = _load(cache_path) if cache_path else {}
    if use_cache and key in cache:
        bx, by = cache[key]["block"]
        L.set_block(bx, by)
        return bx, by, cache[key]["ms"]
    best = None
    s = L.stream
    for (bx, by) in candidates or lattice_candidates(L.nx):
        L.set_block(bx, by)
        L.step(2)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        L.step(steps)
        e1.record(s)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
        if best is None or ms < best[2]:
            best = (bx, by, ms)
    L.set_block(best[0], best[1])
    if cache_path:
        cache[key] = {"block": [best[0], best[1]], "ms": best[2]}
        _store(cache_path, cache)
    return best


def batch_candidates():
    return [(t, b) for t in (64, 128, 256) for b in (0, 2, 4, 6, 8)]


def tune_batch(B, steps=50, cache_path=DEFAULT_CACHE, candidates=None, use_cache=True,
               table=None):
    """Pick the fastest (threads, blocks_per_sm) for the persistent batched
    kernel; returns (threads, blocks_per_sm, ms per step). ``table``, if a
    dict, receives every candidate's time."""
    sig = ",".join(f"{a}x{b}x{c}" for a, b, c in B.dims.tolist())
    key = f"batch:{_gpu_name(B.device)}:{B.ndom}:{hashlib.sha256(sig.encode()).hexdigest()[:12]}"
    cache = _load(cache_path) if cache_path else {}
    if use_cache and key in cache:
        t, b = cache[key]["tiling"]
        B.set_tiling(t, b)
        return t, b, cache[key]["ms"]
    best = None
    for (t, b) in candidates or batch_candidates():
        B.set_tiling(t, b)
        B.step(2)
        t0 = time.perf_counter()
        B.step(steps)
        ms = (time.perf_counter() - t0) * 1e3 / steps
        if table is not None:
            table[(t, b)] = ms
        if best is None or ms < best[2]:
            best = (t, b, ms)
    B.set_tiling(best[0], best[1])
    if cache_path:
        cache[key] = {"tiling": [best[0], best[1]], "ms": best[2]}
        _store(cache_path, cache)
    return best
