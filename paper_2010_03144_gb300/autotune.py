"""Block-size autotuning with a persistent cache.

The measurement is the library's own (``sdcsz_autotune_block``: CUDA-event timing of the
compressor on a leading slab of the field, one run per candidate edge); the choice is the
fastest edge whose compressed size is within ``size_slack`` (default 10%) of the smallest. This module only keys
and stores the choices, so a later field of the same class skips the measurement. The class
of a field is (dtype, dimensionality, size decade, error-bound decade, bound mode, ABFT).
"""

from __future__ import annotations

import ctypes
import json
import math
import os
import threading

CANDIDATES = {3: (4, 6, 8, 10, 12, 16), 2: (8, 12, 16), 1: (64, 128, 256)}
_lock = threading.Lock()


def field_class(shape, dtype, eb, eb_mode="rel", abft=True) -> str:
    n = 1
    for v in shape:
        n *= int(v)
    dt = "f64" if ("float64" in str(dtype) or "double" in str(dtype)) else "f32"
    return (f"{dt}/{len(shape)}d/n1e{int(math.floor(math.log10(max(n, 1))))}/"
            f"eb1e{int(math.floor(math.log10(eb) + 1e-9))}/{eb_mode}/{'abft' if abft else 'plain'}")


def measure(field, eb, eb_mode="rel", candidates=None, sample_points=1 << 26, size_slack=0.10, abft=True,
            stream=None):
    """Run the library's tuner on ``field``; returns (best edge, [per-candidate dicts])."""
    from . import SdcszError, TuneResult, _stream_handle, lib, make_params
    cands = tuple(candidates or CANDIDATES[field.dim()])
    p = make_params(tuple(field.shape), field.dtype, eb, eb_mode, None, 65536, abft, "auto")
    arr = (ctypes.c_uint32 * len(cands))(*cands)
    res = (TuneResult * len(cands))()
    best = ctypes.c_uint32()
    rc = lib().sdcsz_autotune_block(ctypes.c_void_p(field.data_ptr()), ctypes.byref(p), arr, len(cands),
                                    sample_points, size_slack, _stream_handle(stream), res, ctypes.byref(best))
    if rc:
        raise SdcszError(rc, "autotune_block")
    rows = [{"block": r.block, "ms": r.ms, "bytes": r.bytes, "gbs": r.gbs, "ratio": r.ratio} for r in res]
    return cands[best.value], rows


class Tuner:
    """Cached block-size choices, stored as JSON at ``path`` (None: in memory only)."""

    def __init__(self, path: str | None = None):
        self.path = path
        self.cache = {}
        if path and os.path.exists(path):
            with open(path) as f:
                self.cache = json.load(f)

    def block_for(self, field, eb, eb_mode="rel", abft=True, stream=None) -> int:
        key = field_class(tuple(field.shape), field.dtype, eb, eb_mode, abft)
        with _lock:
            hit = self.cache.get(key)
        if hit is not None:
            return int(hit["block"])
        best, rows = measure(field, eb, eb_mode, abft=abft, stream=stream)
        with _lock:
            self.cache[key] = {"block": best, "candidates": rows}
            if self.path:
                tmp = self.path + ".tmp"
                with open(tmp, "w") as f:
                    json.dump(self.cache, f, indent=1, sort_keys=True)
                os.replace(tmp, self.path)
        return best
