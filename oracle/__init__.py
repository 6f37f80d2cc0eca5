"""CPU oracle for the SDC-resilient independent-block SZ compressor.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``. The product path (the CUDA
library and its binding) never imports this module.

``sdcsz_oracle.cpp`` restates Algorithms 1 and 2 of the paper (compression and
decompression with ABFT checks) in plain single-threaded C++; this module builds it with
g++ on first use and exposes it through ctypes with numpy arrays.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sdcsz_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# status / error codes (same meaning as the library's, defined here independently)
OK, EINVAL, ECAPACITY, EFORMAT, ESDC = 0, -1, -2, -3, -4
SITES = {"input": 1, "code": 2, "coef": 3, "pred": 4, "recon": 5, "decomp": 6}
PREDICTORS = {"auto": 0, "lorenzo": 1, "regression": 2}
ENCODINGS = {"raw": 0, "compact": 1}
DEFAULT_BLOCK = {1: 128, 2: 12, 3: 6}


class Params(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_uint32),
        ("dtype", ctypes.c_uint32),
        ("dims", ctypes.c_uint64 * 3),
        ("block", ctypes.c_uint32 * 3),
        ("eb_mode", ctypes.c_uint32),
        ("eb", ctypes.c_double),
        ("quant_bins", ctypes.c_uint32),
        ("abft", ctypes.c_uint32),
        ("predictor", ctypes.c_uint32),
        ("encoding", ctypes.c_uint32),
    ]


class Report(ctypes.Structure):
    _fields_ = [
        ("blocks", ctypes.c_uint64),
        ("regression_blocks", ctypes.c_uint64),
        ("unpredictable_points", ctypes.c_uint64),
        ("compressed_bytes", ctypes.c_uint64),
        ("input_corrected", ctypes.c_uint64),
        ("codes_corrected", ctypes.c_uint64),
        ("dup_mismatch_corrected", ctypes.c_uint64),
        ("decomp_reexec_corrected", ctypes.c_uint64),
        ("uncorrectable_blocks", ctypes.c_uint64),
        ("bound_violations", ctypes.c_uint64),
        ("eb_abs", ctypes.c_double),
        ("max_abs_err", ctypes.c_double),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class Flip(ctypes.Structure):
    _fields_ = [
        ("site", ctypes.c_uint32),
        ("bit", ctypes.c_uint32),
        ("block", ctypes.c_uint64),
        ("index", ctypes.c_uint64),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (IEEE arithmetic, no contraction)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                   "-o", tmp, _SRC]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        vp, u64, u32, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
        P, R, F = ctypes.POINTER(Params), ctypes.POINTER(Report), ctypes.POINTER(Flip)
        L.orc_compress.argtypes = [vp, P, F, i32, vp, u64, ctypes.POINTER(u64), R]
        L.orc_compress_bound.argtypes = [P, ctypes.POINTER(u64)]
        L.orc_read_header.argtypes = [vp, u64, P, ctypes.POINTER(u64)]
        L.orc_decompress.argtypes = [vp, u64, vp, vp, F, i32, R]
        L.orc_checksum_words.argtypes = [vp, u64, ctypes.POINTER(u64), ctypes.POINTER(u64)]
        L.orc_checksum_words.restype = None
        L.orc_locate_and_repair.argtypes = [vp, u64, u64, u64, u64]
        L.orc_huffman_lengths.argtypes = [vp, u32, vp]
        L.orc_huffman_lengths.restype = None
        L.orc_canonical_codes.argtypes = [vp, u32, vp]
        L.orc_canonical_codes.restype = None
        L.orc_regression.argtypes = [vp, u32, u32, vp, vp]
        L.orc_compress_block.argtypes = [vp, P, ctypes.c_double, u64, vp, vp, vp, vp, ctypes.POINTER(u64)]
        L.orc_truncate_unpredictable.argtypes = [vp, u32, ctypes.c_double, vp]
        L.orc_quantize_coefficient.argtypes = [ctypes.c_float, u32, u32, vp, ctypes.c_double, u32,
                                               ctypes.POINTER(ctypes.c_int32), vp]
        L.orc_ll_frequencies.argtypes = [vp, vp]
        L.orc_ll_frequencies.restype = None
        L.orc_ll_encode.argtypes = [vp, u32, vp, vp, u64]
        L.orc_ll_encode.restype = u64
        L.orc_ll_decode.argtypes = [vp, u64, u32, vp, vp]
        L.orc_ll_decode.restype = None
        L.orc_error_bound.argtypes = [vp, P]
        L.orc_error_bound.restype = ctypes.c_double
        L.orc_sample_mask.argtypes = [u32, vp, vp]
        L.orc_sample_mask.restype = u64
        L.orc_selection_estimates.argtypes = [vp, u32, u32, vp, vp, ctypes.POINTER(ctypes.c_float),
                                              ctypes.POINTER(ctypes.c_float)]
        L.orc_selection_estimates.restype = None
        L.orc_select_regression.argtypes = [ctypes.c_float, ctypes.c_float, u64, u32, ctypes.c_float]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def make_params(shape, dtype, eb, eb_mode="rel", block=None, bins=65536, abft=True, predictor="auto",
                encoding="raw", lossless=False) -> Params:
    ndim = len(shape)
    p = Params()
    p.ndim = ndim
    p.dtype = 0 if np.dtype(dtype) == np.float32 else 1
    for a in range(ndim):
        p.dims[a] = int(shape[a])
    if block is None:
        block = (DEFAULT_BLOCK[ndim],) * ndim
    elif isinstance(block, int):
        block = (block,) * ndim
    for a in range(ndim):
        p.block[a] = int(block[a])
    p.eb_mode = 1 if eb_mode == "rel" else 0
    p.eb = float(eb)
    p.quant_bins = int(bins)
    p.abft = 1 if abft else 0
    p.predictor = PREDICTORS[predictor]
    p.encoding = ENCODINGS[encoding] | (2 if lossless else 0)
    return p


def _flips(flips):
    if not flips:
        return None, 0
    arr = (Flip * len(flips))()
    for n, f in enumerate(flips):
        site, block, index, bit = f
        arr[n].site = SITES[site] if isinstance(site, str) else int(site)
        arr[n].block = int(block)
        arr[n].index = int(index)
        arr[n].bit = int(bit)
    return arr, len(flips)


def compress_bound(p: Params) -> int:
    out = ctypes.c_uint64()
    rc = lib().orc_compress_bound(ctypes.byref(p), ctypes.byref(out))
    if rc:
        raise ValueError(f"oracle compress_bound failed: {rc}")
    return out.value


def compress(field: np.ndarray, eb, eb_mode="rel", block=None, bins=65536, abft=True, predictor="auto",
             flips=None, encoding="raw", lossless=False):
    """Alg. 1. Returns (stream bytes as uint8 array, report dict). ``flips`` is a list of
    (site, block, index, bit) soft errors to simulate (see the site list in the C source);
    ``encoding`` is "raw" (coefficients and unpredictable values in sections of their own) or
    "compact" (both quantized / truncated and kept in the block's payload); ``lossless`` adds the
    final lossless stage (an order-0 rANS coder over everything after the block tables)."""
    field = np.ascontiguousarray(field)
    p = make_params(field.shape, field.dtype, eb, eb_mode, block, bins, abft, predictor, encoding, lossless)
    cap = compress_bound(p)
    out = np.zeros(cap, dtype=np.uint8)
    nbytes = ctypes.c_uint64()
    rep = Report()
    arr, n = _flips(flips)
    rc = lib().orc_compress(_ptr(field), ctypes.byref(p), arr, n, _ptr(out), cap, ctypes.byref(nbytes),
                            ctypes.byref(rep))
    if rc:
        raise ValueError(f"oracle compress failed: {rc}")
    return out[: nbytes.value].copy(), rep.as_dict()


def read_header(stream: np.ndarray):
    stream = np.ascontiguousarray(stream, dtype=np.uint8)
    p = Params()
    total = ctypes.c_uint64()
    rc = lib().orc_read_header(_ptr(stream), stream.size, ctypes.byref(p), ctypes.byref(total))
    if rc:
        return None
    shape = tuple(int(p.dims[a]) for a in range(p.ndim))
    return {"shape": shape, "dtype": np.float32 if p.dtype == 0 else np.float64,
            "block": tuple(int(p.block[a]) for a in range(p.ndim)), "total": total.value, "abft": bool(p.abft),
            "encoding": "compact" if p.encoding & 1 else "raw", "lossless": bool(p.encoding & 2)}


def decompress(stream: np.ndarray, flips=None):
    """Alg. 2. Returns (rc, field or None, per-block status, report dict)."""
    stream = np.ascontiguousarray(stream, dtype=np.uint8)
    h = read_header(stream)
    if h is None:
        return EFORMAT, None, None, None
    field = np.zeros(h["shape"], dtype=h["dtype"])
    nb = 1
    for n, b in zip(h["shape"], h["block"]):
        nb *= (n + b - 1) // b
    status = np.zeros(max(nb, 1), dtype=np.uint8)
    rep = Report()
    arr, n = _flips(flips)
    rc = lib().orc_decompress(_ptr(stream), stream.size, _ptr(field), _ptr(status), arr, n, ctypes.byref(rep))
    return rc, field, status[:nb], rep.as_dict()


# ---- pieces for pinning ---------------------------------------------------------------

def checksum_words(words: np.ndarray):
    w = np.ascontiguousarray(words, dtype=np.uint32)
    s, i = ctypes.c_uint64(), ctypes.c_uint64()
    lib().orc_checksum_words(_ptr(w), w.size, ctypes.byref(s), ctypes.byref(i))
    return s.value, i.value


def locate_and_repair(words: np.ndarray, sum0: int, isum0: int, maxval: int = 0xFFFFFFFF):
    w = np.ascontiguousarray(words, dtype=np.uint32).copy()
    st = lib().orc_locate_and_repair(_ptr(w), w.size, sum0 & (2**64 - 1), isum0 & (2**64 - 1), maxval)
    return st, w


def huffman_lengths(hist) -> np.ndarray:
    h = np.ascontiguousarray(hist, dtype=np.uint64)
    out = np.zeros(h.size, dtype=np.uint8)
    lib().orc_huffman_lengths(_ptr(h), h.size, _ptr(out))
    return out


def canonical_codes(lengths) -> np.ndarray:
    ln = np.ascontiguousarray(lengths, dtype=np.uint8)
    out = np.zeros(ln.size, dtype=np.uint32)
    lib().orc_canonical_codes(_ptr(ln), ln.size, _ptr(out))
    return out


def regression(block_values: np.ndarray):
    v = np.ascontiguousarray(block_values)
    ext = np.array(v.shape, dtype=np.uint32)
    coef = np.zeros(4, dtype=np.float32)
    ok = lib().orc_regression(_ptr(v), 0 if v.dtype == np.float32 else 1, v.ndim, _ptr(ext), _ptr(coef))
    return bool(ok), coef[: v.ndim + 1]


def compress_block(field: np.ndarray, eb_abs: float, b: int, block=None, bins=65536, predictor="auto",
                   encoding="raw"):
    """One block of Algorithm 1's prediction loop at a given absolute bound (no ABFT verification)."""
    field = np.ascontiguousarray(field)
    p = make_params(field.shape, field.dtype, eb_abs, "abs", block, bins, False, predictor, encoding)
    codes = np.zeros(4096, dtype=np.uint16)
    coef = np.zeros(4, dtype=field.dtype)
    is_reg = np.zeros(1, dtype=np.uint8)
    sums = np.zeros(3, dtype=np.uint64)
    npts = ctypes.c_uint64()
    rc = lib().orc_compress_block(_ptr(field), ctypes.byref(p), float(eb_abs), int(b), _ptr(codes), _ptr(coef),
                                  _ptr(is_reg), _ptr(sums), ctypes.byref(npts))
    if rc:
        raise ValueError(f"oracle compress_block failed: {rc}")
    n = npts.value
    return {"codes": codes[:n].copy(), "coef": coef[: field.ndim + 1].copy(), "regression": bool(is_reg[0]),
            "sum_q": int(sums[0]), "isum_q": int(sums[1]), "sum_dc": int(sums[2])}


def truncate_unpredictable(x, eb, dtype):
    """Compact encoding: (value an unpredictable x decompresses to, mantissa bits kept)."""
    dt = np.dtype(dtype)
    v = np.array([x], dtype=dt)
    out = np.zeros(1, dtype=dt)
    m = lib().orc_truncate_unpredictable(_ptr(v), 0 if dt == np.float32 else 1, float(eb), _ptr(out))
    return out[0], m


def quantize_coefficient(c, eb, dtype, block, a):
    """Compact encoding: (ok, integer, dequantized value) of coefficient a of a block shape."""
    dt = np.dtype(dtype)
    blk = np.ascontiguousarray(block, dtype=np.uint32)
    k = ctypes.c_int32()
    out = np.zeros(1, dtype=dt)
    ok = lib().orc_quantize_coefficient(float(np.float32(c)), 0 if dt == np.float32 else 1, blk.size, _ptr(blk),
                                        float(eb), int(a), ctypes.byref(k), _ptr(out))
    if ok < 0:
        raise ValueError("bad block shape or coefficient index")
    return bool(ok), int(k.value), out[0]


def ll_frequencies(counts) -> np.ndarray:
    """Lossless stage: the 12-bit frequencies of a 256-bin byte histogram."""
    c = np.ascontiguousarray(counts, dtype=np.uint64)
    f = np.zeros(256, dtype=np.uint16)
    lib().orc_ll_frequencies(_ptr(c), _ptr(f))
    return f


def ll_encode(data, freqs) -> np.ndarray:
    """Lossless stage: one chunk (at most 16384 bytes) coded with the given frequencies."""
    d = np.ascontiguousarray(data, dtype=np.uint8)
    f = np.ascontiguousarray(freqs, dtype=np.uint16)
    out = np.zeros(128 + 2 * d.size + 4, dtype=np.uint8)
    n = lib().orc_ll_encode(_ptr(d), d.size, _ptr(f), _ptr(out), out.size)
    return out[:n].copy()


def ll_decode(chunk, n, freqs) -> np.ndarray:
    c = np.ascontiguousarray(chunk, dtype=np.uint8)
    f = np.ascontiguousarray(freqs, dtype=np.uint16)
    out = np.zeros(n, dtype=np.uint8)
    lib().orc_ll_decode(_ptr(c), c.size, n, _ptr(f), _ptr(out))
    return out


def sample_mask(ext) -> np.ndarray:
    """Sample membership (1 = in the selection sample) of every point of a block of extents ext."""
    ext = [int(e) for e in ext]
    e = np.array(ext, dtype=np.uint32)
    m = np.zeros(int(np.prod(ext)), dtype=np.uint8)
    n = lib().orc_sample_mask(len(ext), _ptr(e), _ptr(m))
    assert n == int(m.sum()), "sample count disagrees with the mask"
    return m.reshape(ext)


def selection_estimates(block_values: np.ndarray, coef):
    """(E_reg, E_lor) of one block for the given fp32 coefficients (b_0..b_ndim)."""
    v = np.ascontiguousarray(block_values)
    e = np.array(v.shape, dtype=np.uint32)
    c = np.zeros(4, dtype=np.float32)
    c[: len(coef)] = coef
    er, el = ctypes.c_float(), ctypes.c_float()
    lib().orc_selection_estimates(_ptr(v), 0 if v.dtype == np.float32 else 1, v.ndim, _ptr(e), _ptr(c),
                                  ctypes.byref(er), ctypes.byref(el))
    return er.value, el.value


def select_regression(Ereg, Elor, S, ndim, eb) -> bool:
    """Algorithm 1's indicator for the given estimates: True = regression."""
    return bool(lib().orc_select_regression(Ereg, Elor, S, ndim, eb))


def error_bound(field: np.ndarray, eb, eb_mode="rel") -> float:
    field = np.ascontiguousarray(field)
    p = make_params(field.shape, field.dtype, eb, eb_mode)
    return lib().orc_error_bound(_ptr(field), ctypes.byref(p))
