"""Python binding of libsdcsz: SDC-resilient error-bounded lossy compression on GB300.

Thin ctypes marshalling over the C ABI of ``include/sdcsz.h`` (same function names without
the ``sdcsz_`` prefix). PyTorch provides device memory and the current CUDA stream; every
step of compression and decompression runs in the library's CUDA kernels. There is no CPU
fallback: if ``libsdcsz.so`` is missing or CUDA is unavailable the calls raise.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsdcsz.so")

OK, EINVAL, ECAPACITY, EFORMAT, ESDC, ETIMEOUT, ECUDA = 0, -1, -2, -3, -4, -5, -6
SITES = {"input": 1, "code": 2, "coef": 3, "pred": 4, "recon": 5, "decomp": 6, "rewalk": 7}
PREDICTORS = {"auto": 0, "lorenzo": 1, "regression": 2}
ENCODINGS = {"raw": 0, "compact": 1}
BLOCK_OK, BLOCK_CORRECTED, BLOCK_SDC, BLOCK_BAD = 0, 1, 2, 3

# Symbols the header declares (checked by tests against the shared object's exports).
EXPORTS = ("sdcsz_compress_bound", "sdcsz_workspace_size", "sdcsz_decompress_workspace_size", "sdcsz_compress",
           "sdcsz_decompress", "sdcsz_verify", "sdcsz_read_header", "sdcsz_strerror",
           "sdcsz_debug_compress_flips", "sdcsz_debug_decompress_flips", "sdcsz_compress_traced",
           "sdcsz_decompress_traced", "sdcsz_trace_begin", "sdcsz_trace_end", "sdcsz_compress_noalloc", "sdcsz_kernel_launches", "sdcsz_batch_create",
           "sdcsz_batch_workspace_size", "sdcsz_batch_bind", "sdcsz_batch_set_fields", "sdcsz_batch_compress",
           "sdcsz_batch_capture", "sdcsz_batch_launch", "sdcsz_batch_results", "sdcsz_batch_destroy",
           "sdcsz_autotune_block", "sdcsz_server_create", "sdcsz_server_submit", "sdcsz_server_poll",
           "sdcsz_server_release", "sdcsz_server_get_stats", "sdcsz_server_destroy", "sdcsz_decompress_region",
           "sdcsz_decompress_workspace_size_for", "sdcsz_shard_workspace_size", "sdcsz_shard_prep",
           "sdcsz_shard_predict", "sdcsz_shard_encode", "sdcsz_shard_assemble")


class SdcszError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})")


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


OP_COMPRESS, OP_DECOMPRESS, OP_VERIFY = 1, 2, 3


class ServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_uint64), ("slots", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class Request(ctypes.Structure):
    _fields_ = [
        ("op", ctypes.c_uint32),
        ("reserved", ctypes.c_uint32),
        ("id", ctypes.c_uint64),
        ("d_in", ctypes.c_void_p),
        ("in_bytes", ctypes.c_size_t),
        ("params", Params),
        ("d_out", ctypes.c_void_p),
        ("out_cap", ctypes.c_size_t),
        ("d_original", ctypes.c_void_p),
        ("d_flips", ctypes.c_void_p),
        ("n_flips", ctypes.c_size_t),
    ]


class Completion(ctypes.Structure):
    _fields_ = [
        ("id", ctypes.c_uint64),
        ("op", ctypes.c_uint32),
        ("status", ctypes.c_int),
        ("d_result", ctypes.c_void_p),
        ("result_bytes", ctypes.c_size_t),
        ("report", Report),
        ("t_submit", ctypes.c_double),
        ("t_admit", ctypes.c_double),
        ("t_done", ctypes.c_double),
    ]


class ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("pending", "in_flight", "admitted", "completed", "bytes_in_use",
                                               "peak_bytes")]


class TuneResult(ctypes.Structure):
    _fields_ = [
        ("block", ctypes.c_uint32),
        ("ms", ctypes.c_double),
        ("bytes", ctypes.c_uint64),
        ("gbs", ctypes.c_double),
        ("ratio", ctypes.c_double),
    ]


class BatchItem(ctypes.Structure):
    _fields_ = [
        ("d_field", ctypes.c_void_p),
        ("params", Params),
        ("d_out", ctypes.c_void_p),
        ("out_cap", ctypes.c_size_t),
    ]


class Flip(ctypes.Structure):
    _fields_ = [("site", ctypes.c_uint32), ("bit", ctypes.c_uint32), ("block", ctypes.c_uint64),
                ("index", ctypes.c_uint64)]


_lib = None


def lib():
    """The loaded shared library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libsdcsz.so is not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, sz, i32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int
        P, R = ctypes.POINTER(Params), ctypes.POINTER(Report)
        L.sdcsz_compress_bound.argtypes = [P, ctypes.POINTER(sz)]
        L.sdcsz_workspace_size.argtypes = [P, ctypes.POINTER(sz)]
        L.sdcsz_decompress_workspace_size.argtypes = []
        L.sdcsz_decompress_workspace_size.restype = sz
        L.sdcsz_compress.argtypes = [vp, P, vp, sz, ctypes.POINTER(sz), vp, sz, R, vp]
        L.sdcsz_debug_compress_flips.argtypes = [vp, P, vp, sz, ctypes.POINTER(sz), vp, sz, R, vp, vp, sz]
        L.sdcsz_decompress.argtypes = [vp, sz, vp, sz, vp, vp, sz, R, vp]
        L.sdcsz_debug_decompress_flips.argtypes = [vp, sz, vp, sz, vp, vp, sz, R, vp, vp, sz]
        L.sdcsz_verify.argtypes = [vp, sz, vp, vp, vp, sz, R, vp]
        fp = ctypes.POINTER(ctypes.c_float)
        L.sdcsz_compress_traced.argtypes = [vp, P, vp, sz, ctypes.POINTER(sz), vp, sz, R, vp, fp]
        L.sdcsz_decompress_traced.argtypes = [vp, sz, vp, sz, vp, vp, sz, R, vp, fp]
        L.sdcsz_compress_traced.restype = i32
        L.sdcsz_compress_noalloc.argtypes = [vp, P, vp, sz, ctypes.POINTER(sz), R, vp]
        L.sdcsz_compress_noalloc.restype = i32
        L.sdcsz_decompress_traced.restype = i32
        L.sdcsz_read_header.argtypes = [vp, sz, P, ctypes.POINTER(ctypes.c_uint64)]
        L.sdcsz_strerror.argtypes = [i32]
        L.sdcsz_strerror.restype = ctypes.c_char_p
        u64p = ctypes.POINTER(ctypes.c_uint64)
        L.sdcsz_decompress_region.argtypes = [vp, sz, u64p, u64p, vp, sz, vp, vp, sz, R, vp]
        L.sdcsz_decompress_region.restype = i32
        L.sdcsz_decompress_workspace_size_for.argtypes = [vp, sz, ctypes.POINTER(sz)]
        L.sdcsz_decompress_workspace_size_for.restype = i32
        L.sdcsz_trace_begin.argtypes = [sz]
        L.sdcsz_trace_begin.restype = i32
        L.sdcsz_trace_end.argtypes = [ctypes.POINTER(ctypes.c_int32), fp, sz, ctypes.POINTER(sz)]
        L.sdcsz_trace_end.restype = i32
        L.sdcsz_kernel_launches.argtypes = []
        L.sdcsz_kernel_launches.restype = ctypes.c_ulonglong
        u64, u64a = ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)
        L.sdcsz_shard_workspace_size.argtypes = [P, u64, u64, ctypes.POINTER(sz)]
        L.sdcsz_shard_prep.argtypes = [vp, P, u64, u64, vp, sz, u64a, vp]
        L.sdcsz_shard_predict.argtypes = [vp, P, u64, u64, vp, sz, u64a, u64a, ctypes.POINTER(ctypes.c_void_p), vp]
        L.sdcsz_shard_encode.argtypes = [P, u64, u64, vp, sz, u64a, i32, vp, sz, u64a, vp]
        L.sdcsz_shard_assemble.argtypes = [P, u64, u64, vp, sz, u64a, u64a, i32, vp, sz, ctypes.POINTER(sz), R, vp]
        for f in ("sdcsz_shard_workspace_size", "sdcsz_shard_prep", "sdcsz_shard_predict", "sdcsz_shard_encode",
                  "sdcsz_shard_assemble"):
            getattr(L, f).restype = i32
        BI, BP = ctypes.POINTER(BatchItem), ctypes.c_void_p
        L.sdcsz_batch_create.argtypes = [BI, ctypes.c_uint32, ctypes.POINTER(BP)]
        L.sdcsz_batch_workspace_size.argtypes = [BP, ctypes.POINTER(sz)]
        L.sdcsz_batch_bind.argtypes = [BP, vp, sz, vp]
        L.sdcsz_batch_set_fields.argtypes = [BP, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(sz), vp]
        L.sdcsz_batch_compress.argtypes = [BP, vp]
        L.sdcsz_batch_capture.argtypes = [BP, vp]
        L.sdcsz_batch_launch.argtypes = [BP, vp]
        L.sdcsz_batch_results.argtypes = [BP, ctypes.POINTER(sz), R, vp]
        L.sdcsz_autotune_block.argtypes = [vp, P, ctypes.POINTER(ctypes.c_uint32), ctypes.c_uint32,
                                           ctypes.c_uint64, ctypes.c_double, vp, ctypes.POINTER(TuneResult),
                                           ctypes.POINTER(ctypes.c_uint32)]
        L.sdcsz_autotune_block.restype = i32
        SP = ctypes.c_void_p
        L.sdcsz_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(SP)]
        L.sdcsz_server_submit.argtypes = [SP, ctypes.POINTER(Request)]
        L.sdcsz_server_poll.argtypes = [SP, ctypes.POINTER(Completion), ctypes.c_uint32,
                                        ctypes.POINTER(ctypes.c_uint32), ctypes.c_uint32]
        L.sdcsz_server_release.argtypes = [SP, ctypes.c_uint64]
        L.sdcsz_server_get_stats.argtypes = [SP, ctypes.POINTER(ServerStats)]
        L.sdcsz_server_destroy.argtypes = [SP]
        L.sdcsz_server_destroy.restype = None
        for f in (L.sdcsz_server_create, L.sdcsz_server_submit, L.sdcsz_server_poll, L.sdcsz_server_release,
                  L.sdcsz_server_get_stats):
            f.restype = i32
        L.sdcsz_batch_destroy.argtypes = [BP]
        L.sdcsz_batch_destroy.restype = None
        for f in (L.sdcsz_batch_create, L.sdcsz_batch_workspace_size, L.sdcsz_batch_bind, L.sdcsz_batch_set_fields,
                  L.sdcsz_batch_compress, L.sdcsz_batch_capture, L.sdcsz_batch_launch, L.sdcsz_batch_results):
            f.restype = i32
        for f in (L.sdcsz_compress_bound, L.sdcsz_workspace_size, L.sdcsz_compress, L.sdcsz_debug_compress_flips,
                  L.sdcsz_decompress, L.sdcsz_debug_decompress_flips, L.sdcsz_verify, L.sdcsz_read_header):
            f.restype = i32
        _lib = L
    return _lib


def kernel_launches() -> int:
    """Kernels launched by the library in this process so far."""
    return int(lib().sdcsz_kernel_launches())


def strerror(code: int) -> str:
    return lib().sdcsz_strerror(int(code)).decode()


def make_params(shape, dtype, eb, eb_mode="rel", block=None, bins=65536, abft=True, predictor="auto",
                encoding="raw", lossless=False) -> Params:
    import torch
    ndim = len(shape)
    p = Params()
    p.ndim = ndim
    if dtype in (torch.float32, np.float32, "float32"):
        p.dtype = 0
    elif dtype in (torch.float64, np.float64, "float64"):
        p.dtype = 1
    else:
        raise ValueError(f"unsupported dtype {dtype}")
    for a in range(ndim):
        p.dims[a] = int(shape[a])
    if block is not None:
        if isinstance(block, int):
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


def compress_bound(p: Params) -> int:
    out = ctypes.c_size_t()
    rc = lib().sdcsz_compress_bound(ctypes.byref(p), ctypes.byref(out))
    if rc:
        raise SdcszError(rc, "compress_bound")
    return out.value


def workspace_size(p: Params) -> int:
    out = ctypes.c_size_t()
    rc = lib().sdcsz_workspace_size(ctypes.byref(p), ctypes.byref(out))
    if rc:
        raise SdcszError(rc, "workspace_size")
    return out.value


def decompress_workspace_size(stream=None) -> int:
    """Decompression workspace bytes: for any stream without the lossless stage, or for the
    given stream (a uint8 CUDA tensor or host bytes)."""
    if stream is None:
        return int(lib().sdcsz_decompress_workspace_size())
    import torch
    n = stream.numel() if isinstance(stream, torch.Tensor) else len(stream)
    hb = (stream[:128].cpu().numpy() if isinstance(stream, torch.Tensor) else np.frombuffer(bytes(stream[:128]),
                                                                                                dtype=np.uint8))
    buf = np.zeros(128, dtype=np.uint8)
    buf[: hb.size] = hb
    out = ctypes.c_size_t()
    rc = lib().sdcsz_decompress_workspace_size_for(buf.ctypes.data_as(ctypes.c_void_p), n, ctypes.byref(out))
    if rc:
        raise SdcszError(rc, "decompress_workspace_size_for")
    return int(out.value)


def _stream_handle(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def flips_tensor(flips, device):
    """Device array of flip records sorted by (block, site, index)."""
    import torch
    recs = []
    for site, block, index, bit in flips:
        recs.append((SITES[site] if isinstance(site, str) else int(site), int(bit), int(block), int(index)))
    recs.sort(key=lambda r: (r[2], r[0], r[3]))
    arr = np.zeros(len(recs), dtype=np.dtype([("site", "<u4"), ("bit", "<u4"), ("block", "<u8"), ("index", "<u8")]))
    for n, r in enumerate(recs):
        arr[n] = r
    return torch.from_numpy(arr.view(np.uint8).copy()).to(device)


class Workspace:
    """Reusable device buffers for repeated calls with one parameter set."""

    def __init__(self, p: Params, device):
        import torch
        self.p = p
        self.cap = compress_bound(p)
        self.out = torch.empty(self.cap, dtype=torch.uint8, device=device)
        self.ws = torch.empty(workspace_size(p), dtype=torch.uint8, device=device)


def compress(field, eb, eb_mode="rel", block=None, bins=65536, abft=True, predictor="auto", flips=None,
             workspace: Workspace | None = None, stream=None, sync=True, encoding="raw", lossless=False):
    """Compress a CUDA tensor (float32/float64, 1-3 dims, contiguous). Returns
    (stream bytes as a uint8 CUDA tensor view, report dict or None). ``encoding`` "compact"
    keeps the regression coefficients as bound-relative integers and the unpredictable values
    truncated to the bits the bound needs, both inside the block payloads; ``lossless`` adds the
    final lossless stage (an order-0 rANS coder over everything after the block tables)."""
    import torch
    if not field.is_cuda or not field.is_contiguous():
        raise ValueError("field must be a contiguous CUDA tensor")
    p = make_params(tuple(field.shape), field.dtype, eb, eb_mode, block, bins, abft, predictor, encoding, lossless)
    if workspace is not None and workspace.p.encoding != p.encoding:
        raise ValueError("workspace was sized for another encoding")
    w = workspace if workspace is not None else Workspace(p, field.device)
    rep = Report()
    nbytes = ctypes.c_size_t()
    h = _stream_handle(stream)
    if flips:
        ft = flips_tensor(flips, field.device)
        rc = lib().sdcsz_debug_compress_flips(ctypes.c_void_p(field.data_ptr()), ctypes.byref(p),
                                              ctypes.c_void_p(w.out.data_ptr()), w.cap, ctypes.byref(nbytes),
                                              ctypes.c_void_p(w.ws.data_ptr()), w.ws.numel(), ctypes.byref(rep), h,
                                              ctypes.c_void_p(ft.data_ptr()), len(flips))
    elif sync:
        rc = lib().sdcsz_compress(ctypes.c_void_p(field.data_ptr()), ctypes.byref(p), ctypes.c_void_p(w.out.data_ptr()),
                                  w.cap, ctypes.byref(nbytes), ctypes.c_void_p(w.ws.data_ptr()), w.ws.numel(),
                                  ctypes.byref(rep), h)
    else:
        rc = lib().sdcsz_compress(ctypes.c_void_p(field.data_ptr()), ctypes.byref(p), ctypes.c_void_p(w.out.data_ptr()),
                                  w.cap, None, ctypes.c_void_p(w.ws.data_ptr()), w.ws.numel(), None, h)
        if rc:
            raise SdcszError(rc, "compress")
        return w.out, None
    if rc:
        raise SdcszError(rc, "compress")
    return w.out[: nbytes.value], rep.as_dict()


def read_header(stream_bytes):
    """Parse a stream header from host bytes (numpy uint8 or bytes)."""
    b = np.ascontiguousarray(np.frombuffer(bytes(stream_bytes), dtype=np.uint8) if isinstance(stream_bytes, (bytes, bytearray))
                             else stream_bytes, dtype=np.uint8)
    p = Params()
    total = ctypes.c_uint64()
    rc = lib().sdcsz_read_header(b.ctypes.data_as(ctypes.c_void_p), b.size, ctypes.byref(p), ctypes.byref(total))
    if rc:
        raise SdcszError(rc, "read_header")
    shape = tuple(int(p.dims[a]) for a in range(p.ndim))
    block = tuple(int(p.block[a]) for a in range(p.ndim))
    return {"shape": shape, "dtype": "float32" if p.dtype == 0 else "float64", "block": block,
            "total": int(total.value), "abft": bool(p.abft), "bins": int(p.quant_bins),
            "encoding": "compact" if p.encoding & 1 else "raw", "lossless": bool(p.encoding & 2)}


def _geometry(stream):
    import torch
    hb = stream[:128].cpu().numpy()
    h = read_header_partial(hb, stream.numel())
    nb = 1
    for n, b in zip(h["shape"], h["block"]):
        nb *= (n + b - 1) // b
    dt = torch.float32 if h["dtype"] == "float32" else torch.float64
    return h, nb, dt


def read_header_partial(header_bytes: np.ndarray, nbytes: int):
    """Header parse when only the first 128 bytes are on the host."""
    b = np.ascontiguousarray(header_bytes, dtype=np.uint8)
    p = Params()
    total = ctypes.c_uint64()
    buf = np.zeros(max(128, b.size), dtype=np.uint8)
    buf[: b.size] = b
    rc = lib().sdcsz_read_header(buf.ctypes.data_as(ctypes.c_void_p), int(nbytes), ctypes.byref(p),
                                 ctypes.byref(total))
    if rc:
        raise SdcszError(rc, "read_header")
    return {"shape": tuple(int(p.dims[a]) for a in range(p.ndim)), "dtype": "float32" if p.dtype == 0 else "float64",
            "block": tuple(int(p.block[a]) for a in range(p.ndim)), "total": int(total.value)}


def decompress(stream, out=None, status=None, flips=None, ws=None, cuda_stream=None, report=True):
    """Decompress a uint8 CUDA tensor holding a stream. Returns (rc, field, block status, report dict).
    rc is 0 or ESDC (blocks that failed twice are named in the status); other errors raise.
    When out, status and ws are all given (status holding a byte per block), the binding reads
    nothing from the device itself and returns status whole."""
    import torch
    if out is not None and status is not None and ws is not None:
        nb, dt = status.numel(), out.dtype
    else:
        h, nb, dt = _geometry(stream)
    field = out if out is not None else torch.empty(h["shape"], dtype=dt, device=stream.device)
    st = status if status is not None else torch.empty(max(nb, 1), dtype=torch.uint8, device=stream.device)
    w = ws if ws is not None else torch.empty(decompress_workspace_size(stream), dtype=torch.uint8, device=stream.device)
    rep = Report()
    hs = _stream_handle(cuda_stream)
    args = [ctypes.c_void_p(stream.data_ptr()), stream.numel(), ctypes.c_void_p(field.data_ptr()),
            field.numel() * field.element_size(), ctypes.c_void_p(st.data_ptr()), ctypes.c_void_p(w.data_ptr()),
            w.numel(), ctypes.byref(rep) if report else None, hs]
    if flips:
        ft = flips_tensor(flips, stream.device)
        rc = lib().sdcsz_debug_decompress_flips(*args, ctypes.c_void_p(ft.data_ptr()), len(flips))
    else:
        rc = lib().sdcsz_decompress(*args)
    if rc not in (OK, ESDC):
        raise SdcszError(rc, "decompress")
    return rc, field, st[:nb], (rep.as_dict() if report else None)


def region_blocks(shape, block, lo, hi) -> int:
    """Blocks intersecting the box [lo, hi) of a field with this shape and block size."""
    n = 1
    for a in range(len(shape)):
        n *= (hi[a] - 1) // block[a] - lo[a] // block[a] + 1
    return n


def decompress_region(stream, lo, hi, out=None, status=None, ws=None, cuda_stream=None, report=True):
    """Decode only the blocks that intersect the box [lo, hi) (element coordinates, the
    field's axis order). Returns (rc, box tensor, per-block status, report dict or None)."""
    import torch
    h, nb, dt = _geometry(stream)
    lo, hi = [int(v) for v in lo], [int(v) for v in hi]
    box = tuple(max(b - a, 0) for a, b in zip(lo, hi))  # an empty box is rejected by the library
    res = out if out is not None else torch.empty(box, dtype=dt, device=stream.device)
    nblk = region_blocks(h["shape"], h["block"], lo, hi) if all(b > a for a, b in zip(lo, hi)) else 1
    if status is not None and status.numel() < nblk:
        raise SdcszError(ECAPACITY, "decompress_region status")
    st = status if status is not None else torch.empty(max(nblk, 1), dtype=torch.uint8, device=stream.device)
    w = ws if ws is not None else torch.empty(decompress_workspace_size(stream), dtype=torch.uint8, device=stream.device)
    rep = Report()
    lo_a = (ctypes.c_uint64 * 3)(*(lo + [0] * (3 - len(lo))))
    hi_a = (ctypes.c_uint64 * 3)(*(hi + [0] * (3 - len(hi))))
    rc = lib().sdcsz_decompress_region(ctypes.c_void_p(stream.data_ptr()), stream.numel(), lo_a, hi_a,
                                       ctypes.c_void_p(res.data_ptr()), res.numel() * res.element_size(),
                                       ctypes.c_void_p(st.data_ptr()), ctypes.c_void_p(w.data_ptr()), w.numel(),
                                       ctypes.byref(rep) if report else None, _stream_handle(cuda_stream))
    if rc not in (OK, ESDC):
        raise SdcszError(rc, "decompress_region")
    return rc, res, st[:nblk], (rep.as_dict() if report else None)


def verify(stream, original=None, status=None, ws=None, cuda_stream=None):
    """Alg. 2 checks without writing a field; with ``original`` also the bound on every point.
    Returns (rc, block status, report dict)."""
    import torch
    h, nb, dt = _geometry(stream)
    st = status if status is not None else torch.empty(max(nb, 1), dtype=torch.uint8, device=stream.device)
    w = ws if ws is not None else torch.empty(decompress_workspace_size(stream), dtype=torch.uint8, device=stream.device)
    rep = Report()
    orig = ctypes.c_void_p(original.data_ptr()) if original is not None else None
    rc = lib().sdcsz_verify(ctypes.c_void_p(stream.data_ptr()), stream.numel(), orig, ctypes.c_void_p(st.data_ptr()),
                            ctypes.c_void_p(w.data_ptr()), w.numel(), ctypes.byref(rep), _stream_handle(cuda_stream))
    if rc not in (OK, ESDC):
        raise SdcszError(rc, "verify")
    return rc, st[:nb], rep.as_dict()


def compress_traced(field, p: Params, workspace: Workspace, stream=None):
    """Compress with per-stage CUDA-event timing. Returns (nbytes, stage milliseconds[5])."""
    ms = (ctypes.c_float * 5)()
    nbytes = ctypes.c_size_t()
    rc = lib().sdcsz_compress_traced(ctypes.c_void_p(field.data_ptr()), ctypes.byref(p),
                                     ctypes.c_void_p(workspace.out.data_ptr()), workspace.cap, ctypes.byref(nbytes),
                                     ctypes.c_void_p(workspace.ws.data_ptr()), workspace.ws.numel(), None,
                                     _stream_handle(stream), ms)
    if rc:
        raise SdcszError(rc, "compress_traced")
    return nbytes.value, list(ms)


def decompress_traced(stream_t, out, ws, stream=None):
    """Decompress with CUDA-event timing of the decode kernel. Returns milliseconds."""
    ms = (ctypes.c_float * 1)()
    rc = lib().sdcsz_decompress_traced(ctypes.c_void_p(stream_t.data_ptr()), stream_t.numel(),
                                       ctypes.c_void_p(out.data_ptr()), out.numel() * out.element_size(), None,
                                       ctypes.c_void_p(ws.data_ptr()), ws.numel(), None, _stream_handle(stream), ms)
    if rc not in (OK,):
        raise SdcszError(rc, "decompress_traced")
    return ms[0]


def trace_begin(max_calls: int):
    """Open the deferred stage recorder: the next compress/decompress/verify calls (up to
    max_calls) record stage events without a host wait."""
    rc = lib().sdcsz_trace_begin(int(max_calls))
    if rc:
        raise SdcszError(rc, "trace_begin")


def trace_end(max_calls: int):
    """Wait for the recorded events and close the recorder. Returns a list of
    (kind, stage milliseconds) per call, kind "compress" (reset, K1, K2, K3, K4),
    "decompress" or "verify" (K5)."""
    kinds = (ctypes.c_int32 * max(1, max_calls))()
    ms = (ctypes.c_float * (5 * max(1, max_calls)))()
    n = ctypes.c_size_t()
    rc = lib().sdcsz_trace_end(kinds, ms, int(max_calls), ctypes.byref(n))
    if rc:
        raise SdcszError(rc, "trace_end")
    names = ("compress", "decompress", "verify")
    return [(names[kinds[c]], [ms[5 * c + q] for q in range(5)]) for c in range(n.value)]


def compress_noalloc(field, out, eb, eb_mode="rel", block=None, bins=65536, abft=True, predictor="auto",
                     stream=None, encoding="raw", lossless=False):
    """Compress into the caller's uint8 CUDA tensor `out` with the library's fixed scratch
    (no device allocation by the library). Returns (stream bytes view, report dict)."""
    p = make_params(tuple(field.shape), field.dtype, eb, eb_mode, block, bins, abft, predictor, encoding, lossless)
    n = ctypes.c_size_t()
    rep = Report()
    rc = lib().sdcsz_compress_noalloc(ctypes.c_void_p(field.data_ptr()), ctypes.byref(p),
                                      ctypes.c_void_p(out.data_ptr()), out.numel(), ctypes.byref(n),
                                      ctypes.byref(rep), _stream_handle(stream))
    if rc:
        raise SdcszError(rc, "compress_noalloc")
    return out[: n.value], rep.as_dict()


class Batch:
    """Many fields compressed together: one persistent launch per stage and kernel shape over
    a device-side job table (see sdcsz_batch_* in the C header). ``eb``, ``eb_mode``,
    ``abft`` and ``predictor`` are one value for every field or a list/tuple with one entry
    per field; ``block`` is None, an int or a tuple for every field, or a list with one entry
    per field. Each field's stream is byte-identical to ``compress`` of that field."""

    def __init__(self, fields, eb, eb_mode="rel", block=None, bins=65536, abft=True, predictor="auto", stream=None,
                 encoding="raw"):
        import torch
        n = len(fields)
        encs = list(encoding) if isinstance(encoding, (list, tuple)) else [encoding] * n
        ebs = list(eb) if isinstance(eb, (list, tuple)) else [eb] * n
        modes = list(eb_mode) if isinstance(eb_mode, (list, tuple)) else [eb_mode] * n
        blocks = list(block) if isinstance(block, list) else [block] * n
        abfts = list(abft) if isinstance(abft, (list, tuple)) else [abft] * n
        preds = list(predictor) if isinstance(predictor, (list, tuple)) else [predictor] * n
        self.fields = list(fields)
        self.params = [make_params(tuple(f.shape), f.dtype, ebs[i], modes[i], blocks[i], bins, abfts[i], preds[i],
                                   encs[i]) for i, f in enumerate(self.fields)]
        self.caps = [compress_bound(p) for p in self.params]
        dev = self.fields[0].device
        self.outs = [torch.empty(c, dtype=torch.uint8, device=dev) for c in self.caps]
        items = (BatchItem * n)()
        for i, f in enumerate(self.fields):
            if not f.is_cuda or not f.is_contiguous():
                raise ValueError("fields must be contiguous CUDA tensors")
            items[i].d_field = f.data_ptr()
            items[i].params = self.params[i]
            items[i].d_out = self.outs[i].data_ptr()
            items[i].out_cap = self.caps[i]
        self.h = ctypes.c_void_p()
        rc = lib().sdcsz_batch_create(items, n, ctypes.byref(self.h))
        if rc:
            raise SdcszError(rc, "batch_create")
        nb = ctypes.c_size_t()
        lib().sdcsz_batch_workspace_size(self.h, ctypes.byref(nb))
        self.ws = torch.empty(nb.value, dtype=torch.uint8, device=dev)
        rc = lib().sdcsz_batch_bind(self.h, ctypes.c_void_p(self.ws.data_ptr()), self.ws.numel(),
                                    _stream_handle(stream))
        if rc:
            raise SdcszError(rc, "batch_bind")

    def set_fields(self, fields, stream=None):
        """Point the batch at new field tensors of the same shapes and dtypes."""
        n = len(self.fields)
        if len(fields) != n:
            raise ValueError("one tensor per field")
        for a, b in zip(fields, self.fields):
            if tuple(a.shape) != tuple(b.shape) or a.dtype != b.dtype or not a.is_contiguous():
                raise ValueError("set_fields keeps shapes and dtypes")
        arr = (ctypes.c_void_p * n)(*[f.data_ptr() for f in fields])
        rc = lib().sdcsz_batch_set_fields(self.h, arr, None, None, _stream_handle(stream))
        if rc:
            raise SdcszError(rc, "batch_set_fields")
        self.fields = list(fields)

    def compress(self, stream=None):
        """Enqueue the compression of every field (asynchronous)."""
        rc = lib().sdcsz_batch_compress(self.h, _stream_handle(stream))
        if rc:
            raise SdcszError(rc, "batch_compress")

    def capture(self, stream):
        """Capture the batch compression into a CUDA graph (``stream``: a non-default torch stream)."""
        rc = lib().sdcsz_batch_capture(self.h, ctypes.c_void_p(stream.cuda_stream))
        if rc:
            raise SdcszError(rc, "batch_capture")

    def launch(self, stream=None):
        """Replay the captured graph (or enqueue directly when nothing was captured)."""
        rc = lib().sdcsz_batch_launch(self.h, _stream_handle(stream))
        if rc:
            raise SdcszError(rc, "batch_launch")

    def results(self, stream=None, check=True):
        """Wait, then return [(stream bytes view, report dict)] per field."""
        n = len(self.fields)
        sizes = (ctypes.c_size_t * n)()
        reps = (Report * n)()
        rc = lib().sdcsz_batch_results(self.h, sizes, reps, _stream_handle(stream))
        if rc and check:
            raise SdcszError(rc, "batch_results")
        return [(self.outs[i][: sizes[i]], reps[i].as_dict()) for i in range(n)]

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            lib().sdcsz_batch_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request server (sdcsz_server_* in the C header).

    ``submit_*`` return immediately; ``poll`` returns completions as dicts with the result as
    a device pointer and size (for server-provided outputs ``result_view`` wraps it as a uint8
    CUDA tensor view, valid until ``release``). Caller tensors passed to a request must stay
    alive until its completion is polled: the server keeps references until then."""

    def __init__(self, hbm_budget: int, slots: int = 8):
        cfg = ServerConfig(int(hbm_budget), int(slots), 0)
        self.h = ctypes.c_void_p()
        rc = lib().sdcsz_server_create(ctypes.byref(cfg), ctypes.byref(self.h))
        if rc:
            raise SdcszError(rc, "server_create")
        self._keep = {}

    def _submit(self, req: Request, keep):
        rc = lib().sdcsz_server_submit(self.h, ctypes.byref(req))
        if rc:
            raise SdcszError(rc, "server_submit")
        self._keep[int(req.id)] = keep

    def submit_compress(self, rid, field, eb, eb_mode="rel", block=None, bins=65536, abft=True, predictor="auto",
                        out=None, flips=None, encoding="raw", lossless=False):
        r = Request()
        r.op, r.id, r.d_in = OP_COMPRESS, rid, field.data_ptr()
        r.params = make_params(tuple(field.shape), field.dtype, eb, eb_mode, block, bins, abft, predictor, encoding,
                               lossless)
        if out is not None:
            r.d_out, r.out_cap = out.data_ptr(), out.numel()
        ft = flips_tensor(flips, field.device) if flips else None
        if ft is not None:
            r.d_flips, r.n_flips = ft.data_ptr(), len(flips)
        self._submit(r, (field, out, ft))

    def submit_decompress(self, rid, stream_t, out=None, flips=None):
        r = Request()
        r.op, r.id, r.d_in, r.in_bytes = OP_DECOMPRESS, rid, stream_t.data_ptr(), stream_t.numel()
        if out is not None:
            r.d_out, r.out_cap = out.data_ptr(), out.numel() * out.element_size()
        ft = flips_tensor(flips, stream_t.device) if flips else None
        if ft is not None:
            r.d_flips, r.n_flips = ft.data_ptr(), len(flips)
        self._submit(r, (stream_t, out, ft))

    def submit_verify(self, rid, stream_t, original=None):
        r = Request()
        r.op, r.id, r.d_in, r.in_bytes = OP_VERIFY, rid, stream_t.data_ptr(), stream_t.numel()
        if original is not None:
            r.d_original = original.data_ptr()
        self._submit(r, (stream_t, original))

    def poll(self, max_n: int = 256, wait_us: int = 0):
        arr = (Completion * max_n)()
        n = ctypes.c_uint32()
        rc = lib().sdcsz_server_poll(self.h, arr, max_n, ctypes.byref(n), wait_us)
        if rc:
            raise SdcszError(rc, "server_poll")
        out = []
        for c in arr[: n.value]:
            self._keep.pop(int(c.id), None)
            out.append({"id": int(c.id), "op": int(c.op), "status": int(c.status), "d_result": c.d_result,
                        "result_bytes": int(c.result_bytes), "report": c.report.as_dict(), "t_submit": c.t_submit,
                        "t_admit": c.t_admit, "t_done": c.t_done})
        return out

    def release(self, rid):
        rc = lib().sdcsz_server_release(self.h, rid)
        if rc:
            raise SdcszError(rc, "server_release")

    def stats(self):
        st = ServerStats()
        lib().sdcsz_server_get_stats(self.h, ctypes.byref(st))
        return {n: int(getattr(st, n)) for n, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            lib().sdcsz_server_destroy(self.h)
            self.h = ctypes.c_void_p()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def result_view(completion, device=None):
    """A uint8 CUDA tensor view of a server-provided result (valid until Server.release)."""
    import torch
    n = completion["result_bytes"]
    if not n:
        return torch.empty(0, dtype=torch.uint8, device=device or "cuda")
    return _device_view(completion["d_result"], n, device)


def _device_view(ptr, nbytes, device=None):
    """Wrap raw device memory as a uint8 tensor (no copy, no ownership)."""
    import torch

    class _Arr:
        pass

    a = _Arr()
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    a.__cuda_array_interface__ = {"shape": (int(nbytes),), "typestr": "|u1", "data": (int(ptr), False),
                                  "version": 3, "strides": None}
    return torch.as_tensor(a, device=dev)


# ---------------------------------------------------------------- sharded compression (C ABI stages)
# Argument marshalling for the four stages of sdcsz_shard_*; the exchanges between them and
# their order are in paper_2010_03144_gb300.shard.

def _u64s(vals):
    return (ctypes.c_uint64 * len(vals))(*[int(v) for v in vals])


def shard_workspace_size(p: Params, b0: int, b1: int) -> int:
    out = ctypes.c_size_t()
    rc = lib().sdcsz_shard_workspace_size(ctypes.byref(p), b0, b1, ctypes.byref(out))
    if rc:
        raise SdcszError(rc, "shard_workspace_size")
    return out.value


def shard_prep(slab, p: Params, b0: int, b1: int, ws, stream=None):
    keys = (ctypes.c_uint64 * 2)()
    rc = lib().sdcsz_shard_prep(ctypes.c_void_p(slab.data_ptr()), ctypes.byref(p), b0, b1, ctypes.c_void_p(ws.data_ptr()),
                                ws.numel(), keys, _stream_handle(stream))
    if rc:
        raise SdcszError(rc, "shard_prep")
    return [int(keys[0]), int(keys[1])]


def shard_predict(slab, p: Params, b0: int, b1: int, ws, field_keys, stream=None):
    """Returns (counts [regression blocks, unpredictable points, uncorrectable blocks], the slab's
    code histogram as an int64 CUDA tensor view of 65536 bins inside the workspace)."""
    import torch
    counts = (ctypes.c_uint64 * 3)()
    hp = ctypes.c_void_p()
    rc = lib().sdcsz_shard_predict(ctypes.c_void_p(slab.data_ptr()), ctypes.byref(p), b0, b1,
                                   ctypes.c_void_p(ws.data_ptr()), ws.numel(), _u64s(field_keys), counts,
                                   ctypes.byref(hp), _stream_handle(stream))
    if rc:
        raise SdcszError(rc, "shard_predict")
    hist = _device_view(hp.value, 8 * 65536, ws.device).view(torch.int64)
    return [int(c) for c in counts], hist


def shard_encode(p: Params, b0: int, b1: int, ws, field_counts, header: bool, out, stream=None):
    """Returns the slab's totals [payload bytes, unpredictable values, regression blocks,
    uncorrectable blocks]; `out` (the field's stream buffer, zero on entry) receives the slab's
    per-block tables and, with header, the header and code table."""
    totals = (ctypes.c_uint64 * 4)()
    rc = lib().sdcsz_shard_encode(ctypes.byref(p), b0, b1, ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                  _u64s(field_counts), 1 if header else 0, ctypes.c_void_p(out.data_ptr()),
                                  out.numel(), totals, _stream_handle(stream))
    if rc:
        raise SdcszError(rc, "shard_encode")
    return [int(t) for t in totals]


def shard_assemble(p: Params, b0: int, b1: int, ws, prefix, field_totals, header: bool, out, stream=None):
    """Places the slab's data in `out`; returns (the field's stream size, the slab's report)."""
    nbytes = ctypes.c_size_t()
    rep = Report()
    rc = lib().sdcsz_shard_assemble(ctypes.byref(p), b0, b1, ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                    _u64s(prefix), _u64s(field_totals), 1 if header else 0,
                                    ctypes.c_void_p(out.data_ptr()), out.numel(), ctypes.byref(nbytes),
                                    ctypes.byref(rep), _stream_handle(stream))
    if rc:
        raise SdcszError(rc, "shard_assemble")
    return nbytes.value, rep.as_dict()
