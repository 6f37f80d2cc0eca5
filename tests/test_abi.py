"""The C-ABI library without a GPU: it loads, exports every symbol the header declares, and its
host-only entry points (bounds, workspace sizes, header parsing, errors) behave."""

import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sz():
    from paper_2010_03144_gb300 import build
    build.build()
    import paper_2010_03144_gb300 as pkg
    pkg.lib()
    return pkg


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "sdcsz.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sdcsz_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_what_the_binding_expects(sz):
    assert sorted(sz.EXPORTS) == _declared_functions()


def test_every_declared_symbol_is_exported(sz):
    lib = ctypes.CDLL(sz.LIB_PATH)
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_bounds_and_workspace(sz):
    p = sz.make_params((512, 512, 512), np.float32, 1e-3)
    cap = sz.compress_bound(p)
    assert cap > 512**3 * 4  # every point unpredictable plus codes
    ws = sz.workspace_size(p)
    assert ws > 512**3 * 6  # codes and unpredictable staging
    assert sz.decompress_workspace_size() >= 128


@pytest.mark.parametrize("bad", [
    dict(shape=(10, 10, 10), block=1), dict(shape=(10, 10, 10), block=17), dict(shape=(10,) * 2, block=65),
    dict(shape=(10,), block=5000), dict(shape=(10, 10, 10), eb=0.0), dict(shape=(10, 10, 10), eb=float("nan")),
    dict(shape=(10, 10, 10), bins=3), dict(shape=(10, 10, 10), bins=65538)])
def test_invalid_parameters(sz, bad):
    kw = dict(bad)
    shape = kw.pop("shape")
    p = sz.make_params(shape, np.float32, kw.pop("eb", 1e-3), block=kw.pop("block", None), bins=kw.pop("bins", 65536))
    with pytest.raises(sz.SdcszError) as e:
        sz.compress_bound(p)
    assert e.value.code == sz.EINVAL


def test_library_parses_oracle_headers(sz, orc):
    """Stream format agreement on the host: headers written by the oracle parse in the library."""
    import synth
    for shape, dt, blk in [((13, 14, 15), np.float32, 6), ((40, 50), np.float64, 12), ((300,), np.float32, 64)]:
        x = synth.sinusoid_field(shape, 1, dtype=dt)
        s, rep = orc.compress(x, 1e-3, block=blk)
        h = sz.read_header(s)
        assert h["shape"] == shape and h["total"] == s.size and h["block"] == (blk,) * len(shape)
        assert h["dtype"] == np.dtype(dt).name
        bad = s.copy()
        bad[0] ^= 1
        with pytest.raises(sz.SdcszError):
            sz.read_header(bad)
        with pytest.raises(sz.SdcszError):
            sz.read_header(s[:100])


def test_strerror(sz):
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert sz.strerror(code) and sz.strerror(code) != "unknown error"


def test_trace_recorder_argument_checks(sz):
    """The deferred stage recorder rejects a zero or oversized capacity and an end without a
    begin before it touches the device."""
    L = sz.lib()
    assert L.sdcsz_trace_begin(0) == sz.EINVAL
    assert L.sdcsz_trace_begin((1 << 20) + 1) == sz.EINVAL
    n = ctypes.c_size_t(7)
    assert L.sdcsz_trace_end(None, None, 0, ctypes.byref(n)) == sz.EINVAL
    assert n.value == 7


def test_header_prefix_gives_the_stream_size(sz, orc):
    """The end-to-end loop learns a compressed stream's size from its first 128 bytes alone
    (read_header_partial): the total equals the stream's length, for every encoding."""
    import synth
    x = synth.sinusoid_field((30, 31, 32), 5, spikes=0.01)
    for kw in (dict(), dict(encoding="compact"), dict(lossless=True)):
        s, _ = orc.compress(x, 1e-3, **kw)
        h = sz.read_header_partial(s[:128], 1 << 30)
        assert h["total"] == s.size and h["shape"] == x.shape
        with pytest.raises(sz.SdcszError):
            sz.read_header_partial(s[:128], s.size - 1)  # a buffer shorter than the stream


def test_header_is_plain_c(tmp_path):
    """include/sdcsz.h is a C header: it compiles as C99 and as C++17 on its own, warnings on."""
    import shutil
    import subprocess
    src = tmp_path / "use.c"
    src.write_text('#include "sdcsz.h"\nint main(void) { return sdcsz_decompress_workspace_size() == 0; }\n')
    for comp, std, name in (("gcc", "-std=c99", "use.c"), ("g++", "-std=c++17", "use.cpp")):
        exe = shutil.which(comp)
        if exe is None:
            pytest.skip(f"{comp} not found")
        f = tmp_path / name
        f.write_text(src.read_text())
        r = subprocess.run([exe, std, "-Wall", "-Wextra", "-Werror", "-fsyntax-only", "-I",
                            os.path.join(ROOT, "include"), str(f)], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
