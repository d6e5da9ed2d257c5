"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/h2gb.h declares (no device calls)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2506_16759_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "h2gb.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(h2_[a-z0-9_]+)\s*\(", text))
    # typedef'd function pointer types are not entry points
    return sorted(n for n in names if not n.endswith("_fn"))


@pytest.fixture(scope="module")
def built_lib():
    if not os.path.exists(_lib.LIB_PATH):
        from paper_2506_16759_gb300 import build
        build.build()
    return _lib.LIB_PATH


def test_header_parses():
    names = declared_functions()
    assert "h2_build" in names and "h2_matvec" in names and "h2_build_cluster_tree" in names


def test_every_declared_symbol_is_exported(built_lib):
    out = subprocess.run(["nm", "-D", "--defined-only", built_lib], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (h2_[a-z0-9_]+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert missing == []


def test_bindings_cover_the_header(built_lib):
    assert sorted(_lib.SIGNATURES) == declared_functions()
    L = _lib.lib()
    for name in _lib.SIGNATURES:
        assert getattr(L, name) is not None


def test_structs_match_c_layout(built_lib):
    # default options are written by the library itself
    o = _lib.BuildOpts()
    _lib.lib().h2_default_opts(ctypes.byref(o))
    assert (o.d0, o.d_inc, o.d_max, o.prec, o.omega_mode, o.sketch) == (32, 16, 256, 0, 0, 0)
    assert o.seed == 0 and not o.omega_stored and o.timing == 0
    # the low-rank term is off by default (the struct's last fields)
    assert o.lowrank_rank == 0 and not o.lowrank_u and not o.lowrank_v
    assert ctypes.sizeof(_lib.BuildOpts) % 8 == 0


def test_options_struct_has_the_c_size(built_lib):
    # h2_default_opts clears sizeof(h2_build_opts) bytes: on a buffer filled
    # with a pattern it must clear exactly the binding's struct (a longer C
    # struct would write past it, a shorter one would leave its tail)
    n = ctypes.sizeof(_lib.BuildOpts)
    buf = (ctypes.c_ubyte * (n + 64))(*([0xAB] * (n + 64)))
    _lib.lib().h2_default_opts(ctypes.cast(buf, ctypes.POINTER(_lib.BuildOpts)))
    assert all(b == 0xAB for b in buf[n:]), "the C struct is longer than the binding's"
    o = _lib.BuildOpts.from_buffer(buf)
    assert o.sum_engine == 0 and o.queue_order == 0 and o.nonsym == 0
    tail = bytes(buf[n - 8:n])
    assert tail != bytes([0xAB] * 8), "the C struct is shorter than the binding's"


def test_library_targets_sm103a():
    # the build compiles and links every translation unit for sm_103a only
    from paper_2506_16759_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert sorted(build.SOURCES) == sorted(
        f for f in os.listdir(build.CSRC) if f.endswith(".cu"))


def test_argument_errors_without_a_device(built_lib):
    # argument validation happens before any device work
    h = ctypes.c_void_p()
    st = _lib.lib().h2_build_cluster_tree(None, 10, 2, 8, 0.7, None, ctypes.byref(h))
    assert st == -1
    assert b"points" in _lib.lib().h2_last_error()


@pytest.mark.parametrize("n,dim,leaf,eta,word", [(0, 2, 8, 0.7, b"n must"), (10, 0, 8, 0.7, b"dim"),
                                                 (10, 4, 8, 0.7, b"dim"), (10, 2, 1, 0.7, b"leaf"),
                                                 (10, 2, 8, -1.0, b"eta"),
                                                 (10, 2, 8, float("inf"), b"eta")])
def test_degenerate_tree_arguments(built_lib, n, dim, leaf, eta, word):
    # empty and degenerate inputs are rejected before the points are touched
    # (the pointer below is never dereferenced)
    h = ctypes.c_void_p()
    dummy = ctypes.c_void_p(16)
    st = _lib.lib().h2_build_cluster_tree(dummy, n, dim, leaf, eta, None, ctypes.byref(h))
    assert st == -1
    assert word in _lib.lib().h2_last_error()
    assert not h.value
