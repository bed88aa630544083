"""The C ABI library loads without a GPU and exports every entry point that
include/gputx.h declares; the Python binding names the same functions."""
import ctypes
import os
import re

import pytest

import paper_1103_3105_gb300 as G
from paper_1103_3105_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(gputx_\w+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def libpath():
    return _build.build()


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    declared = _declared()
    assert len(declared) >= 14
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_abi(libpath):
    assert set(G.EXPORTED) <= _declared()
    assert _declared() <= set(G.EXPORTED) | {n for n in _declared() if n.startswith("gputx_")
                                            and hasattr(G, n)}
    assert G.gputx_version().startswith("gputx-gb300")


def _declared_arity():
    """name -> parameter count of every function the headers declare."""
    out = {}
    for f in os.listdir(os.path.join(ROOT, "include")):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for name, params in re.findall(r"\b(gputx_\w+)\s*\(([^;{]*?)\)\s*;", text, flags=re.S):
            params = params.strip()
            out[name] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_signatures_match_the_header():
    """Every declared function has a ctypes signature with as many arguments
    as the header gives it (a stale binding would pass garbage silently)."""
    arity = _declared_arity()
    sig = G.signatures()
    assert len(arity) >= 30
    assert set(arity) == set(sig), (set(arity) ^ set(sig))
    wrong = {n: (arity[n], len(sig[n][0])) for n in arity if arity[n] != len(sig[n][0])}
    assert not wrong, wrong


def test_structs_match_header_sizes():
    # the binding's ctypes mirrors must keep the header's field order and sizes
    assert ctypes.sizeof(G.SchemaDesc) == 10 * 8
    assert ctypes.sizeof(G.Config) == 8 + 4 + 4 + 8 * 4
    assert ctypes.sizeof(G.ExecOpts) == 24
    assert ctypes.sizeof(G.ExecStats) == 8 + 6 * 8 + 6 * 4
    assert ctypes.sizeof(G.ServeConfig) == 8 * 2 + 4 * 4 + 8 * 2 + 4 * 2
    assert ctypes.sizeof(G.ServeStats) == 5 * 8 + 4 * 8
    assert ctypes.sizeof(G.BatchConfig) == 4 * 4 + 2 * 8 + 2 * 4
    assert ctypes.sizeof(G.PoolConfig) == 8 + 2 * 4 + 2 * 8
    assert ctypes.sizeof(G.BatchChoice) == 4 * 4 + 2 * 8 + 16 * 4 * 2 + 16 * 8 * 2 + 2 * 8


def test_probe_rejects_bad_shapes_without_a_gpu():
    """Argument checks come before any CUDA call, so they run on CPU."""
    import paper_1103_3105_gb300 as G
    if not os.path.exists(G.LIB_PATH):
        pytest.skip("library not built")
    for args in [(0, 16, 64, 3, 10), (10, 17, 64, 3, 10), (10, 16, 48, 3, 10), (10, 16, 64, 9, 10),
                 (10, 16, 64, 3, 0), (10, 16, 64, 3, 17), (10, 16, 64, 3, 3, -1), (10, 16, 64, 3, 3, 14),
                 (10, 16, 64, 0, 3, 7, 3), (10, 16, 64, 0, 3, 7, -1)]:
        with pytest.raises(G.GputxError) as e:
            G.gputx_probe_level_chain(*args)
        assert e.value.status == G.EINVAL
    for args in [(0, 0), (-5, 1), ((1 << 32) + 1, 0), (1000, 2), (1000, -1)]:
        with pytest.raises(G.GputxError) as e:
            G.gputx_probe_atomics(*args)
        assert e.value.status == G.EINVAL


def test_debug_build_exports_every_declared_symbol():
    """The bounds-checked build (-DGPUTX_DEBUG) compiles from the same sources
    into its own library with the same entry points."""
    path = _build.build(debug=True)
    assert path.endswith("libgputx_debug.so") and path != _build.LIB
    lib = ctypes.CDLL(path)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing
