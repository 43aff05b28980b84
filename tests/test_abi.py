"""The C-ABI library builds, loads and exports every entry point of include/snn.h,
and the binding's structs match the C layout (no GPU needed, no compute calls)."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

from paper_2512_09502_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "snn.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^(?:int|void|const char\*)\s+(snn_\w+)\(", src, re.M)))


def test_header_declares_binding_names():
    assert declared() == sorted(_lib.EXPORTED)


def test_every_symbol_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True, text=True).stdout
    syms = set(re.findall(r" T (snn_\w+)$", out, re.M))
    for name in declared():
        assert name in syms, name
        assert hasattr(lib, name)


def test_struct_layouts_match_c():
    names = ["snn_config", "snn_iaf_psc_exp_params", "snn_rule", "snn_dist", "snn_stats_t", "snn_allocator"]
    prog = "#include <stdio.h>\n#include <stddef.h>\n#include \"snn.h\"\nint main(){" + "".join(
        f'printf("%zu\\n", sizeof({n}));' for n in names) + \
        'printf("%zu %zu\\n", offsetof(snn_stats_t, t_generate_ms), offsetof(snn_stats_t, sort_passes));return 0;}'
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(prog)
        exe = os.path.join(d, "t")
        subprocess.run(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe], check=True)
        got = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    sizes = [ctypes.sizeof(getattr(_lib, n)) for n in names]
    assert [int(x) for x in got[:len(names)]] == sizes
    assert int(got[-2]) == _lib.snn_stats_t.t_generate_ms.offset
    assert int(got[-1]) == _lib.snn_stats_t.sort_passes.offset


def test_every_struct_field_offset_matches_c():
    """Every field of every bound struct sits at the C compiler's offset (a field added
    or reordered on one side only is caught even when the sizes agree)."""
    names = ["snn_config", "snn_iaf_psc_exp_params", "snn_rule", "snn_dist", "snn_stats_t", "snn_allocator"]
    fields = [(n, f[0]) for n in names for f in getattr(_lib, n)._fields_]
    prog = "#include <stdio.h>\n#include <stddef.h>\n#include \"snn.h\"\nint main(){" + "".join(
        f'printf("%zu\\n", offsetof({n}, {f}));' for n, f in fields) + "return 0;}"
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(prog)
        exe = os.path.join(d, "t")
        subprocess.run(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe], check=True)
        got = [int(x) for x in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    want = [getattr(getattr(_lib, n), f).offset for n, f in fields]
    assert got == want, [(nf, g, w) for nf, g, w in zip(fields, got, want) if g != w]


def test_missing_library_fails_loudly(tmp_path):
    saved = _lib._lib
    try:
        _lib._lib = None
        with pytest.raises(RuntimeError, match="no CPU fallback"):
            _lib.load(str(tmp_path / "absent.so"))
    finally:
        _lib._lib = saved
