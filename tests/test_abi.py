"""CPU checks of the C ABI: the library builds, loads without a GPU and exports
every function include/sesc.h declares; the binding's structure matches the
header's struct layout."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sesc.h")


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"\b(sesc_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2011_03338_gb300 import build, sesc
    build.build()            # incremental: recompiles only what changed
    return sesc.load()


def test_library_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True, text=True).stdout
    for n in names:
        assert re.search(rf"\bT {n}$", out, re.M), n


def test_binding_covers_header(lib):
    from paper_2011_03338_gb300 import sesc
    assert sorted(sesc.SYMBOLS) == _declared()


def test_config_struct_layout_matches_header(tmp_path):
    """Compile a tiny C program against the header and compare offsetof/sizeof
    with the ctypes structure."""
    from paper_2011_03338_gb300.sesc import sesc_config
    fields = [f[0] for f in sesc_config._fields_]
    src = tmp_path / "layout.c"
    body = "\n".join(f'printf("{f} %zu\\n", offsetof(sesc_config, {f}));' for f in fields)
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "sesc.h"\nint main(void){\n'
                   + body + '\nprintf("size %zu\\n", sizeof(sesc_config));\nreturn 0;}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split("\n") if line)
    for f in fields:
        assert int(got[f]) == getattr(sesc_config, f).offset, f
    assert int(got["size"]) == ctypes.sizeof(sesc_config)


def test_error_strings_and_argument_errors(lib):
    from paper_2011_03338_gb300 import sesc
    assert "permissible" in sesc.strerror(sesc.SESC_ENONPERMISSIBLE)
    assert sesc.strerror(99) == "unknown error"
    # invalid configurations are rejected before any device call
    bad = sesc.make_config(dict(dim=2, M=6, nel=(2, 2), xlo=(0, 0), xhi=(1, 1), bc=(0, 0, 0, 0), gamma=1.4,
                                tauA=100, tauS=0.05, alphaH=0.99, alphaL=0.01, betaL=0.95, cfl=0.5))
    h = ctypes.c_void_p()
    assert lib.sesc_create(ctypes.byref(bad), ctypes.byref(h)) == sesc.SESC_EINVAL and not h.value
    bad = sesc.make_config(dict(dim=2, M=8, nel=(2, 2), xlo=(0, 0), xhi=(1, 1), bc=(0, 1, 0, 0), gamma=1.4,
                                tauA=100, tauS=0.05, alphaH=0.99, alphaL=0.01, betaL=0.95, cfl=0.5))
    assert lib.sesc_create(ctypes.byref(bad), ctypes.byref(h)) == sesc.SESC_EINVAL
    assert lib.sesc_create(None, ctypes.byref(h)) == sesc.SESC_EINVAL
    assert lib.sesc_rhs(None, None, None, None, None, None) == sesc.SESC_EINVAL
    lib.sesc_destroy(None)
