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
    assert lib.sesc_set_indicator_filter(None, 1) == sesc.SESC_EINVAL
    assert lib.sesc_set_stage_cap(None, 1) == sesc.SESC_EINVAL
    lib.sesc_destroy(None)


_VALID = dict(dim=2, M=8, nel=(4, 3), xlo=(0.0, 0.0), xhi=(1.0, 0.75), bc=(1, 1, 2, 2), gamma=1.4, tauA=100.0,
              tauS=0.05, alphaH=0.99, alphaL=0.01, betaL=0.95, cfl=0.5)
_NAN = float("nan")
_INVALID = [("dim", 1), ("dim", 4), ("M", 2), ("M", 6), ("M", 16), ("node_family", 2), ("node_family", -1),
            ("precision", 2), ("scheme", 2),
            ("nel", (0, 3)), ("nel", (-1, 3)), ("xhi", (0.0, 0.75)), ("xhi", (_NAN, 0.75)), ("bc", (4, 1, 2, 2)), ("bc", (3, 0, 2, 2)),
            ("bc", (-1, 1, 2, 2)), ("bc", (0, 1, 2, 2)), ("gamma", 1.0), ("gamma", 0.5), ("gamma", _NAN),
            ("tauA", 0.0), ("tauA", _NAN), ("tauS", -0.1), ("cfl", 0.0), ("cfl", _NAN), ("alphaL", -0.1),
            ("alphaH", 1.1), ("alphaL", 0.99), ("alphaH", _NAN), ("betaL", -0.1), ("betaL", 1.5), ("betaL", _NAN)]


@pytest.mark.parametrize("field,value", _INVALID, ids=[f"{f}={v}" for f, v in _INVALID])
def test_invalid_configurations_are_rejected_before_any_device_call(lib, field, value):
    """Every rule of the configuration (include/sesc.h: the ranges of dim, M, nel, the
    box, the boundary pairs, gamma, the indicator parameters, the thresholds
    0 <= alphaL < alphaH <= 1 and 0 <= betaL <= 1, cfl) rejects a violating value with
    SESC_EINVAL at handle creation, in a batch, and in the allocation-free entry point,
    before any device work (so on a host without a GPU too)."""
    from paper_2011_03338_gb300 import sesc
    if field in ("dim", "M", "node_family", "precision", "scheme"):   # set in the struct itself
        bad = sesc.make_config(_VALID)
        setattr(bad, field, value)
    else:
        bad = sesc.make_config(dict(_VALID, **{field: value}))
    h = ctypes.c_void_p()
    assert lib.sesc_create(ctypes.byref(bad), ctypes.byref(h)) == sesc.SESC_EINVAL and not h.value
    pair = (sesc.sesc_config * 2)(sesc.make_config(_VALID), bad)
    assert lib.sesc_batch_create(pair, 2, ctypes.byref(h)) == sesc.SESC_EINVAL and not h.value
    u, r = (ctypes.c_double * 4)(), (ctypes.c_double * 4)()       # never touched: validation comes first
    assert lib.sesc_rhs_static(ctypes.byref(bad), ctypes.addressof(u), ctypes.addressof(r), None) == sesc.SESC_EINVAL


def test_too_many_elements_are_rejected(lib):
    """More than 2^30 elements: SESC_EINVAL at creation and in the allocation-free
    entry point (same configuration rules); a valid problem larger than that entry
    point's static scratch (256^2 elements, M = 8: about 190 MB of scratch):
    SESC_ETOOLARGE, before any device call."""
    from paper_2011_03338_gb300 import sesc
    big = sesc.make_config(dict(_VALID, nel=(1 << 16, 1 << 15)))
    h = ctypes.c_void_p()
    assert lib.sesc_create(ctypes.byref(big), ctypes.byref(h)) == sesc.SESC_EINVAL
    u, r = (ctypes.c_double * 4)(), (ctypes.c_double * 4)()
    assert lib.sesc_rhs_static(ctypes.byref(big), ctypes.addressof(u), ctypes.addressof(r), None) == sesc.SESC_EINVAL
    large = sesc.make_config(dict(_VALID, nel=(256, 256)))
    assert lib.sesc_rhs_static(ctypes.byref(large), ctypes.addressof(u), ctypes.addressof(r), None) == sesc.SESC_ETOOLARGE
    split = sesc.make_config(dict(_VALID, precision="fp32_split"))
    assert lib.sesc_rhs_static(ctypes.byref(split), ctypes.addressof(u), ctypes.addressof(r), None) == sesc.SESC_EINVAL


def test_binding_requires_tensors_on_the_calls_device():
    """The binding passes a tensor's memory only when it lives on the device the
    call runs on (the handle's device; the current device for the allocation-free
    entry point): a tensor of another GPU would have its memory read by kernels on
    the wrong device."""
    import types

    import torch

    from paper_2011_03338_gb300.sesc import on_device
    t0 = types.SimpleNamespace(device=torch.device("cuda", 0))
    t1 = types.SimpleNamespace(device=torch.device("cuda", 1))
    assert on_device(t0, 0) and not on_device(t1, 0) and on_device(t1, 1)
    assert not on_device(torch.zeros(1), 0) and not on_device(object(), 0)


def test_product_path_has_no_oracle_and_no_fallback(tmp_path):
    """The package computes nothing on the host: no module of it imports the oracle,
    and with the library missing the binding raises instead of falling back."""
    import ast
    import subprocess
    import sys
    pkg = os.path.join(ROOT, "paper_2011_03338_gb300")
    for f in sorted(os.listdir(pkg)):
        if not f.endswith(".py"):
            continue
        tree = ast.parse(open(os.path.join(pkg, f)).read())
        for node in ast.walk(tree):
            names = []
            if isinstance(node, ast.Import):
                names = [a.name for a in node.names]
            elif isinstance(node, ast.ImportFrom):
                names = [node.module or ""]
            assert not any(n == "oracle" or n.startswith("oracle.") for n in names), (f, names)
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_2011_03338_gb300 import sesc\n"
            "sesc.LIB_PATH = %r\n"
            "try:\n    sesc.load()\nexcept RuntimeError as e:\n    print('raised:', e)\n") % (ROOT, str(tmp_path / "absent.so"))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "raised: CUDA library not built" in r.stdout, r.stdout + r.stderr
