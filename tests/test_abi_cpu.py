"""Host-side checks of the C ABI that need no GPU: the library builds, loads, exports every
symbol include/vrc.h declares, and its host-only calls behave."""
import ctypes as C
import os
import re
import shutil

import pytest

from paper_2005_01442_gb300 import build, native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "vrc.h")).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+char\s*\*\s*|vrc_status\s+|int\s+|size_t\s+)(vrc_\w+)\s*\(",
                                 src, re.M)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(build.LIB):
        if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("nvcc not available to build libvrc")
        build.build()
    return native.load()


def test_header_and_binding_agree():
    assert _declared() == sorted(native.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_host_only_calls(lib):
    assert lib.vrc_version() == 100
    assert lib.vrc_status_str(0) == b"VRC_OK"
    assert lib.vrc_status_str(-6) == b"VRC_ERR_STATE"
    assert lib.vrc_status_str(12345) == b"VRC_UNKNOWN"
    assert lib.vrc_last_error_message(None) == b""
    # NULL context and NULL outputs are rejected before touching the device
    assert lib.vrc_create(None, 0) == -1
    assert lib.vrc_destroy(None) == 0
    assert lib.vrc_render(None, 1, 1, None, None, None, None, None, None) == -1
    assert lib.vrc_ckpt_bytes(None, None, 1, None) == 0
    assert lib.vrc_microbench(None, 0, None, None) == -1
    assert lib.vrc_bricks_build(None, 1, 8, None) == -1


def _header_struct(name):
    # (field name, C type, array length) of `typedef struct { ... } name;` in include/vrc.h
    text = open(os.path.join(ROOT, "include", "vrc.h")).read()
    body = re.search(r"typedef struct \{([^}]*)\}\s*" + name + ";", text).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        typ, names = decl.split(None, 1)
        for n in names.split(","):
            m = re.match(r"\s*(\w+)\s*(?:\[(\d+)\])?", n)
            fields.append((m.group(1), typ, int(m.group(2) or 1)))
    return fields


def test_struct_layouts_match_header():
    ctype = {"int": C.c_int, "float": C.c_float}
    for py, name in ((native.vrc_camera, "vrc_camera"), (native.vrc_params, "vrc_params")):
        hdr = _header_struct(name)
        got = [(f, t) for f, t in py._fields_]
        assert [f for f, _ in got] == [f for f, _, _ in hdr], name
        for (f, t), (_, typ, n) in zip(got, hdr):
            want = ctype[typ] * n if n > 1 else ctype[typ]
            assert C.sizeof(t) == C.sizeof(want) and getattr(t, "_type_", t) == getattr(
                want, "_type_", want), (name, f)
