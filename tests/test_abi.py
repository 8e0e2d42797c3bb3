"""The C-ABI library builds, loads and exports every entry point of gs.h
(no GPU needed: only calls that do no device work are made)."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gs_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2510_15352_b300 import build
    build.build()
    from paper_2510_15352_b300 import gs
    return gs


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("gs_context_create", "gs_scene_create", "gs_render_batch", "gs_get_stats"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    raw = ctypes.CDLL(lib.LIB_PATH)
    for name in declared_functions():
        assert hasattr(raw, name), name
    assert set(declared_functions()) == set(lib.SIGNATURES), "binding and header differ"


def test_host_only_calls(lib):
    assert lib.gs_abi_version() == lib.ABI_VERSION
    c = lib.default_config()
    assert abs(c.alpha_min - 1 / 255) < 1e-9 and c.alpha_max == pytest.approx(0.99)
    assert c.T_min == pytest.approx(1e-4) and c.dilation == pytest.approx(0.3)
    assert lib.gs_status_string(lib.GS_ERR_CAPACITY) == b"capacity exceeded"
    assert lib.gs_config_default(None) == lib.GS_ERR_INVALID_ARG
    assert lib.gs_last_error(None) == b"NULL context"
    out = ctypes.c_void_p(123)
    bad = lib.default_config(camera_group=129)  # past the largest camera group (128)
    assert lib.gs_context_create(ctypes.byref(bad), 0, ctypes.byref(out)) == lib.GS_ERR_INVALID_ARG
    assert out.value is None


def test_struct_layouts_match_header(lib, tmp_path):
    """sizeof / offsetof of every ABI struct, from gcc compiling gs.h, equal
    the ctypes mirrors of the binding."""
    structs = {"gs_config": lib.gs_config, "gs_scene_desc": lib.gs_scene_desc,
               "gs_stats": lib.gs_stats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gs.h"', "int main(void){"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines.append("return 0;}")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    import subprocess
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)]).decode().splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(cls, f).offset, f"{name}.{f}"
