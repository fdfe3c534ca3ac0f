"""The C-ABI library loads and exports every entry point include/*.h declares; host-side argument
validation rejects bad calls before touching the GPU (no GPU needed)."""
import ctypes as C
import glob
import os
import re

import pytest

from paper_2504_05562_gb300 import stf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:stf_status|const char\*|int)\s+(stf_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("stf_create_texture", "stf_render_views", "stf_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    L = stf.load()
    missing = [n for n in sorted(_declared()) if not hasattr(L, n)]
    assert not missing, missing
    assert stf.version() >= 10000


def test_invalid_arguments_rejected_on_host():
    L = stf.load()
    assert L.stf_render_views(None, 0, 0, 0, 0) == stf.ERR_INVALID_ARG
    assert "n >= 1" in stf.last_error()
    v = stf.View()
    v.width, v.height = 16, 16
    arr = (stf.View * 1)(v)
    assert L.stf_render_views(arr, 1, 0, 4, 0) == stf.ERR_INVALID_ARG  # null texture
    assert "null texture" in stf.last_error()
    assert L.stf_render_views(arr, 1, 7, 4, 0) == stf.ERR_INVALID_ARG  # bad filter
    assert L.stf_render_views(arr, 1, 0, 9, 0) == stf.ERR_INVALID_ARG  # bad mode
    assert L.stf_create_texture(None, None) == stf.ERR_INVALID_ARG
    d = stf.TextureDesc()
    d.width, d.height, d.num_planes = 0, 4, 1
    h = C.c_void_p()
    assert L.stf_create_texture(C.byref(d), C.byref(h)) == stf.ERR_INVALID_ARG
    d.width, d.height, d.num_planes = 4, 4, 5
    assert L.stf_create_texture(C.byref(d), C.byref(h)) == stf.ERR_INVALID_ARG
    d.num_planes = 1
    d.planes[0].fmt, d.planes[0].channels, d.planes[0].data = 9, 4, 1
    assert L.stf_create_texture(C.byref(d), C.byref(h)) == stf.ERR_INVALID_ARG
    assert "format" in stf.last_error()
    d.planes[0].fmt, d.planes[0].channels = 0, 9
    assert L.stf_create_texture(C.byref(d), C.byref(h)) == stf.ERR_INVALID_ARG
    assert h.value is None
    assert L.stf_destroy(None) == stf.OK
