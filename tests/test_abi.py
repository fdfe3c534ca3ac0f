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
    for mode in (stf.MODE_FULL, stf.MODE_ONE_TAP):  # exact filtering needs a sharing mode
        assert L.stf_render_views(arr, 1, 0, mode | stf.MODE_FLAG_EXACT, 0) == stf.ERR_INVALID_ARG
        assert "exact filtering" in stf.last_error()
    assert L.stf_render_views(arr, 1, 0, 9 | stf.MODE_FLAG_EXACT, 0) == stf.ERR_INVALID_ARG
    assert L.stf_create_texture(None, None) == stf.ERR_INVALID_ARG
    assert L.stf_update_texture(None, None, 0) == stf.ERR_INVALID_ARG
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


def _ckpt_bytes(nlat=16 * 16 * 16, nparams=6280, crc_ok=True, magic=b"STFDEC01"):
    import struct
    import zlib
    hdr = struct.pack("<8sI5i5f4xQqqii", magic, 1, 64, 64, 16, 16, 1024, 1e-2, 5e-3, 0.9, 0.99, 1e-10, 7, 10,
                      nlat, nparams, 0)
    assert len(hdr) == 88
    payload = bytes(4 * (3 * nlat + 3 * nparams))
    crc = zlib.crc32(hdr + payload)
    if not crc_ok:
        crc ^= 1
    return hdr + payload + struct.pack("<I", crc)


def test_corrupted_checkpoints_rejected_before_any_gpu_work(tmp_path):
    """Checkpoint validation (magic, header consistency, CRC-32, length) happens on the host."""
    from paper_2504_05562_gb300 import neural  # noqa: F401  (binds the decoder entry points)
    L = stf.load()
    h = C.c_void_p()
    cases = {"bad_magic": _ckpt_bytes(magic=b"NOTADEC!"), "bad_crc": _ckpt_bytes(crc_ok=False),
             "truncated": _ckpt_bytes()[:-100], "bad_header": _ckpt_bytes(nlat=5),
             "trailing": _ckpt_bytes() + b"x"}
    for name, data in cases.items():
        p = tmp_path / (name + ".ckpt")
        p.write_bytes(data)
        assert L.stf_decoder_load(str(p).encode(), C.byref(h)) == stf.ERR_INVALID_ARG, name
        assert h.value is None
    assert "checksum" in (L.stf_decoder_load(str(tmp_path / "bad_crc.ckpt").encode(), C.byref(h)) and stf.last_error())
    assert L.stf_decoder_load(str(tmp_path / "missing.ckpt").encode(), C.byref(h)) == stf.ERR_INVALID_ARG
    # a well-formed file passes validation (its CRC-32 agrees with zlib's); without a GPU the load
    # then stops at the first device allocation
    p = tmp_path / "good.ckpt"
    p.write_bytes(_ckpt_bytes())
    rc = L.stf_decoder_load(str(p).encode(), C.byref(h))
    assert rc != stf.ERR_INVALID_ARG, stf.last_error()
    if rc == stf.OK:
        L.stf_decoder_destroy(h)


def test_binding_constants_match_the_header():
    """The Python binding's enum values equal the header's (the binding only marshals)."""
    import re
    text = open(os.path.join(os.path.dirname(__file__), "..", "include", "stf.h")).read()
    pairs = {
        "STF_MODE_SPARSE9": stf.MODE_SPARSE9, "STF_MODE_FLAG_EXACT": stf.MODE_FLAG_EXACT,
        "STF_MODE_FLAG_BLUE_NOISE": stf.MODE_FLAG_BLUE_NOISE, "STF_MODE_EST_SHIFT": stf.MODE_EST_SHIFT,
        "STF_MODE_FLAG_CLAMP": stf.MODE_FLAG_CLAMP, "STF_OPT_BATCH_GRAPHS": stf.OPT_BATCH_GRAPHS,
        "STF_OPT_PIPELINE_BLOCKS": stf.OPT_PIPELINE_BLOCKS, "STF_OPT_TEST_DECODE_STALL": stf.OPT_TEST_DECODE_STALL,
    }
    for name, value in pairs.items():
        m = re.search(r"\b%s\s*(?:=\s*)?\(?\s*(\d+)" % name, text)
        assert m, name
        assert int(m.group(1)) == value, (name, m.group(1), value)


def test_autotune_table_round_trip_and_rejections(tmp_path):
    """The autotune table's text format (host logic, no GPU): a valid table loads and saves back
    with the same entries; files without the header or with a tile shape or schedule the kernels
    do not have are rejected and leave the table unchanged."""
    L = stf.load()
    assert L.stf_autotune_clear() == stf.OK
    good = tmp_path / "good.txt"
    good.write_text("# stf autotune v1 gpu=test\n"
                    "k3f0m4r2m8 8 4 2 0.012500\n"
                    "k3f1m4r1m32 4 8 8 0.250000\n"
                    "k6f1m4r0m2 16 2 1 0.001000\n")
    assert L.stf_autotune_load(str(good).encode()) == stf.OK
    out = tmp_path / "saved.txt"
    assert L.stf_autotune_save(str(out).encode()) == stf.OK
    lines = out.read_text().splitlines()
    assert lines[0].startswith("# stf autotune v1")
    entries = {ln.split()[0]: ln.split()[1:4] for ln in lines[1:]}
    assert entries == {"k3f0m4r2m8": ["8", "4", "2"], "k3f1m4r1m32": ["4", "8", "8"], "k6f1m4r0m2": ["16", "2", "1"]}
    for bad in ("k3f0m4r2m8 8 4 2 0.1\n",                                # no header
                "# stf autotune v1\nk3f0m4r2m8 5 5 2 0.1\n",             # no such tile shape
                "# stf autotune v1\nk3f0m4r2m8 8 4 0 0.1\n"):            # schedule out of range
        p = tmp_path / "bad.txt"
        p.write_text(bad)
        assert L.stf_autotune_load(str(p).encode()) == stf.ERR_INVALID_ARG
    assert L.stf_autotune_load(str(tmp_path / "missing.txt").encode()) == stf.ERR_INVALID_ARG
    assert L.stf_autotune_save(str(out).encode()) == stf.OK
    assert len(out.read_text().splitlines()) == 4  # unchanged by the rejected loads
    assert L.stf_autotune_clear() == stf.OK
