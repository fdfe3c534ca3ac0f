"""The allocation-free batch entry point (stf_render_views_noalloc) against stf_render_views.

stf_render_views_noalloc serves callers that cannot let the library allocate device memory (a
render thread inside a fixed, pre-reserved memory budget, or a frame loop that must not stall on
cudaMalloc / cudaFree): its scratch is a fixed array inside the library. It must produce the
same pixels as the regular entry point, call after call, although every call reuses (and must
reset) that shared scratch, and it must leave the device's free memory unchanged. This file is
collected last so that a run stopping at the first failure has run everything else first; it
also passes alone in a fresh process.
"""
import ctypes as C
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2504_05562_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-5  # the colour tolerance of the GPU tests
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _stf():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2504_05562_gb300 import stf
    return stf


def _batch(stf, views, tex_of, frame, noalloc, mode=None):
    mode = stf.MODE_WAVE3 if mode is None else mode
    outs = [torch.full((v["height"], v["width"], 4), -1.0, device="cuda") for v in views]
    cv = [stf.make_view(dict(v, frame=frame), tex_of(i), o) for i, (v, o) in enumerate(zip(views, outs))]
    if noalloc:
        stf.render_views_noalloc(cv, stf.FILTER_PER_VIEW, mode, 11)
    else:
        stf.render_views(cv, stf.FILTER_PER_VIEW, mode, 11)
    torch.cuda.synchronize()
    stf.sync()
    return outs


def _assert_same(got, want):
    for g, w in zip(got, want):
        tol = RTOL * torch.clamp(w.abs(), min=1e-3)
        bad = ~((g - w).abs() <= tol)
        assert not bool(bad.any()), "%d pixels differ" % int(bad.sum())


def test_noalloc_matches_regular_entry_point_on_consecutive_calls():
    stf = _stf()
    t16 = stf.Texture(W.material_c3(W.FP16, size=512))
    t8 = stf.Texture(W.material_c2(size=512))
    views = W.config5_views(n=20, tex=512, seed=2, scale=0.2)
    tiles = [(8, 4), (4, 8), (16, 2)]
    for i, v in enumerate(views):
        v["tile"] = tiles[i % 3]
        if i % 4 == 3:  # a second material kind in the same batch: 4 channels + normal, c2 layout
            v.update(ch_albedo=0, ch_normal=4, ch_rough=-1, ch_ao=-1)
    tex_of = lambda i: t8 if i % 4 == 3 else t16  # noqa: E731
    for frame in (0, 1):  # two calls in a row: the shared scratch must be reset each time
        got = _batch(stf, views, tex_of, frame, noalloc=True)
        want = _batch(stf, views, tex_of, frame, noalloc=False)
        _assert_same(got, want)


def _random_decoder(neural, tex, lat, seed):
    import oracle as O
    dec = neural.Decoder(tex, tex, lat, lat, batch=1024, seed=seed)
    rng = np.random.default_rng(seed)
    dec.set_params(rng.normal(0, 0.5, (lat, lat, 16)).astype(np.float32),
                   rng.normal(0, 0.25, O.NN_PARAMS).astype(np.float32))
    return dec


def test_noalloc_neural_views_share_one_decoder():
    """A batch mixing neural-material views with FP16 ones renders as stf_render_views does; a
    second decoder in one call is refused before anything is enqueued."""
    stf = _stf()
    from paper_2504_05562_gb300 import neural
    dec = _random_decoder(neural, 256, 64, 7)
    ntex = dec.texture()
    t16 = stf.Texture(W.material_c3(W.FP16, size=256))
    views = W.config5_views(n=6, tex=256, seed=5, scale=0.15)
    tex_of = lambda i: ntex if i % 2 == 0 else t16  # noqa: E731
    for frame in (0, 1):
        _assert_same(_batch(stf, views, tex_of, frame, noalloc=True), _batch(stf, views, tex_of, frame, noalloc=False))
    dec2 = _random_decoder(neural, 256, 64, 8)
    ntex2 = dec2.texture()
    outs = [torch.zeros((v["height"], v["width"], 4), device="cuda") for v in views[:2]]
    cv = [stf.make_view(views[0], ntex, outs[0]), stf.make_view(views[1], ntex2, outs[1])]
    arr = (stf.View * 2)(*cv)
    assert stf.load().stf_render_views_noalloc(arr, 2, stf.FILTER_PER_VIEW, stf.MODE_WAVE3, 0) == stf.ERR_INVALID_ARG
    assert "second neural decoder" in stf.last_error()
    torch.cuda.synchronize()
    assert all(bool((o == 0).all()) for o in outs)


def test_noalloc_coarsens_work_items_beyond_its_list(tmp_path):
    """Nine 3840x2160 views at one tile per warp per work item make 291,600 items, more than the
    fixed list holds (STF_NOALLOC_MAX_ITEMS): items are coarsened, and no pixel changes."""
    stf = _stf()
    tex = stf.Texture(W.material_c3(W.FP16, size=2048))
    views = [dict(W.config3_view(0, frame=0), view_id=i) for i in range(9)]
    for i, v in enumerate(views):
        v["H"] = list(v["H"])
        v["H"][2] += 1e-3 * i  # distinct views
        v["tile"] = (8, 4)
    tab = tmp_path / "tune.txt"
    # class of these views: FP16 x 8 kind, bilinear, WAVE3, magnification bucket [2, 8), >= 3 Mpixel
    tab.write_text("# stf autotune v1 gpu=test\nkind3/filter0/mode4/mag1/res2 8 4 1 0.0\n")
    stf.autotune_clear()
    stf.autotune_load(str(tab))
    try:
        probe = torch.empty((views[0]["height"], views[0]["width"], 4), device="cuda")
        assert stf.view_config(stf.make_view(views[0], tex, probe)) == (8, 4, 1)
        del probe
        items = sum(-(-((v["width"] // 8) * (v["height"] // 4)) // 8) for v in views)
        assert items > stf.NOALLOC_MAX_ITEMS
        got = _batch(stf, views, lambda i: tex, 3, noalloc=True)
        want = _batch(stf, views, lambda i: tex, 3, noalloc=False)
        _assert_same(got, want)
    finally:
        stf.autotune_clear()


_CHILD = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
import torch
from paper_2504_05562_gb300 import stf, workloads as W
torch.cuda.init()
t16 = stf.Texture(W.material_c3(W.FP16, size=512))
t8 = stf.Texture(W.material_c2(size=512))
views = W.config5_views(n=12, tex=512, seed=4, scale=0.2)
tiles = [(8, 4), (4, 8), (16, 2)]
for i, v in enumerate(views):
    v["tile"] = tiles[i % 3]
    if i % 4 == 3:
        v.update(ch_albedo=0, ch_normal=4, ch_rough=-1, ch_ao=-1)
outs = [torch.empty((v["height"], v["width"], 4), device="cuda") for v in views]
cvs = [stf.make_view(v, t8 if i % 4 == 3 else t16, o) for i, (v, o) in enumerate(zip(views, outs))]
torch.cuda.synchronize()
torch.cuda.mem_get_info()
free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
calls = [(cvs, stf.MODE_WAVE3), (cvs[:1], stf.MODE_WAVE3), (cvs[3:9], stf.MODE_QUAD2), (cvs, stf.MODE_ONE_TAP),
         (cvs[::2], stf.MODE_WAVE4 | stf.MODE_FLAG_EXACT), (cvs, stf.MODE_WAVE3)]
for k, (batch, mode) in enumerate(calls):
    stf.render_views_noalloc(batch, stf.FILTER_PER_VIEW, mode, k)
torch.cuda.synchronize()
stf.sync()
free1, alloc1 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
print(json.dumps({"free0": free0, "free1": free1, "alloc0": alloc0, "alloc1": alloc1}))
"""


def test_noalloc_leaves_device_memory_unchanged_in_a_fresh_process():
    """In a fresh process whose kernels are loaded eagerly (so the driver's lazy module loading
    allocates nothing later), textures and outputs are created first; then no-alloc calls of
    different view counts, tile mixes and modes, with no regular render before them, leave the
    device's free memory and the torch allocator unchanged."""
    _stf()
    env = dict(os.environ, CUDA_MODULE_LOADING="EAGER")
    r = subprocess.run([sys.executable, "-c", _CHILD, ROOT], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["free1"] == res["free0"], res
    assert res["alloc1"] == res["alloc0"], res


def test_noalloc_rejects_more_views_than_its_scratch_holds():
    stf = _stf()
    L = stf.load()
    arr = (stf.View * (stf.NOALLOC_MAX_VIEWS + 1))()
    assert L.stf_render_views_noalloc(arr, stf.NOALLOC_MAX_VIEWS + 1, 0, 4, 0) == stf.ERR_INVALID_ARG
    assert "scratch limit" in stf.last_error()
    assert L.stf_render_views_noalloc(C.cast(arr, C.POINTER(stf.View)), 0, 0, 4, 0) == stf.ERR_INVALID_ARG
