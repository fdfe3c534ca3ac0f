"""The allocation-free batch entry point (stf_render_views_noalloc) against stf_render_views.

stf_render_views_noalloc serves callers that cannot let the library allocate device memory (a
render thread inside a fixed, pre-reserved memory budget, or a frame loop that must not stall on
cudaMalloc / cudaFree): its scratch is a fixed array inside the library. It must produce the
same pixels as the regular entry point, call after call, although every call reuses (and must
reset) that shared scratch. This file is collected last so that a run stopping at the first
failure has run everything else first; it also passes alone in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2504_05562_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-5  # the colour tolerance of the GPU tests


def _stf():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2504_05562_gb300 import stf
    return stf


def _batch(stf, views, tex_of, frame, noalloc):
    outs = [torch.full((v["height"], v["width"], 4), -1.0, device="cuda") for v in views]
    cv = [stf.make_view(dict(v, frame=frame), tex_of(i), o) for i, (v, o) in enumerate(zip(views, outs))]
    if noalloc:
        stf.render_views_noalloc(cv, stf.FILTER_PER_VIEW, stf.MODE_WAVE3, 11)
    else:
        stf.render_views(cv, stf.FILTER_PER_VIEW, stf.MODE_WAVE3, 11)
    torch.cuda.synchronize()
    stf.sync()
    return outs


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
        for g, w in zip(got, want):
            g, w = g.cpu().numpy().astype(np.float64), w.cpu().numpy().astype(np.float64)
            assert np.all(np.abs(g - w) <= RTOL * np.maximum(np.abs(w), 1e-3))


def test_noalloc_rejects_more_views_than_its_scratch_holds():
    stf = _stf()
    L = stf.load()
    arr = (stf.View * (stf.NOALLOC_MAX_VIEWS + 1))()
    assert L.stf_render_views_noalloc(arr, stf.NOALLOC_MAX_VIEWS + 1, 0, 4, 0) == stf.ERR_INVALID_ARG
    assert "scratch limit" in stf.last_error()
    assert L.stf_render_views_noalloc(C.cast(arr, C.POINTER(stf.View)), 0, 0, 4, 0) == stf.ERR_INVALID_ARG
