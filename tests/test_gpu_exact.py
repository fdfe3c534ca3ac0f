"""Exact filtering on the GPU (Section "Exact Filtering"), through the C interface.

Every pixel's filtered channels in an exact-filtering render must equal, bit for bit, either the
full bilinear filter (where its footprint's samples cover its filter's texels, found from the
sampled indices by exact_support.py) or the plain estimate of the same sharing mode; and the render
must match the oracle's exact-filtering render within the colour tolerance. Also for the neural
material, the multi-view batch, and every tile shape. Unshaded colours are the channels and compare
bit for bit too; shaded colours compare within 1e-5 relative, because some of the compared renders
run one pixel per thread (the neural material, tile shapes whose pixel pairs do not share a
window) and others the paired path, whose packed shading the compiler may contract differently
(an ulp).
"""
import numpy as np
import pytest

import oracle as O
from exact_support import qualifying
from paper_2504_05562_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHARING = [O.QUAD2, O.WAVE2, O.WAVE3, O.WAVE4]


def _stf():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2504_05562_gb300 import stf
    return stf


def _render(stf, tex, view, mode, seed):
    out, idx, ch = stf.render(tex, view, mode, seed=seed, debug=True)
    torch.cuda.synchronize()
    stf.sync()
    return out.cpu().numpy(), idx.cpu().numpy().view(np.uint32), ch.cpu().numpy()


def _same_colour(a, b, shaded):
    if not shaded:
        return np.array_equal(a, b)
    return bool(np.all(np.abs(a - b) <= 1e-5 * np.maximum(np.abs(b), 1e-3)))


def _check_split(stf, tex, view, mode, seed, tex_w, tex_h):
    full, _, full_ch = _render(stf, tex, view, O.FULL, seed)
    wis, idx, wis_ch = _render(stf, tex, view, mode, seed)
    ex, idx2, ex_ch = _render(stf, tex, view, mode | stf.MODE_FLAG_EXACT, seed)
    assert np.array_equal(idx, idx2)
    q = qualifying(view, tex_w, tex_h, idx, mode)
    assert q.any()
    shaded = bool(view.get("shading"))
    assert np.array_equal(ex_ch[q], full_ch[q]) and _same_colour(ex[q], full[q], shaded)
    assert np.array_equal(ex_ch[~q], wis_ch[~q]) and _same_colour(ex[~q], wis[~q], shaded)
    return ex, idx, ex_ch, q


@pytest.mark.parametrize("tile", [(8, 4), (4, 8), (16, 2)])
@pytest.mark.parametrize("mode", SHARING)
def test_exact_split_and_oracle_parity_config1(mode, tile):
    stf = _stf()
    mat = W.material_c1()
    view = dict(W.config1_view(tile=tile), width=128, height=64)
    tex = stf.Texture(mat)
    ex, idx, ch, q = _check_split(stf, tex, view, mode, 7, mat["width"], mat["height"])
    r_out, r_idx, r_ch = O.render(mat, view, mode | O.FLAG_EXACT, seed=7, want_channels=True)
    assert np.array_equal(idx, r_idx)
    scale = np.maximum(np.abs(W.decoded_reference(mat)).reshape(-1, 4).max(0), 1e-3)
    tol = 1e-5 * np.maximum(np.abs(r_ch[..., :4]), scale)
    assert np.all(np.abs(ch[..., :4] - r_ch[..., :4]) <= tol)


def test_exact_split_fp16_shaded_material():
    stf = _stf()
    mat = W.material_c3(W.FP16, size=256)
    view = W.with_shading(W.screen_aligned_view(128, 64, 256, 256, 4.0, 0, origin=(3.0, 5.0)), "c3")
    _check_split(stf, stf.Texture(mat), view, O.WAVE3, 1, 256, 256)


def test_exact_split_neural_material():
    stf = _stf()
    from paper_2504_05562_gb300 import neural
    dec = neural.Decoder(128, 128, 32, 32, batch=1024, seed=4)
    view = W.with_shading(W.screen_aligned_view(96, 64, 128, 128, 4.0, 0, origin=(8.0, 9.0)), "c3")
    for mode in (O.QUAD2, O.WAVE3, O.WAVE4):
        _check_split(stf, dec.texture(), view, mode, 2, 128, 128)


def test_exact_flag_ignored_by_bspline_views():
    stf = _stf()
    mat = W.material_c1()
    view = dict(W.config1_view(1), width=64, height=32)
    tex = stf.Texture(mat)
    a, _, _ = _render(stf, tex, view, O.WAVE3, 3)
    b, _, _ = _render(stf, tex, view, O.WAVE3 | stf.MODE_FLAG_EXACT, 3)
    assert np.array_equal(a, b)


def test_exact_batch_equals_single_view_renders():
    stf = _stf()
    tex = stf.Texture(W.material_c3(W.FP16, size=512))
    views = W.config5_views(n=12, tex=512, seed=3, scale=0.2)
    tiles = [(8, 4), (4, 8), (16, 2)]
    for i, v in enumerate(views):
        v["tile"] = tiles[i % 3]
    mode = O.WAVE3 | stf.MODE_FLAG_EXACT
    outs = [torch.full((v["height"], v["width"], 4), -1.0, device="cuda") for v in views]
    stf.render_views([stf.make_view(v, tex, o) for v, o in zip(views, outs)], stf.FILTER_PER_VIEW, mode, 4)
    torch.cuda.synchronize()
    for v, o in zip(views, outs):
        want, _, _ = stf.render(tex, v, mode, seed=4)
        torch.cuda.synchronize()
        assert torch.equal(o, want)
    na = [torch.full((v["height"], v["width"], 4), -1.0, device="cuda") for v in views]
    stf.render_views_noalloc([stf.make_view(v, tex, o) for v, o in zip(views, na)], stf.FILTER_PER_VIEW, mode, 4)
    torch.cuda.synchronize()
    for a, b in zip(na, outs):
        assert torch.equal(a, b)
