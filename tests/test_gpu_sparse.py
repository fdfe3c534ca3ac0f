"""Rendering with pseudorandom sparse footprints (STF_MODE_SPARSE9) on the GPU against the CPU
oracle, through the C interface. The footprint tables are seeded random valid tables (any table
is a valid input of the sharing step), set on the GPU and handed to the oracle."""
import numpy as np
import pytest

import oracle as O
from paper_2504_05562_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _stf():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2504_05562_gb300 import stf
    return stf


def _table(patterns, seed, tile):
    tw, th = tile
    rng = np.random.default_rng(seed)
    tab = np.zeros((patterns, 32, 9), np.int8)
    for p in range(patterns):
        for lane in range(32):
            # 8 other lanes, nearer ones likelier (the generator's locality, any valid table works)
            d = np.array([np.hypot(j % tw - lane % tw, j // tw - lane // tw) for j in range(32)])
            w = np.exp(-d ** 2 / 8.0)
            w[lane] = 0
            tab[p, lane] = [lane] + list(rng.choice(32, 8, replace=False, p=w / w.sum()))
    return tab


@pytest.mark.parametrize("tile", [(8, 4), (4, 8), (16, 2)])
@pytest.mark.parametrize("exact", [False, True])
def test_sparse_parity_config1(tile, exact):
    stf = _stf()
    mat = W.material_c1()
    tab = _table(3, 5, tile)
    stf.set_sparse_footprints(tab, tile)
    tex = stf.Texture(mat)
    mode = stf.MODE_SPARSE9 | (stf.MODE_FLAG_EXACT if exact else 0)
    scale = np.maximum(np.abs(W.decoded_reference(mat)).reshape(-1, 4).max(0), 1e-3)
    for frame in (0, 1, 2, 4):
        view = dict(W.screen_aligned_view(64, 32, 64, 64, 3.6, 0, origin=(4.2, 6.9), tile=tile), frame=frame)
        out, idx, ch = stf.render(tex, view, mode, seed=2, debug=True)
        torch.cuda.synchronize()
        stf.sync()
        r_out, r_idx, r_ch = O.render(mat, dict(view, footprints=tab), mode, seed=2, want_channels=True)
        assert np.array_equal(idx.cpu().numpy().view(np.uint32), r_idx)
        g, r = ch.cpu().numpy()[..., :4].astype(np.float64), r_ch[..., :4].astype(np.float64)
        assert np.all(np.abs(g - r) <= 1e-5 * np.maximum(np.abs(r), scale))


def test_sparse_parity_shaded_fp16_bspline():
    stf = _stf()
    mat = W.material_c3(W.FP16, size=256)
    tab = _table(2, 9, (8, 4))
    stf.set_sparse_footprints(tab, (8, 4))
    view = W.with_shading(W.screen_aligned_view(64, 32, 256, 256, 4.0, 1, origin=(7.1, 3.3)), "c3")
    out, idx, ch = stf.render(stf.Texture(mat), view, stf.MODE_SPARSE9, seed=3, debug=True)
    torch.cuda.synchronize()
    r_out, r_idx, r_ch = O.render(mat, dict(view, footprints=tab), O.SPARSE9, seed=3, want_channels=True)
    assert np.array_equal(idx.cpu().numpy().view(np.uint32), r_idx)
    sens = O.shade_sensitivity(view, r_ch, 8)
    k = np.concatenate([sens, np.zeros(sens.shape[:2] + (1,))], -1)
    ref = r_out.astype(np.float64)
    assert np.all(np.abs(out.cpu().numpy() - ref) <= 1e-5 * np.maximum(np.abs(ref), 1e-3) + 2.0 ** -20 * k)


def test_sparse_neural_material():
    stf = _stf()
    from paper_2504_05562_gb300 import neural
    from test_gpu_neural import _random_decoder, assert_neural_close
    dec, L, P = _random_decoder(neural, tex=128, lat=32, seed=6, scale=0.25)
    tex = dec.texture()
    lat16, w16, b32 = O.nn_pack_inference(L, P)
    mat = O.neural_material(128, 128, lat16, 4, w16, b32)
    tab = _table(2, 4, (8, 4))
    stf.set_sparse_footprints(tab, (8, 4))
    view = W.with_shading(W.screen_aligned_view(96, 64, 128, 128, 3.0, 0, origin=(10.0, 20.0)), "c3")
    out, idx, ch = stf.render(tex, view, stf.MODE_SPARSE9, seed=2, debug=True)
    torch.cuda.synchronize()
    r_out, r_idx, r_ch = O.render(mat, dict(view, footprints=tab), O.SPARSE9, seed=2, want_channels=True)
    assert np.array_equal(idx.cpu().numpy().view(np.uint32), r_idx)
    assert_neural_close(ch.cpu().numpy(), r_ch, "sparse render channels", frac=0.08)


def test_sparse_batch_and_noalloc_equal_single_view_renders():
    stf = _stf()
    tex = stf.Texture(W.material_c3(W.FP16, size=512))
    tab = _table(4, 1, (8, 4))
    stf.set_sparse_footprints(tab, (8, 4))
    views = W.config5_views(n=10, tex=512, seed=6, scale=0.2)
    for i, v in enumerate(views):
        v["tile"] = (0, 0) if i % 2 else (8, 4)
        v["frame"] = i
    outs = [torch.full((v["height"], v["width"], 4), -1.0, device="cuda") for v in views]
    stf.render_views([stf.make_view(v, tex, o) for v, o in zip(views, outs)], stf.FILTER_PER_VIEW, stf.MODE_SPARSE9, 4)
    na = [torch.full((v["height"], v["width"], 4), -1.0, device="cuda") for v in views]
    stf.render_views_noalloc([stf.make_view(v, tex, o) for v, o in zip(views, na)], stf.FILTER_PER_VIEW, stf.MODE_SPARSE9, 4)
    torch.cuda.synchronize()
    for v, o, n in zip(views, outs, na):
        want, _, _ = stf.render(tex, v, stf.MODE_SPARSE9, seed=4)
        torch.cuda.synchronize()
        assert torch.equal(o, want) and torch.equal(n, want)


def test_sparse_mode_needs_matching_patterns():
    stf = _stf()
    tex = stf.Texture(W.material_c1())
    stf.set_sparse_footprints(_table(1, 2, (8, 4)), (8, 4))
    view = dict(W.config1_view(tile=(4, 8)), width=32, height=32)
    with pytest.raises(stf.StfError, match="differs from the sparse footprints"):
        stf.render(tex, view, stf.MODE_SPARSE9)
