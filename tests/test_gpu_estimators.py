"""The alternative estimators (IS, MIS, pairwise MIS, regression, each optionally clamped) on the
GPU against the CPU oracle, through the C interface: texel choice bit-exact, filtered channels
within the colour tolerance (both sides evaluate the same sums in the same order)."""
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


@pytest.mark.parametrize("filt", [0, 1])
@pytest.mark.parametrize("mode", [O.QUAD2, O.WAVE3, O.WAVE4])
@pytest.mark.parametrize("est", [O.EST_IS, O.EST_MIS, O.EST_PMIS, O.EST_REG])
@pytest.mark.parametrize("clamp", [False, True])
def test_estimator_parity(filt, mode, est, clamp):
    stf = _stf()
    mat = W.material_c1()
    view = W.screen_aligned_view(72, 44, 64, 64, 3.7, filt, origin=(5.3, 9.1))
    m = O.est_mode(mode, est, clamp)
    out, idx, ch = stf.render(stf.Texture(mat), view, m, seed=5, debug=True)
    torch.cuda.synchronize()
    stf.sync()
    r_out, r_idx, r_ch = O.render(mat, view, m, seed=5, want_channels=True)
    assert np.array_equal(idx.cpu().numpy().view(np.uint32), r_idx)
    g = ch.cpu().numpy()[..., :4].astype(np.float64)
    r = r_ch[..., :4].astype(np.float64)
    scale = np.maximum(np.abs(W.decoded_reference(mat)).reshape(-1, 4).max(0), 1e-3)
    assert np.all(np.abs(g - r) <= 1e-5 * np.maximum(np.abs(r), scale))


def test_estimator_shaded_fp16_material():
    stf = _stf()
    mat = W.material_c3(W.FP16, size=256)
    view = W.with_shading(W.screen_aligned_view(64, 32, 256, 256, 4.0, 0, origin=(3.3, 5.7)), "c3")
    m = O.est_mode(O.WAVE3, O.EST_REG, True)
    out, idx, ch = stf.render(stf.Texture(mat), view, m, seed=1, debug=True)
    torch.cuda.synchronize()
    r_out, r_idx, r_ch = O.render(mat, view, m, seed=1, want_channels=True)
    assert np.array_equal(idx.cpu().numpy().view(np.uint32), r_idx)
    sens = O.shade_sensitivity(view, r_ch, 8)
    k = np.concatenate([sens, np.zeros(sens.shape[:2] + (1,))], -1)
    ref = r_out.astype(np.float64)
    assert np.all(np.abs(out.cpu().numpy() - ref) <= 1e-5 * np.maximum(np.abs(ref), 1e-3) + 2.0 ** -20 * k)


def test_estimator_restrictions():
    stf = _stf()
    L = stf.load()
    mat = W.material_c1()
    tex = stf.Texture(mat)
    m = O.est_mode(O.WAVE3, O.EST_MIS)
    outs = [torch.zeros((16, 16, 4), device="cuda") for _ in range(2)]
    v = W.screen_aligned_view(16, 16, 64, 64, 4.0, 0)
    two = [stf.make_view(v, tex, o) for o in outs]
    with pytest.raises(stf.StfError, match="one view"):
        stf.render_views(two, stf.FILTER_PER_VIEW, m, 0)
    with pytest.raises(stf.StfError, match="8x4"):
        stf.render_views([stf.make_view(dict(v, tile=(4, 8)), tex, outs[0])], stf.FILTER_PER_VIEW, m, 0)
    from paper_2504_05562_gb300 import neural
    dec = neural.Decoder(64, 64, 16, 16, batch=1024, seed=1)
    tn = dec.texture()  # kept alive while its view is in use
    with pytest.raises(stf.StfError, match="stored material"):
        stf.render_views([stf.make_view(v, tn, outs[0])], stf.FILTER_PER_VIEW, m, 0)
    with pytest.raises(stf.StfError, match="weighted estimator"):
        stf.render_views_noalloc([stf.make_view(v, tex, outs[0])], stf.FILTER_PER_VIEW, m, 0)
