"""Blue-noise selection uniforms on the GPU against the CPU oracle (texel choice bit-exact,
channels within the colour bar), for the texture kinds, the neural material and batches. The
masks are made by the host generator and handed to both sides as an input of the selection."""
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


@pytest.mark.parametrize("size", [16, 64])
@pytest.mark.parametrize("mode", [O.ONE_TAP, O.QUAD2, O.WAVE3, O.WAVE3 | O.FLAG_EXACT])
@pytest.mark.parametrize("filt", [0, 1])
def test_blue_noise_parity(size, mode, filt):
    stf = _stf()
    ranks = np.stack([np.random.default_rng(size + c).permutation(size * size).reshape(size, size) for c in range(2)])
    ranks = ranks.astype(np.uint16)
    stf.set_blue_noise(ranks)
    mat = W.material_c1()
    tex = stf.Texture(mat)
    if (mode & O.FLAG_EXACT) and filt == 1:
        mode &= ~O.FLAG_EXACT
    scale = np.maximum(np.abs(W.decoded_reference(mat)).reshape(-1, 4).max(0), 1e-3)
    for frame, seed in ((0, 0), (3, 99), (100, 2 ** 35 + 1)):
        view = dict(W.screen_aligned_view(72, 40, 64, 64, 3.4, filt, origin=(2.6, 5.1)), frame=frame)
        out, idx, ch = stf.render(tex, view, mode | stf.MODE_FLAG_BLUE_NOISE, seed=seed, debug=True)
        torch.cuda.synchronize()
        stf.sync()
        r_out, r_idx, r_ch = O.render(mat, dict(view, blue=ranks), mode | O.FLAG_BLUE, seed=seed, want_channels=True)
        assert np.array_equal(idx.cpu().numpy().view(np.uint32), r_idx)
        g, r = ch.cpu().numpy()[..., :4].astype(np.float64), r_ch[..., :4].astype(np.float64)
        assert np.all(np.abs(g - r) <= 1e-5 * np.maximum(np.abs(r), scale))


def test_blue_noise_neural_and_batch():
    stf = _stf()
    ranks = stf.blue_noise_masks(32, seed=4)
    stf.set_blue_noise(ranks)
    from paper_2504_05562_gb300 import neural
    from test_gpu_neural import _random_decoder
    dec, L, P = _random_decoder(neural, tex=128, lat=32, seed=6, scale=0.25)
    tex = dec.texture()
    view = W.with_shading(W.screen_aligned_view(64, 32, 128, 128, 3.0, 0, origin=(10.0, 20.0)), "c3")
    lat16, w16, b32 = O.nn_pack_inference(L, P)
    mat = O.neural_material(128, 128, lat16, 4, w16, b32)
    _, idx, _ = stf.render(tex, view, O.WAVE3 | stf.MODE_FLAG_BLUE_NOISE, seed=1, debug=True)
    torch.cuda.synchronize()
    _, r_idx, _ = O.render(mat, dict(view, blue=ranks), O.WAVE3 | O.FLAG_BLUE, seed=1)
    assert np.array_equal(idx.cpu().numpy().view(np.uint32), r_idx)
    t16 = stf.Texture(W.material_c3(W.FP16, size=512))
    views = W.config5_views(n=8, tex=512, seed=9, scale=0.2)
    mode = O.WAVE3 | stf.MODE_FLAG_BLUE_NOISE
    outs = [torch.full((v["height"], v["width"], 4), -1.0, device="cuda") for v in views]
    stf.render_views([stf.make_view(v, t16, o) for v, o in zip(views, outs)], stf.FILTER_PER_VIEW, mode, 2)
    torch.cuda.synchronize()
    for v, o in zip(views, outs):
        want, _, _ = stf.render(t16, v, mode, seed=2)
        torch.cuda.synchronize()
        assert torch.equal(o, want)


def test_blue_noise_needs_masks_and_randomness():
    stf = _stf()
    tex = stf.Texture(W.material_c1())
    view = dict(W.config1_view(), width=32, height=32)
    with pytest.raises(stf.StfError, match="full filter"):
        stf.render(tex, view, O.FULL | stf.MODE_FLAG_BLUE_NOISE)
