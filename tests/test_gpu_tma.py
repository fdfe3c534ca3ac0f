"""The TMA-staged paired render variant (STF_OPT_TMA_STAGE) against the read-only global path.

Only the source of the texel bytes differs (a shared-memory copy of the block's footprint box,
loaded with cp.async.bulk.tensor, or global memory), so every output must be bit for bit the same:
texel choice, filtered channels and colours. Cases: 16-, 32- and 8-byte texel records (FP16 x 8,
FP32 x 8, E4M3 x 8 with tile scales), the magnified 4K frame, a perspective plane (the corner
bound does not hold everywhere, so far fetches take the global path), a ragged screen, a minified
view (too large a box: nothing staged), and a texture whose row pitch rules out a tensor map.
"""
import numpy as np
import pytest

from paper_2504_05562_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _stf():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2504_05562_gb300 import stf
    return stf


def _both(stf, mat, view, mode, seed=5):
    tex = stf.Texture(mat)
    got = []
    for tma in (0, 1):
        stf.set_option(stf.OPT_TMA_STAGE, tma)
        try:
            out, idx, ch = stf.render(tex, view, mode, seed=seed, debug=True)
            torch.cuda.synchronize()
            stf.sync()
        finally:
            stf.set_option(stf.OPT_TMA_STAGE, 0)
        got.append((out.cpu().numpy(), idx.cpu().numpy(), ch.cpu().numpy()))
    for a, b in zip(got[0], got[1]):
        assert np.array_equal(a, b)


CASES = {
    "fp16 4k": (lambda: W.material_c3(W.FP16), lambda: W.config3_view(0, frame=1)),
    "fp32x8 4x": (lambda: W.material_c3(W.FP32, size=512), lambda: W.config3_view(0, width=480, height=272, tex=512)),
    "e4m3 bspline": (lambda: W.material_c3(W.E4M3, size=512), lambda: W.config3_view(1, width=480, height=272, tex=512)),
    "c2 perspective": (lambda: W.material_c2(size=256), lambda: W.config2_view(width=320, height=180, tex=256, frame=2)),
    "ragged": (lambda: W.material_c1(), lambda: W.screen_aligned_view(250, 123, 64, 64, 3.3, 0, origin=(5.2, 7.9), frame=3)),
    "minified": (lambda: W.material_c1(), lambda: W.screen_aligned_view(128, 64, 64, 64, 0.2, 1, origin=(1.0, 2.0))),
    "odd pitch": (lambda: W.make_material(W.brick_material(65)[..., :4].astype(np.float32), W.FP16),
                  lambda: W.screen_aligned_view(96, 64, 65, 65, 2.5, 0, origin=(3.0, 4.0))),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("mode", [0, 1, 2, 4])
def test_tma_staged_equals_global_fetch(case, mode):
    stf = _stf()
    mat, view = CASES[case][0](), CASES[case][1]()
    _both(stf, mat, view, mode)
