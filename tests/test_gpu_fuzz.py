"""Randomised configurations, GPU path against the oracle through the C-ABI.

Each case draws a material kind and size (ragged, not powers of two), a screen-aligned view with
a random size (down to one pixel), magnification (0.1x to 30x, so both minification and strong
magnification), origin (partly outside the texture: clamp-to-edge addressing), tile shape,
filter, sampling mode (exact filtering included), frame and 64-bit seed, with or without
shading. Selected texels must match bit for bit and colours within the parity bar of
test_gpu_parity.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2504_05562_gb300 import workloads as W

from test_gpu_parity import run_both

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KINDS = ["fp32x4", "fp32x8", "fp16x4", "fp16x8", "bf16x8", "e4m3x8", "rgba8+rg16f"]
MODES = [O.ONE_TAP, O.QUAD2, O.WAVE2, O.WAVE3, O.WAVE4, O.FULL]


def random_case(case):
    rng = np.random.default_rng(7000 + case)
    kind = KINDS[case % len(KINDS)]
    tw, th = int(rng.integers(3, 160)), int(rng.integers(3, 160))
    if kind == "rgba8+rg16f":
        tw = th = int(rng.integers(40, 160))
        mat = W.material_c2(size=tw, seed=case)
        nch = 6
    else:
        nch = 4 if kind.endswith("x4") else 8
        ch = np.empty((th, tw, nch), np.float32)
        ch[..., :min(nch, 3)] = rng.uniform(0.0, 1.0, (th, tw, min(nch, 3)))
        if nch == 8:
            ch[..., 3:5] = rng.uniform(-0.6, 0.6, (th, tw, 2))   # normal XY
            ch[..., 5] = rng.uniform(0.2, 0.8, (th, tw))         # roughness
            ch[..., 6] = rng.uniform(0.5, 1.0, (th, tw))         # AO
            ch[..., 7] = rng.uniform(-1.0, 1.0, (th, tw))        # height (signed)
        else:
            ch[..., 3] = rng.uniform(-1.0, 1.0, (th, tw))
        fmt = {"fp32": W.FP32, "fp16": W.FP16, "bf16": W.BF16, "e4m3": W.E4M3}[kind[:4]]
        mat = W.make_material(ch, fmt)
    filt = int(rng.integers(0, 2))
    mag = math.exp(rng.uniform(math.log(0.1), math.log(30.0)))
    w, h = int(rng.integers(1, 97)), int(rng.integers(1, 61))
    origin = (float(rng.uniform(-0.5, 1.2) * tw), float(rng.uniform(-0.5, 1.2) * th))
    tile = [(8, 4), (4, 8), (16, 2)][int(rng.integers(0, 3))]
    view = W.screen_aligned_view(w, h, tw, th, mag, filt, origin=origin, tile=tile,
                                 frame=int(rng.integers(0, 65536)), view_id=int(rng.integers(0, 4)))
    if nch >= 6 and rng.uniform() < 0.6:
        view = W.with_shading(view, "c2" if kind == "rgba8+rg16f" else "c3")
    mode = MODES[int(rng.integers(0, len(MODES)))]
    if filt == 0 and mode not in (O.ONE_TAP, O.FULL) and rng.uniform() < 0.3:
        mode |= O.FLAG_EXACT
    seed = int(rng.integers(0, 2 ** 63)) * 2 + int(rng.integers(0, 2))
    return mat, view, mode, seed


@pytest.mark.parametrize("case", range(42))
def test_random_configuration_matches_oracle(case):
    mat, view, mode, seed = random_case(case)
    run_both(mat, view, mode, seed)


@pytest.mark.parametrize("case", range(12))
def test_random_neural_configuration_matches_oracle(case):
    """Randomised views over an exactly decodable neural material (dyadic latents and sparse
    dyadic weights, so the tensor-core decode equals the oracle's emulation bit for bit): texel
    choice bit-exact and channels within the stored kinds' bar, with a random number of
    persistent pipeline blocks (so blocks run from one to many decode rounds)."""
    from test_gpu_neural import _exact_decoder, _mods
    stf, neural = _mods()
    dec, L, P = _exact_decoder(neural)
    tex = dec.texture()
    lat16, w16, b32 = O.nn_pack_inference(L, P)
    mat = O.neural_material(128, 128, lat16, 4, w16, b32)
    rng = np.random.default_rng(9000 + case)
    filt = int(rng.integers(0, 2))
    mag = math.exp(rng.uniform(math.log(0.2), math.log(12.0)))
    w, h = int(rng.integers(1, 160)), int(rng.integers(1, 96))
    origin = (float(rng.uniform(-20, 120)), float(rng.uniform(-20, 120)))
    tile = [(8, 4), (4, 8), (16, 2)][int(rng.integers(0, 3))]
    view = W.screen_aligned_view(w, h, 128, 128, mag, filt, origin=origin, tile=tile,
                                 frame=int(rng.integers(0, 65536)))
    mode = MODES[int(rng.integers(0, len(MODES)))]
    if filt == 0 and mode not in (O.ONE_TAP, O.FULL) and rng.uniform() < 0.3:
        mode |= O.FLAG_EXACT
    seed = int(rng.integers(0, 2 ** 62))
    stf.set_option(stf.OPT_PIPELINE_BLOCKS, int(rng.integers(1, 7)))
    try:
        out, idx, ch = stf.render(tex, view, mode, seed=seed, debug=True)
        torch.cuda.synchronize()
        stf.sync()
    finally:
        stf.set_option(stf.OPT_PIPELINE_BLOCKS, 0)
    r_out, r_idx, r_ch = O.render(mat, view, mode, seed=seed, want_channels=True)
    if (mode & 15) != O.FULL:
        assert np.array_equal(idx.cpu().numpy().view(np.uint32), r_idx)
    g, r = ch.cpu().numpy().astype(np.float64), r_ch.astype(np.float64)
    assert np.all(np.abs(g - r) <= 1e-5 * np.maximum(np.abs(r), 1.0)), float(np.abs(g - r).max())
