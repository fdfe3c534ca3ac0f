"""Error of every texel precision against the FP64 oracle, and reuse against one-tap on the GPU.

1. Precision. The ground truth is the oracle's FP64 deterministic filter (Eq.
   texture-continuous-sum, Section 2.1) of the FP32 texels, shaded in FP64. The GPU renders the
   same 3840 x 2160 frame over the 2048^2 material stored as FP32, FP16, BF16 and E4M3 (per
   64 x 64 tile and channel scales) with its deterministic filter, and the neural decoder's
   frame. Each result's max abs error and linear-RGB PSNR against the truth are printed and
   bounded:
   - filtered channels: the filter is a convex combination of texels, so storing each texel
     t as q(t) with |q(t) - t| <= u |t| + a moves it by at most u * S_c + a (S_c = the
     channel's largest |texel|, a = the format's subnormal half-spacing); FP32 sums add at
     most 2^-20 S_c;
   - shaded colours: to first order the channel errors move the colour by at most
     sum_k |d rgb / d ch_k| * |d ch_k| <= (u + 2^-20) K, with K the oracle's FP64 sensitivity
     sum_k |d rgb / d ch_k| max(|ch_k|, 1) (every channel of these materials lies in [-1, 1]).
     Shading has kinks (the terminator N.L = 0, the clamps of N.V and N.H), where the
     derivative on one side can be zero, so K is taken as the larger of its values at the true
     and at the GPU's channels (the colour is Lipschitz with that constant across one kink).
     The bound asserted is twice that plus the shading tolerance of the parity tests (the
     second-order terms and the GPU's own shading rounding);
   - the PSNR floor printed beside each measurement is the one those per-pixel bounds imply.
   The neural decoder (FP16 latents, weights and activations, FP32 sums) is compared with the
   oracle's FP64 decoder on the same parameters, texel by texel.
2. Reuse MSE <= one-tap MSE (the paper's bound claim, Eq. stf_error in Section 3; abstract):
   on every configuration the sharing mode's mean squared error against the FP64 full filter,
   over all pixels and several frames, is no larger than one-tap STF's.
"""
import functools

import numpy as np
import pytest

import oracle as O
from paper_2504_05562_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FORMATS = {"fp32": W.FP32, "fp16": W.FP16, "bf16": W.BF16, "e4m3": W.E4M3}
# unit roundoff u and subnormal half-spacing a of each stored format (relative to the tile scale
# for E4M3: the scale maps the tile's largest |value| to 448, so a = 2^-10 * S / 448)
UNIT = {"fp32": 0.0, "fp16": 2.0 ** -11, "bf16": 2.0 ** -8, "e4m3": 2.0 ** -4}
SUB = {"fp32": 0.0, "fp16": 2.0 ** -25, "bf16": 0.0, "e4m3": 2.0 ** -10 / 448.0}
ARITH = 2.0 ** -20  # FP32 sums of up to 16 terms


def _stf():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2504_05562_gb300 import stf
    return stf


def _psnr_from_mse(mse):
    return float("inf") if mse == 0 else 10.0 * np.log10(1.0 / mse)


@functools.lru_cache(maxsize=None)
def _truth_c3(filt):
    """FP64 filter of the FP32 texels and FP64 shading, frame-independent (deterministic)."""
    mat = W.material_c3(W.FP32)
    view = W.config3_view(filt)
    rgb, ch = O.render_exact_f64(mat, view, want_channels=True)
    sens = O.shade_sensitivity(view, ch.astype(np.float32), 8)
    scale = np.abs(W.decoded_reference(mat)).reshape(-1, 8).max(0)
    return rgb, ch, sens, scale


@pytest.mark.parametrize("fmt", list(FORMATS))
def test_c3_precision_against_fp64_oracle(fmt):
    stf = _stf()
    rgb_t, ch_t, sens, S = _truth_c3(0)
    tex = stf.Texture(W.material_c3(FORMATS[fmt]))
    view = W.config3_view(0)
    out, _, ch = stf.render(tex, view, stf.MODE_FULL, seed=0, debug=True)
    torch.cuda.synchronize()
    stf.sync()
    g_ch = ch.cpu().numpy().astype(np.float64)
    g_rgb = out.cpu().numpy().astype(np.float64)[..., :3]
    err_ch = np.abs(g_ch - ch_t)
    bound_ch = (UNIT[fmt] + ARITH) * S + SUB[fmt] * np.maximum(S, 1.0)
    err_rgb = np.abs(g_rgb - rgb_t[..., :3])
    sens = np.maximum(sens, O.shade_sensitivity(view, g_ch.astype(np.float32), 8))
    bound_rgb = 2.0 * (UNIT[fmt] + ARITH) * sens + 2e-5 * np.maximum(np.abs(rgb_t[..., :3]), 1e-3)
    psnr_ch = _psnr_from_mse(float(np.mean(err_ch ** 2)))
    psnr_rgb = _psnr_from_mse(float(np.mean(err_rgb ** 2)))
    floor_rgb = _psnr_from_mse(float(np.mean(bound_rgb ** 2)))
    frac_ch = float(np.max(err_ch / bound_ch))
    frac_rgb = float(np.max(err_rgb / bound_rgb))
    print("precision %s: channels max abs %.3g (PSNR %.2f dB), rgb max abs %.3g PSNR %.2f dB "
          "(floor %.2f dB); worst error / bound: channels %.3f, rgb %.3f"
          % (fmt, err_ch.max(), psnr_ch, err_rgb.max(), psnr_rgb, floor_rgb, frac_ch, frac_rgb))
    assert frac_ch <= 1.0
    assert frac_rgb <= 1.0
    assert psnr_rgb >= floor_rgb


@functools.lru_cache(maxsize=None)
def _trained_decoder():
    """The c4 decoder: the 2048^2 material compressed into 512^2 x 16 FP16 latents and the MLP,
    trained on the GPU for 2,000 steps (seed 0)."""
    stf = _stf()
    from paper_2504_05562_gb300 import neural
    src = W.brick_material(2048).astype(np.float32)
    target = stf.Texture(W.make_material(src, W.FP32))
    dec = neural.Decoder(2048, 2048, 512, 512, batch=65536, seed=0)
    dec.train(target, 2000)
    target.close()
    return dec


def _decode_all(dec):
    n = dec.width * dec.height
    out = torch.empty((n, 8), dtype=torch.float32, device="cuda")
    for c0 in range(0, n, 1 << 21):
        idx = torch.arange(c0, min(n, c0 + (1 << 21)), dtype=torch.int64, device="cuda")
        packed = ((idx % dec.width) | ((idx // dec.width) << 16)).to(torch.int32)
        out[c0:c0 + packed.numel()] = dec.decode(packed)
    return out.view(dec.height, dec.width, 8)


def test_c4_neural_decode_precision_against_fp64_oracle():
    """GPU inference (FP16 latents, weights and hidden activations, FP32 sums) against the
    oracle's FP64 decoder on the same parameters, over 40,000 random texels."""
    _stf()
    dec = _trained_decoder()
    L, P = dec.get_params()
    rng = np.random.default_rng(1)
    xs, ys = rng.integers(0, 2048, 40000), rng.integers(0, 2048, 40000)
    idx = (xs | (ys << 16)).astype(np.int32)
    got = dec.decode(torch.from_numpy(idx).cuda()).cpu().numpy().astype(np.float64)
    ref = O.nn_decode_f64(L.astype(np.float64), 4, P.astype(np.float64), idx)
    err = np.abs(got - ref)
    scale = np.abs(ref).max(0)
    psnr = _psnr_from_mse(float(np.mean(err ** 2)))
    rel = float((err / np.maximum(scale, 1e-3)).max())
    print("neural decode vs FP64: max abs %.3g, max abs / channel scale %.3g, PSNR %.2f dB" % (err.max(), rel, psnr))
    # FP16 rounding of 24 inputs, 6,144 weights and 128 hidden activations (2^-11 relative each),
    # carried through three layers: a few units of 2^-11 of the channel's scale
    assert rel <= 16 * 2.0 ** -11
    assert psnr >= 60.0


def test_c4_neural_frame_precision_against_fp64_filter_of_fp64_decodes():
    """The 4K neural frame's deterministic filter against the FP64 filter of FP64 decodes of the
    texels it covers (the screen-aligned 4x view reads a 961 x 541 texel window)."""
    stf = _stf()
    dec = _trained_decoder()
    L, P = dec.get_params()
    view = W.config3_view(0)
    # texel window under the bilinear supports: uv * 2048 = H[2] * 2048 + (x + 0.5) / 4
    x0, y0 = int(np.floor(view["H"][2] * 2048)) - 2, int(np.floor(view["H"][5] * 2048)) - 2
    x1, y1 = min(2048, x0 + 3840 // 4 + 5), min(2048, y0 + 2160 // 4 + 5)
    x0, y0 = max(0, x0), max(0, y0)
    ys, xs = np.mgrid[y0:y1, x0:x1]
    idx = (xs.ravel() | (ys.ravel() << 16)).astype(np.int32)
    dec64 = O.nn_decode_f64(L.astype(np.float64), 4, P.astype(np.float64), idx).reshape(y1 - y0, x1 - x0, 8)
    full = np.zeros((2048, 2048, 8), np.float32)
    full[y0:y1, x0:x1] = dec64.astype(np.float32)  # texels outside the supports are never read
    mat = W.make_material(full, W.FP32)
    rgb_t, ch_t = O.render_exact_f64(mat, view, want_channels=True)
    out, _, ch = stf.render(dec.texture(), view, stf.MODE_FULL, seed=0, debug=True)
    torch.cuda.synchronize()
    stf.sync()
    err_ch = np.abs(ch.cpu().numpy().astype(np.float64) - ch_t)
    err_rgb = np.abs(out.cpu().numpy().astype(np.float64)[..., :3] - rgb_t[..., :3])
    S = np.abs(dec64).reshape(-1, 8).max(0)
    psnr_rgb = _psnr_from_mse(float(np.mean(err_rgb ** 2)))
    rel = float((err_ch / np.maximum(S, 1e-3)).max())
    print("neural frame vs FP64: channels max abs %.3g (max / scale %.3g), rgb max abs %.3g, PSNR %.2f dB"
          % (err_ch.max(), rel, err_rgb.max(), psnr_rgb))
    assert rel <= 16 * 2.0 ** -11  # a convex combination of decodes: no more than the decode bound
    assert psnr_rgb >= 50.0


# ----------------------------------------------------------------------------- reuse vs one-tap

def _mse_frames(stf, tex, views, truth, mode, frames, seed=0):
    """Mean squared RGB error of `mode` against the per-view truths over all pixels and frames
    (every view of a frame in one stf_render_views call)."""
    se, n = 0.0, 0
    outs = [torch.empty((v["height"], v["width"], 4), device="cuda") for v in views]
    tt = [torch.from_numpy(np.ascontiguousarray(t[..., :3])).cuda() for t in truth]
    for f in frames:
        cvs = [stf.make_view(dict(v, frame=f), tex, o) for v, o in zip(views, outs)]
        stf.render_views(cvs, stf.FILTER_PER_VIEW, mode, seed)
        for o, t in zip(outs, tt):
            se += float(((o[..., :3].double() - t) ** 2).sum())
            n += t.numel()
    torch.cuda.synchronize()
    stf.sync()
    return se / n


def _check_reuse(name, mse_one, mse_reuse):
    print("%s: MSE one-tap %.4g (%.2f dB), reuse %.4g (%.2f dB)"
          % (name, mse_one, _psnr_from_mse(mse_one), mse_reuse, _psnr_from_mse(mse_reuse)))
    assert mse_reuse <= mse_one, "%s: reuse MSE above one-tap MSE" % name


def test_reuse_mse_not_above_one_tap_c2_full_frame():
    """1920 x 1080 perspective ground plane, B-spline, RGBA8 + RG16F, 16 frames."""
    stf = _stf()
    mat = W.material_c2()
    view = W.config2_view()
    truth, _ = O.render_exact_f64(mat, view)
    tex = stf.Texture(mat)
    one = _mse_frames(stf, tex, [view], [truth], stf.MODE_ONE_TAP, range(16))
    for name in ("wave2", "wave3", "wave4"):
        _check_reuse("c2 " + name, one, _mse_frames(stf, tex, [view], [truth], stf.MODE_NAMES[name], range(16)))


@pytest.mark.parametrize("fmt", list(FORMATS))
def test_reuse_mse_not_above_one_tap_c3_formats(fmt):
    """3840 x 2160 at 4x over the 2048^2 material in each stored format: bilinear QUAD2 and
    WAVE3, B-spline WAVE3, 3 frames each, against the FP64 filter of the FP32 texels."""
    stf = _stf()
    tex = stf.Texture(W.material_c3(FORMATS[fmt]))
    for filt, modes in ((0, ("quad2", "wave3")), (1, ("wave3",))):
        truth = _truth_c3(filt)[0]
        view = W.config3_view(filt)
        one = _mse_frames(stf, tex, [view], [truth], stf.MODE_ONE_TAP, range(3))
        for name in modes:
            got = _mse_frames(stf, tex, [view], [truth], stf.MODE_NAMES[name], range(3))
            _check_reuse("c3 %s filter %d %s" % (fmt, filt, name), one, got)


def test_reuse_mse_not_above_one_tap_c4_neural():
    """The 4K neural frame, WAVE3 and QUAD2 against the FP64 filter of the decoded texels."""
    stf = _stf()
    dec = _trained_decoder()
    decoded = _decode_all(dec).cpu().numpy()
    view = W.config3_view(0)
    truth, _ = O.render_exact_f64(W.make_material(decoded, W.FP32), view)
    ntex = dec.texture()
    one = _mse_frames(stf, ntex, [view], [truth], stf.MODE_ONE_TAP, range(3))
    for name in ("quad2", "wave3"):
        _check_reuse("c4 " + name, one, _mse_frames(stf, ntex, [view], [truth], stf.MODE_NAMES[name], range(3)))


def test_reuse_mse_not_above_one_tap_c5_batch():
    """The 64-view batch (resolutions scaled by 1/4 so that the FP64 truth stays quick), FP16
    material, one persistent launch per frame, 2 frames."""
    stf = _stf()
    mat = W.material_c3(W.FP16)
    views = W.config5_views(64, scale=0.25)
    truths = [O.render_exact_f64(mat, v)[0] for v in views]
    tex = stf.Texture(mat)
    one = _mse_frames(stf, tex, views, truths, stf.MODE_ONE_TAP, range(2))
    _check_reuse("c5 wave3", one, _mse_frames(stf, tex, views, truths, stf.MODE_WAVE3, range(2)))
