"""The neural decoder's E4M3 inference variant on the GPU (FP8 tensor-core products for layers 2
and 3) against the CPU oracle, through the C interface:

- the power-of-two scalings the library picks equal the oracle's, computed from the same rule;
- decodes agree with the oracle's emulation of the variant (FP32 sums in another order can move
  an activation to the neighbouring E4M3 value, a rare and bounded difference);
- the error against the FP64 decode stays within the first-order E4M3 rounding bound, and its
  size is stated;
- a rendered frame over the E4M3 material matches the same frame over a stored texture that holds
  the oracle's E4M3 decodes (same texel choice, same channels up to those rare differences);
- the choice survives a parameter refresh and switches back to FP16.
"""
import numpy as np
import pytest

import oracle as O
from nn_bounds import e4m3_first_order_bound
from paper_2504_05562_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _mods():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2504_05562_gb300 import neural, stf
    return stf, neural


def _decoder(neural, tex=64, lat=16, seed=3, scale=0.3, lscale=0.5):
    dec = neural.Decoder(tex, tex, lat, lat, batch=1024, seed=seed)
    rng = np.random.default_rng(seed)
    L = rng.normal(0, lscale, (lat, lat, 16)).astype(np.float32)
    P = rng.normal(0, scale, O.NN_PARAMS).astype(np.float32)
    dec.set_params(L, P)
    return dec, L, P


def _all_texels(w, h):
    return np.array([x | (y << 16) for y in range(h) for x in range(w)], np.int32)


def assert_e4m3_close(gpu, ref, bound, what, frac=0.03):
    """Most decodes agree with the emulation to FP32 rounding; the rest (an activation rounded to
    the neighbouring E4M3 value after a differently ordered FP32 sum) stay within twice the
    first-order bound of the variant's rounding error (each side is within it of the FP64 decode)."""
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    err = np.abs(gpu - ref)
    rel = err / (1.0 + np.abs(ref))
    info = "%s: max %.3g, median %.3g, fraction above 1e-5 %.4f" % (what, rel.max(), np.median(rel), np.mean(rel > 1e-5))
    assert np.median(rel) <= 1e-6, info
    assert np.mean(rel > 1e-5) <= frac, info
    assert np.all(err <= 2.0 * bound + 1e-5 * (1.0 + np.abs(ref))), info


@pytest.mark.parametrize("scale,lscale", [(0.3, 0.5), (0.8, 4.0), (0.05, 0.1)])
def test_e4m3_scales_and_decode_match_oracle(scale, lscale):
    stf, neural = _mods()
    dec, L, P = _decoder(neural, seed=int(scale * 10 + lscale), scale=scale, lscale=lscale)
    lat16, _, _ = O.nn_pack_inference(L, P)
    e = dec.set_inference("e4m3")
    assert e == O.nn_e4m3_scales(lat16, P)
    idx = _all_texels(64, 64)
    out = dec.decode(torch.from_numpy(idx).cuda()).cpu().numpy()
    stf.sync()
    ref = O.nn_decode_e4m3(lat16, 4, P, idx)
    latr = lat16.view(np.float16).astype(np.float64)
    bound = e4m3_first_order_bound(latr, 4, P, idx, e)
    assert_e4m3_close(out, ref, bound, "e4m3 decode")


def test_e4m3_error_against_fp64_is_bounded():
    """The variant's error against the FP64 decode of the FP32 parameters and latents: within the
    first-order bound for every texel, and well above the FP16 path's (its precision is stated in
    the benchmark line and the design notes)."""
    stf, neural = _mods()
    dec, L, P = _decoder(neural, seed=8, scale=0.25)
    idx = _all_texels(64, 64)
    t = torch.from_numpy(idx).cuda()
    y16 = dec.decode(t).cpu().numpy().astype(np.float64)
    e = dec.set_inference("e4m3")
    y8 = dec.decode(t).cpu().numpy().astype(np.float64)
    stf.sync()
    y64 = O.nn_decode_f64(L.astype(np.float64), 4, P.astype(np.float64), idx)
    bound = e4m3_first_order_bound(L.astype(np.float64), 4, P, idx, e)
    err8, err16 = np.abs(y8 - y64), np.abs(y16 - y64)
    print("E4M3 decode vs FP64: max %.4g, mean %.4g, rms %.4g (FP16: max %.4g, mean %.4g); mean |y| %.4g"
          % (err8.max(), err8.mean(), np.sqrt(np.mean(err8 ** 2)), err16.max(), err16.mean(), np.abs(y64).mean()))
    assert np.all(err8 <= bound + 1e-6)
    assert err8.mean() > 4 * err16.mean()


def test_e4m3_frame_matches_stored_texture_of_oracle_decodes():
    """WAVE3 over the E4M3 material against WAVE3 over an FP32 texture holding the oracle's E4M3
    decodes of every texel: the texel choice is identical (it never depends on the decode), the
    filtered channels agree where the decodes do."""
    stf, neural = _mods()
    dec, L, P = _decoder(neural, seed=5, scale=0.25)
    lat16, _, _ = O.nn_pack_inference(L, P)
    view = W.screen_aligned_view(96, 64, 64, 64, 3.3, 0, origin=(2.6, 3.1))
    _, idx16, _ = stf.render(dec.texture(), view, O.WAVE3, seed=4, debug=True)
    dec.set_inference("e4m3")
    ntex = dec.texture()
    out, idx, ch = stf.render(ntex, view, O.WAVE3, seed=4, debug=True)
    torch.cuda.synchronize()
    stf.sync()
    texels = O.nn_decode_e4m3(lat16, 4, P, _all_texels(64, 64)).reshape(64, 64, 8)
    stored = stf.Texture(W.make_material(texels.astype(np.float32), W.FP32))
    out_s, idx_s, ch_s = stf.render(stored, view, O.WAVE3, seed=4, debug=True)
    torch.cuda.synchronize()
    assert torch.equal(idx, idx16)
    assert torch.equal(idx, idx_s)
    g, r = ch.cpu().numpy().astype(np.float64), ch_s.cpu().numpy().astype(np.float64)
    rel = np.abs(g - r) / (1.0 + np.abs(r))
    assert np.median(rel) <= 1e-6
    assert np.mean(rel > 1e-5) <= 0.10  # a shared-sample estimate mixes up to 9 decodes
    assert rel.max() <= 0.1


def test_e4m3_survives_refresh_and_switches_back():
    stf, neural = _mods()
    dec, L, P = _decoder(neural, seed=6, scale=0.2)
    e = dec.set_inference("e4m3")
    P2 = P * 2.0
    dec.set_params(L, P2)  # the inference copy is refreshed in the E4M3 variant, scales redone
    lat16, w16, b32 = O.nn_pack_inference(L, P2)
    idx = _all_texels(64, 64)
    t = torch.from_numpy(idx).cuda()
    out = dec.decode(t).cpu().numpy()
    stf.sync()
    e2 = O.nn_e4m3_scales(lat16, P2)
    assert e2 != e
    bound = e4m3_first_order_bound(lat16.view(np.float16).astype(np.float64), 4, P2, idx, e2)
    assert_e4m3_close(out, O.nn_decode_e4m3(lat16, 4, P2, idx), bound, "after set_params")
    assert dec.set_inference("fp16") == [0, 0, 0, 0]
    out16 = dec.decode(t).cpu().numpy().astype(np.float64)
    ref16 = O.nn_decode_f32(lat16, 4, w16, b32, idx).astype(np.float64)
    rel = np.abs(out16 - ref16) / (1.0 + np.abs(ref16))
    assert np.median(rel) <= 1e-6 and rel.max() <= 1e-2
    with pytest.raises(stf.StfError):
        stf._check(stf.load().stf_decoder_set_inference(dec.handle, 7, None))


def test_e4m3_full_size_sampled():
    """The c4 decoder's size (2048^2 texels over a 512^2 x 16 latent grid): the scale exponents from
    the whole grid, and 8192 sampled decodes against the oracle's emulation."""
    stf, neural = _mods()
    dec = neural.Decoder(2048, 2048, 512, 512, batch=65536, seed=12)
    L, P = dec.get_params()
    L = np.ascontiguousarray(L, np.float32).reshape(512, 512, 16)
    P = np.ascontiguousarray(P, np.float32)
    lat16, _, _ = O.nn_pack_inference(L, P)
    e = dec.set_inference("e4m3")
    assert e == O.nn_e4m3_scales(lat16, P)
    rng = np.random.default_rng(12)
    idx = (rng.integers(0, 2048, 8192) | (rng.integers(0, 2048, 8192) << 16)).astype(np.int32)
    out = dec.decode(torch.from_numpy(idx).cuda()).cpu().numpy()
    stf.sync()
    ref = O.nn_decode_e4m3(lat16, 4, P, idx)
    bound = e4m3_first_order_bound(lat16.view(np.float16).astype(np.float64), 4, P, idx, e)
    assert_e4m3_close(out, ref, bound, "e4m3 decode, full size")


def test_e4m3_batch_equals_single_view_renders():
    """The multi-view kernel runs the same decode pipeline: a batch of views over the E4M3 material
    renders exactly as the views do one by one."""
    stf, neural = _mods()
    dec, L, P = _decoder(neural, tex=256, lat=64, seed=9, scale=0.2)
    dec.set_inference("e4m3")
    ntex = dec.texture()
    views = W.config5_views(n=6, tex=256, seed=7, scale=0.15)
    mode = O.WAVE3
    outs = [torch.full((v["height"], v["width"], 4), -1.0, device="cuda") for v in views]
    stf.render_views([stf.make_view(v, ntex, o) for v, o in zip(views, outs)], stf.FILTER_PER_VIEW, mode, 3)
    torch.cuda.synchronize()
    for v, o in zip(views, outs):
        want, _, _ = stf.render(ntex, v, mode, seed=3)
        torch.cuda.synchronize()
        assert torch.equal(o, want)
