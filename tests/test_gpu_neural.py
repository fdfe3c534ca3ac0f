"""Neural texel decoder on the GPU against the CPU oracle (through the C interface).

- inference (tensor cores, FP16 storage) against the oracle's FP32 emulation of that precision;
- training gradients (FP32) against the oracle's FP64 gradients;
- training reduces the loss and beats a non-learned baseline of equal storage;
- rendering a neural material: texel choice bit-exact, decoded channels within the inference
  tolerance;
- checkpoint / resume is bit-exact.
"""
import numpy as np
import pytest

import oracle as O
from paper_2504_05562_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _mods():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2504_05562_gb300 import neural, stf
    return stf, neural


def _random_decoder(neural, tex=64, lat=16, seed=3, scale=0.3):
    dec = neural.Decoder(tex, tex, lat, lat, batch=1024, seed=seed)
    rng = np.random.default_rng(seed)
    L = rng.normal(0, 0.5, (lat, lat, 16)).astype(np.float32)
    P = rng.normal(0, scale, O.NN_PARAMS).astype(np.float32)
    dec.set_params(L, P)
    return dec, L, P


def _all_texels(w, h):
    return np.array([x | (y << 16) for y in range(h) for x in range(w)], np.int32)


# Inference tolerance. Both sides round the same 24 FP16 inputs; they sum FP32 products in a
# different order (tensor cores), so a hidden activation that lands within a few FP32 ulps of an
# FP16 rounding boundary may round to the neighbouring FP16 value (2^-11 relative), which the
# following layers carry to the output. Most outputs agree to FP32 rounding; a small fraction of
# decodes (about 1 in 200 here) carries such a flip, and a shared-sample estimate combines up to
# 16 decodes, so the fraction of pixels that may exceed 1e-5 grows with the footprint.
def assert_neural_close(gpu, ref, what, frac=0.02):
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    err = np.abs(gpu - ref) / (1.0 + np.abs(ref))
    frac_tight = float(np.mean(err > 1e-5))
    info = "%s: max %.3g, median %.3g, fraction above 1e-5 %.4f" % (what, err.max(), np.median(err), frac_tight)
    assert err.max() <= 1e-2, info
    assert np.median(err) <= 1e-6, info
    assert frac_tight <= frac, info


def test_decode_matches_oracle_emulation():
    stf, neural = _mods()
    dec, L, P = _random_decoder(neural)
    idx = _all_texels(64, 64)
    out = dec.decode(torch.from_numpy(idx).cuda()).cpu().numpy()
    lat16, w16, b32 = O.nn_pack_inference(L, P)
    ref = O.nn_decode_f32(lat16, 4, w16, b32, idx)
    assert_neural_close(out, ref, "decode")
    # a non-multiple of 32 texels, and out-of-range coordinates clamp to the edge: each row of the
    # products is summed independently of the others, so these decodes equal the same texels'
    # rows of the full decode bit for bit (the oracle comparison of those rows is the one above)
    idx2 = np.array([5 | (7 << 16), 63 | (63 << 16), 100 | (3 << 16)], np.int32)
    out2 = dec.decode(torch.from_numpy(idx2).cuda()).cpu().numpy()
    assert np.array_equal(out2, out[[7 * 64 + 5, 63 * 64 + 63, 3 * 64 + 63]])


def test_gradients_match_oracle():
    stf, neural = _mods()
    dec, L, P = _random_decoder(neural, seed=4, scale=0.2)
    src = W.brick_material(64).astype(np.float32)
    tex = stf.Texture(W.make_material(src, W.FP32))
    rng = np.random.default_rng(5)
    idx = np.array([int(x) | (int(y) << 16) for x, y in rng.integers(0, 64, (777, 2))], np.int32)
    loss_g, dP_g, dl_g = dec.gradients(tex, idx)
    loss_o, dP_o, dl_o = O.nn_loss_grad(L.astype(np.float64), 4, P.astype(np.float64), src, idx)
    # FP32 forward and backward against FP64: measured within 2e-7 of the largest component on
    # this case and two others; 1e-5 leaves room for the order of the FP32 sums
    assert abs(loss_g - loss_o) <= 1e-5 * loss_o
    assert np.max(np.abs(dP_g - dP_o)) <= 1e-5 * np.max(np.abs(dP_o))
    assert np.max(np.abs(dl_g - dl_o)) <= 1e-5 * np.max(np.abs(dl_o))
    # the parameters did not move
    L2, P2 = dec.get_params()
    assert np.array_equal(L2, L) and np.array_equal(P2, P)


def _psnr(a, b):
    return 10.0 * np.log10(1.0 / np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))


def _bilinear_baseline(src, R):
    """Non-learned decoder of the same storage: the material box-filtered R x R, 8 channels FP32
    (as many bytes as the 16-channel FP16 latent grid), bilinearly upsampled at the texel centres."""
    t = torch.from_numpy(src).permute(2, 0, 1)[None].double()
    low = torch.nn.functional.avg_pool2d(t, R)
    up = torch.nn.functional.interpolate(low, scale_factor=R, mode="bilinear", align_corners=False)
    return up[0].permute(1, 2, 0).numpy()


def test_training_beats_untrained_and_equal_storage_baseline():
    stf, neural = _mods()
    src = W.brick_material(256).astype(np.float32)
    tex = stf.Texture(W.make_material(src, W.FP32))
    dec = neural.Decoder(256, 256, 64, 64, batch=16384, seed=0)
    idx = torch.from_numpy(_all_texels(256, 256)).cuda()
    before = dec.decode(idx).cpu().numpy().reshape(256, 256, 8)
    losses = dec.train(tex, 600)
    after = dec.decode(idx).cpu().numpy().reshape(256, 256, 8)
    p0, p1 = _psnr(before, src), _psnr(after, src)
    pb = _psnr(_bilinear_baseline(src, 4), src)
    print("neural decoder PSNR: untrained %.2f dB, trained %.2f dB, equal-storage bilinear %.2f dB" % (p0, p1, pb))
    assert np.all(np.isfinite(losses))
    assert losses[-20:].mean() < 0.1 * losses[:5].mean()
    assert p1 > p0 + 10.0
    assert p1 > pb


def test_render_neural_material_parity():
    stf, neural = _mods()
    dec, L, P = _random_decoder(neural, tex=128, lat=32, seed=6, scale=0.25)
    tex = dec.texture()
    lat16, w16, b32 = O.nn_pack_inference(L, P)
    mat = O.neural_material(128, 128, lat16, 4, w16, b32)
    for filt, mode in ((0, O.WAVE3), (1, O.QUAD2), (0, O.ONE_TAP), (0, O.FULL)):
        v = W.with_shading(W.screen_aligned_view(96, 68, 128, 128, 3.0, filt, origin=(10.0, 20.0)), "c3")
        out, idx, ch = stf.render(tex, v, mode, seed=2, debug=True)
        torch.cuda.synchronize()
        stf.sync()
        r_out, r_idx, r_ch = O.render(mat, v, mode, seed=2, want_channels=True)
        if mode != O.FULL:
            assert np.array_equal(idx.cpu().numpy().view(np.uint32), r_idx)
        assert_neural_close(ch.cpu().numpy(), r_ch, "render channels mode %d" % mode, frac=0.08)


def test_checkpoint_resume_is_bit_exact(tmp_path):
    stf, neural = _mods()
    src = W.brick_material(64).astype(np.float32)
    tex = stf.Texture(W.make_material(src, W.FP32))
    a = neural.Decoder(64, 64, 16, 16, batch=2048, seed=7)
    a.train(tex, 10)
    path = tmp_path / "dec.ckpt"
    a.save(path)
    a.train(tex, 10)
    La, Pa = a.get_params()
    b = neural.Decoder.load(path)
    assert b.step == 10
    b.train(tex, 10)
    Lb, Pb = b.get_params()
    assert np.array_equal(La, Lb) and np.array_equal(Pa, Pb)
    c = neural.Decoder(64, 64, 16, 16, batch=2048, seed=7)
    c.train(tex, 20)
    Lc, Pc = c.get_params()
    assert np.array_equal(La, Lc) and np.array_equal(Pa, Pc)


def _exact_decoder(neural, tex=128, lat=32, seed=11):
    """A decoder whose inference is exact on both sides: latents in (1/8)Z, sparse weights in
    (1/8)Z (8 nonzeros per row, the 8 position features unused), biases in (1/64)Z. Every
    interpolated input lies in (1/512)Z, every FP32 sum of the three layers needs at most 24
    significant bits, and the FP16 roundings of exact values are the same on both sides, so the
    GPU's decode equals the oracle's emulation bit for bit whatever the summation order."""
    dec = neural.Decoder(tex, tex, lat, lat, batch=1024, seed=seed)
    rng = np.random.default_rng(seed)
    L = rng.integers(-8, 9, (lat, lat, 16)).astype(np.float32) / 8.0

    def sparse(rows, cols, used):
        W = np.zeros((rows, cols), np.float32)
        for r in range(rows):
            k = rng.choice(used, 8, replace=False)
            W[r, k] = rng.choice([-1.0, 1.0], 8) / 8.0
        return W

    W1, W2, W3 = sparse(64, 24, 16), sparse(64, 64, 64), sparse(8, 64, 64)
    b1, b2, b3 = (rng.integers(-16, 17, n).astype(np.float32) / 64.0 for n in (64, 64, 8))
    P = np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3.ravel(), b3]).astype(np.float32)
    dec.set_params(L, P)
    return dec, L, P


def test_exact_decoder_is_bit_exact():
    stf, neural = _mods()
    dec, L, P = _exact_decoder(neural)
    idx = _all_texels(128, 128)
    out = dec.decode(torch.from_numpy(idx).cuda()).cpu().numpy()
    lat16, w16, b32 = O.nn_pack_inference(L, P)
    ref = O.nn_decode_f32(lat16, 4, w16, b32, idx)
    assert np.array_equal(out, ref)


@pytest.mark.parametrize("filt,mode", [(0, O.QUAD2), (0, O.WAVE2), (0, O.WAVE3), (0, O.WAVE4), (1, O.WAVE3),
                                       (1, O.WAVE4), (0, O.FULL), (1, O.FULL), (0, O.ONE_TAP),
                                       (0, O.WAVE4 | O.FLAG_EXACT), (0, O.SPARSE9)])
def test_render_neural_material_tight(filt, mode):
    """With exactly decodable texels, a neural render matches the oracle within the colour bar of
    the stored kinds (no allowance for decode roundings): sharing, exact filtering and sparse
    footprints over the decode pipeline, with 3 persistent blocks running ~170 rounds each."""
    stf, neural = _mods()
    dec, L, P = _exact_decoder(neural)
    tex = dec.texture()
    lat16, w16, b32 = O.nn_pack_inference(L, P)
    mat = O.neural_material(128, 128, lat16, 4, w16, b32)
    view = W.screen_aligned_view(256, 128, 128, 128, 2.7, filt, origin=(9.3, 17.1))
    extra = {}
    if (mode & 15) == O.SPARSE9:
        rng = np.random.default_rng(4)
        tab = np.array([[[lane] + list(rng.permutation([j for j in range(32) if j != lane])[:8]) for lane in range(32)]
                        for _ in range(2)], np.int8)
        stf.set_sparse_footprints(tab, (8, 4))
        extra["footprints"] = tab
    # few persistent blocks: each runs many decode rounds, reusing its two round slots
    stf.set_option(stf.OPT_PIPELINE_BLOCKS, 3)
    try:
        out, idx, ch = stf.render(tex, view, mode, seed=3, debug=True)
        torch.cuda.synchronize()
        stf.sync()
    finally:
        stf.set_option(stf.OPT_PIPELINE_BLOCKS, 0)
    r_out, r_idx, r_ch = O.render(mat, dict(view, **extra), mode, seed=3, want_channels=True)
    if (mode & 15) != O.FULL:
        assert np.array_equal(idx.cpu().numpy().view(np.uint32), r_idx)
    g, r = ch.cpu().numpy().astype(np.float64), r_ch.astype(np.float64)
    assert np.all(np.abs(g - r) <= 1e-5 * np.maximum(np.abs(r), 1.0)), float(np.abs(g - r).max())


def test_decode_stall_times_out_and_recovers():
    """Failure detection without a device fault: the test switch makes the next decode pipeline
    withhold its first layer-1 products, so the epilogue's bounded wait runs out; every role then
    drains (no TMEM access after the timeout), stf_sync reports STF_ERR_TIMEOUT and clears the
    switch, and the context stays usable: the next decode equals the oracle bit for bit."""
    stf, neural = _mods()
    dec, L, P = _exact_decoder(neural)
    idx = _all_texels(128, 128)
    t = torch.from_numpy(idx).cuda()
    lat16, w16, b32 = O.nn_pack_inference(L, P)
    ref = O.nn_decode_f32(lat16, 4, w16, b32, idx)
    stf.set_option(stf.OPT_TEST_DECODE_STALL, 1)
    try:
        dec.decode(t)
        torch.cuda.synchronize()
        assert stf.load().stf_sync() == stf.ERR_TIMEOUT
        assert "gave up" in stf.last_error()
    finally:
        stf.set_option(stf.OPT_TEST_DECODE_STALL, 0)  # never leave the switch on for later tests
    out = dec.decode(t).cpu().numpy()
    stf.sync()
    assert np.array_equal(out, ref)
