"""Multi-view batches (persistent kernel, CUDA-graph replay, autotuner) through the C interface.

Every view of a batch must come out bit-identical to rendering it alone (the same tile code runs
in both kernels), and match the CPU oracle (texel choice bit-exact, colours within tolerance).
"""
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


def _outs(views):
    return [torch.full((v["height"], v["width"], 4), -1.0, device="cuda") for v in views]


def _render_batch(stf, tex_of, views, mode, seed, debug=False):
    outs = _outs(views)
    idxs = [torch.zeros((v["height"], v["width"]), dtype=torch.int32, device="cuda") for v in views] if debug else None
    cv = [stf.make_view(v, tex_of(v), o, idxs[i] if debug else None) for i, (v, o) in enumerate(zip(views, outs))]
    stf.render_views(cv, stf.FILTER_PER_VIEW, mode, seed)
    torch.cuda.synchronize()
    stf.sync()
    return outs, idxs


def _render_each(stf, tex_of, views, mode, seed):
    res = []
    for v in views:
        o, _, _ = stf.render(tex_of(v), v, mode, seed=seed)
        res.append(o)
    torch.cuda.synchronize()
    return res


def _mixed_views(scale=0.2, n=24, seed=1, tex=512):
    views = W.config5_views(n=n, tex=tex, seed=seed, scale=scale)
    tiles = [(8, 4), (4, 8), (16, 2)]
    for i, v in enumerate(views):
        v["tile"] = tiles[i % 3]
    return views


@pytest.mark.parametrize("mode", [1, 2, 4, 5, 0])
def test_batch_equals_single_view_renders(mode):
    stf = _stf()
    tex = stf.Texture(W.material_c3(W.FP16, size=512))
    views = _mixed_views()
    got, _ = _render_batch(stf, lambda v: tex, views, mode, seed=5)
    want = _render_each(stf, lambda v: tex, views, mode, seed=5)
    for g, w in zip(got, want):
        assert torch.equal(g, w)


def test_batch_matches_oracle():
    stf = _stf()
    mat = W.material_c3(W.FP16, size=512)
    tex = stf.Texture(mat)
    views = _mixed_views(n=6)
    got, idxs = _render_batch(stf, lambda v: tex, views, 4, seed=9, debug=True)
    for v, g, ix in zip(views, got, idxs):
        r_out, r_idx, _ = O.render(mat, v, 4, seed=9)
        assert np.array_equal(ix.cpu().numpy().view(np.uint32), r_idx)
        sens = O.shade_sensitivity(v, O.render(mat, v, 4, seed=9, want_channels=True)[2], 8)
        k = np.concatenate([sens, np.zeros(sens.shape[:2] + (1,))], -1)
        ref = r_out.astype(np.float64)
        assert np.all(np.abs(g.cpu().numpy() - ref) <= 1e-5 * np.maximum(np.abs(ref), 1e-3) + 2.0 ** -20 * k)


def test_mixed_material_kinds_and_neural_in_one_batch():
    stf = _stf()
    from paper_2504_05562_gb300 import neural
    t16 = stf.Texture(W.material_c3(W.FP16, size=256))
    t32 = stf.Texture(W.material_c3(W.FP32, size=256))
    dec = neural.Decoder(256, 256, 64, 64, batch=1024, seed=2)
    tn = dec.texture()
    views = _mixed_views(n=9, tex=256, scale=0.15)
    texs = [t16, t32, tn]
    tex_of = {id(v): texs[i % 3] for i, v in enumerate(views)}
    got, _ = _render_batch(stf, lambda v: tex_of[id(v)], views, 3, seed=1)
    want = _render_each(stf, lambda v: tex_of[id(v)], views, 3, seed=1)
    for g, w in zip(got, want):
        assert torch.equal(g, w)


def test_graph_replay_with_new_frames():
    stf = _stf()
    tex = stf.Texture(W.material_c3(W.FP16, size=512))
    views = _mixed_views(n=10)
    b0 = stf.get_stat(stf.STAT_GRAPH_BUILDS)
    for frame in range(4):
        fv = [dict(v, frame=frame) for v in views]
        got, _ = _render_batch(stf, lambda v: tex, fv, 4, seed=3)
        want = _render_each(stf, lambda v: tex, fv, 4, seed=3)
        for g, w in zip(got, want):
            assert torch.equal(g, w)
    # the batch kept its shape: at most one graph per staging buffer was built
    assert stf.get_stat(stf.STAT_GRAPH_BUILDS) - b0 <= 2
    assert stf.get_stat(stf.STAT_GRAPH_REPLAYS) >= 2
    stf.set_option(stf.OPT_BATCH_GRAPHS, 0)
    try:
        got, _ = _render_batch(stf, lambda v: tex, views, 4, seed=3)
        want = _render_each(stf, lambda v: tex, views, 4, seed=3)
        for g, w in zip(got, want):
            assert torch.equal(g, w)
    finally:
        stf.set_option(stf.OPT_BATCH_GRAPHS, 1)


def test_autotuner_choices_are_used_and_persist(tmp_path):
    stf = _stf()
    tex = stf.Texture(W.material_c3(W.FP16, size=512))
    views = W.config5_views(n=8, tex=512, seed=4, scale=0.25)
    for v in views:
        v["tile"] = (0, 0)
    outs = _outs(views)
    cv = [stf.make_view(v, tex, o) for v, o in zip(views, outs)]
    stf.autotune_clear()
    stf.autotune(cv, stf.FILTER_PER_VIEW, 4, 0)
    chosen = [stf.view_config(c, stf.FILTER_PER_VIEW, 4) for c in cv]
    for tw, th, sc in chosen:
        assert (tw, th) in ((8, 4), (4, 8), (16, 2)) and sc in (1, 2, 4, 8)
    got, _ = _render_batch(stf, lambda v: tex, views, 4, seed=6)
    fixed = [dict(v, tile=(tw, th)) for v, (tw, th, _) in zip(views, chosen)]
    want = _render_each(stf, lambda v: tex, fixed, 4, seed=6)
    for g, w in zip(got, want):
        assert torch.equal(g, w)
    path = tmp_path / "tune.txt"
    stf.autotune_save(path)
    stf.autotune_clear()
    assert stf.view_config(cv[0], stf.FILTER_PER_VIEW, 4)[:2] == (8, 4)
    stf.autotune_load(path)
    assert [stf.view_config(c, stf.FILTER_PER_VIEW, 4) for c in cv] == chosen
    stf.autotune_clear()


def test_config5_scaled_batch():
    """The 64-view batch workload at 1/4 resolution: every view equals its single render."""
    stf = _stf()
    tex = stf.Texture(W.material_c3(W.FP16))
    views = W.config5_views(n=64, scale=0.25)
    got, _ = _render_batch(stf, lambda v: tex, views, 4, seed=0)
    want = _render_each(stf, lambda v: tex, views, 4, seed=0)
    for g, w in zip(got, want):
        assert torch.equal(g, w)
