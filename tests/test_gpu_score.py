"""Spatial-Temporal Variation Score and keep-set: CUDA path vs the FP64 oracle."""
import math

import numpy as np
import pytest
import torch

import oracle
import parity
from paper_2503_16422_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fd():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2503_16422_gb300 import build, fdgs
    build.build()
    fdgs.lib()
    return fdgs


def _exempt_union(scene, cams, ts):
    P = oracle.Params.from_scene(scene)
    ex = np.zeros(scene.n, bool)
    for t in ts:
        for cam in cams:
            ex |= parity.exempt_gaussians(oracle.preprocess(P, cam, float(t)), cam)
    return ex


@pytest.mark.parametrize("batch", [1, 2, 8])
def test_variation_score_matches_oracle(fd, batch):
    """batch 1: one render at a time through the per-frame path; 2 and 8: the batched
    pipeline with the weighted persistent blend (the 9 renders end in a partial batch)."""
    s = scenes.make_scene(3000, 6, sh_degree=3, lt_short=(-4.0, 0.5), lt_long=(-2.0, 0.5),
                          short_frac=0.7)
    cams = [scenes.arc_camera(th, 96, 72) for th in (-10.0, 0.0, 10.0)]
    ts = [0.1, 0.5, 0.77]
    sc = fd.Scene.from_host(s)
    got = parity.to_np(sc.variation_score(cams, ts, batch=batch)).astype(np.float64)
    sc.close()
    want, parts = oracle.variation_scores(s, cams, ts, "R1", return_parts=True)
    ex = _exempt_union(s, cams, ts)
    sig = want > 1e-6 * want.max()
    rel = np.abs(got - want) / np.maximum(np.abs(want), 1e-30)
    bad = ~ex & sig & (rel > 1e-4)
    assert int(bad.sum()) == 0, (int(bad.sum()), float(rel[~ex & sig].max()))
    small = ~ex & ~sig
    assert np.all(np.abs(got[small] - want[small]) <= 1e-6 * want.max() + 1e-12)
    assert int((want > 0).sum()) > 200
    print("score parity: max rel", float(rel[~ex & sig].max()), "exempt", int(ex.sum()))


def test_keep_set_is_bit_exact_on_identical_scores(fd):
    rng = np.random.default_rng(2)
    n = 50_000
    s32 = rng.gamma(0.7, 1.0, n).astype(np.float32)
    s32[rng.random(n) < 0.1] = 0.0
    sc = fd.Scene.from_host(scenes.tiny_scene())
    for ratio in (0.0, 0.5, 0.8, 1.0):
        keep = parity.to_np(sc.select_keep(torch.as_tensor(s32).cuda(), ratio)).astype(bool)
        want = oracle.keep_set(s32.astype(np.float64), float(np.float32(ratio)))
        assert np.array_equal(keep, want), ratio
    sc.close()


def test_keep_set_from_gpu_scores_matches_up_to_near_ties(fd):
    s = scenes.make_scene(4000, 16, sh_degree=1, lt_short=(-4.0, 0.5), lt_long=(-2.0, 0.5),
                          short_frac=0.7)
    cams = [scenes.arc_camera(th, 80, 64) for th in (-6.0, 6.0)]
    ts = [0.25, 0.75]
    sc = fd.Scene.from_host(s)
    score = sc.variation_score(cams, ts)
    keep = parity.to_np(sc.select_keep(score, 0.8)).astype(bool)
    sc.close()
    want_s = oracle.variation_scores(s, cams, ts)
    want = oracle.keep_set(want_s, 0.8)
    order = np.lexsort((np.arange(s.n), want_s))
    cut = want_s[order[int(math.floor(0.8 * s.n))]]
    near = np.abs(want_s - cut) <= 1e-4 * max(cut, 1e-30)
    ex = _exempt_union(s, cams, ts)
    diff = (keep != want) & ~near & ~ex
    assert int(diff.sum()) == 0, int(diff.sum())
    assert int((~keep).sum()) == int(math.floor(0.8 * s.n))


def test_batched_score_equals_per_frame_score_and_leaves_renders_alone(fd):
    """The batched score pass against the per-frame one on the same scene (both on the GPU):
    equal up to the summation order of the blend weights; a batched render of the same
    geometry afterwards (graph replay) still gives the per-request images."""
    s = scenes.make_scene(6000, 17, sh_degree=1, lt_short=(-3.0, 0.5), lt_long=(-1.5, 0.5),
                          short_frac=0.5)
    cams = [scenes.arc_camera(th, 120, 88) for th in (-8.0, -2.0, 5.0)]
    ts = [0.2, 0.45, 0.9]
    sc = fd.Scene.from_host(s)
    one = parity.to_np(sc.variation_score(cams, ts, batch=1)).astype(np.float64)
    outs = sc.render_batch(cams, ts[:3], use_mask=False)   # captures this geometry's graph
    many = parity.to_np(sc.variation_score(cams, ts, batch=3)).astype(np.float64)
    sig = one > 1e-6 * one.max()
    rel = np.abs(many - one) / np.maximum(one, 1e-30)
    assert float(rel[sig].max()) <= 1e-5, float(rel[sig].max())
    assert np.all(np.abs(many[~sig] - one[~sig]) <= 1e-6 * one.max())
    again = sc.render_batch(cams, ts[:3], use_mask=False)
    for i in range(3):
        assert torch.equal(again[i], outs[i]), i
        assert torch.equal(again[i], sc.render(cams[i], ts[i], use_mask=False)), i
    sc.close()
