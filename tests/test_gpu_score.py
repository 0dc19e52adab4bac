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


def _variant_factor(P, variant, t):
    """The oracle's per-Gaussian factor that multiplies the blend weight in the score of
    ``variant`` at time t (Eq. 7 and the ablation's variants)."""
    with torch.no_grad():
        cov4 = oracle.covariance_4d(P.logscale4, P.q_left, P.q_right)
        gamma = oracle.volume_gamma(P.logscale4)
        if variant == "spatial":
            return np.ones(P.mean4.shape[0])
        if variant == "first_derivative":
            f = oracle.variation_factor(P.mean4, cov4, float(t), derivative=1) * gamma
        elif variant == "sigma_t":
            f = cov4[:, 3, 3] * gamma
        else:
            f = oracle.variation_factor(P.mean4, cov4, float(t)) * gamma
    return f.numpy()


def _gpu_lists(sc, cam, t):
    """The per-frame GPU render of one view (unmasked): its {tile: ids} lists and its records
    with their visibility, the lists, order and records the score pass's renders share."""
    _, fr = sc.render(cam, float(t), use_mask=False, keep_frame=True)
    ex = fr.export()
    r = parity.to_np(ex["tile_ranges"])
    ids = parity.to_np(ex["tile_ids"]).astype(np.int64)
    rec = parity.to_np(ex["records"]).astype(np.float64)
    vis = (parity.to_np(ex["flags"]) & parity.FLAG_VISIBLE) > 0
    fr.release()
    return {tid: ids[int(r[tid, 0]):int(r[tid, 1])] for tid in range(len(r))}, (rec, vis)


def _score_exemptions(scene, cams, ts, want, lists, variant="full", share=5e-5):
    """Per Gaussian, what the 1e-4 score comparison allows for. Exempt: the exempt Gaussians
    of any render (float32 decisions near a threshold), and the Gaussians that take more than
    ``share`` of their oracle score at the renders' exempt pixels (per-pixel alpha-floor,
    stop, membership and depth-order decisions within float32 reach: the weight there may
    differ by up to all of it). Bound: the first-order float32 error bound of the score
    (the weights' bounds of ``parity.score_pixel_weights`` times the variant's factor, plus
    the rounding of the sums), which takes the place of 1e-4 relative where it is larger.
    ``lists[(t, k)]``: the GPU's tile lists and records of time t, camera k (see
    ``_gpu_lists``). Returns (exempt [N],
    bound [N], counts)."""
    P = oracle.Params.from_scene(scene)
    ex = np.zeros(scene.n, bool)
    E = np.zeros(scene.n)
    R = np.zeros(scene.n)
    pix = dict(exempt_pixels=0, pixels=0, alpha=0, stop=0, member=0, order=0)
    for t in ts:
        g = _variant_factor(P, variant, parity.f32(t))
        for k, cam in enumerate(cams):
            gl, rec = lists[(t, k)]
            e, dec, rnd, c = parity.score_pixel_weights(P, cam, t, gl, rec)
            ex |= e
            E += g * dec
            R += g * rnd
            for key in pix:
                pix[key] += c[key]
    by_pixels = ~ex & (E > share * np.abs(want))
    bound = R + 64 * parity.EPS32 * np.abs(want)
    counts = dict(exempt_gaussians=int(ex.sum()), exempt_by_pixel_weight=int(by_pixels.sum()),
                  f32_bound_above_1e4=int((~ex & ~by_pixels & (bound > 1e-4 * want)).sum()),
                  **pix)
    return ex | by_pixels, bound, counts


def _scores_and_lists(fd, s, cams, ts, batch, variant="full"):
    """GPU scores of the (t, camera) renders and the GPU tile lists of each render."""
    sc = fd.Scene.from_host(s)
    got = parity.to_np(sc.variation_score(cams, ts, batch=batch, variant=variant))
    lists = {(t, k): _gpu_lists(sc, cam, t) for t in ts for k, cam in enumerate(cams)}
    sc.close()
    return got.astype(np.float64), lists


def _compare_scores(got, want, ex, name, bound=None, **extra):
    """max(1e-4 relative, the score's float32 bound) on the significant scores outside the
    exemptions, 1e-6 of the largest score absolute below that; reports the counts."""
    sig = want > 1e-6 * want.max()
    tol = 1e-4 * np.abs(want)
    if bound is not None:
        tol = np.maximum(tol, bound)
    err = np.abs(got - want)
    rel = err / np.maximum(np.abs(want), 1e-30)
    bad = ~ex & sig & (err > tol)
    small = ~ex & ~sig
    small_bad = int((np.abs(got[small] - want[small]) > 1e-6 * want.max() + 1e-12).sum())
    chk = ~ex & sig
    counts = dict(scored=int((want > 0).sum()), checked=int(chk.sum()),
                  exempt=int(ex.sum()), mismatches=int(bad.sum()), small_mismatches=small_bad,
                  max_rel=float(rel[chk].max()),
                  over_1e4=int((chk & (rel > 1e-4)).sum()),
                  max_err_over_tol=float((err[chk] / np.maximum(tol[chk], 1e-300)).max()),
                  **extra)
    parity.report(name, **counts)
    worst = np.argsort(-np.where(chk, err / np.maximum(tol, 1e-300), 0))[:5]
    assert int(bad.sum()) == 0, (counts, [(int(i), float(rel[i]), float(want[i]),
                                           float(tol[i] / max(want[i], 1e-300)))
                                          for i in worst])
    assert small_bad == 0, counts
    assert int(ex.sum()) <= 0.02 * len(want) + 5, counts
    return counts


@pytest.mark.parametrize("batch", [1, 2, 8])
def test_variation_score_matches_oracle(fd, batch):
    """batch 1: one render at a time through the per-frame path; 2 and 8: the batched
    pipeline with the weighted persistent blend (the 9 renders end in a partial batch)."""
    s = scenes.make_scene(3000, 6, sh_degree=3, lt_short=(-4.0, 0.5), lt_long=(-2.0, 0.5),
                          short_frac=0.7)
    cams = [scenes.arc_camera(th, 96, 72) for th in (-10.0, 0.0, 10.0)]
    ts = [0.1, 0.5, 0.77]
    got, lists = _scores_and_lists(fd, s, cams, ts, batch)
    want = oracle.variation_scores(s, cams, [parity.f32(t) for t in ts], "R1")
    ex, bound, c = _score_exemptions(s, cams, ts, want, lists)
    r = _compare_scores(got, want, ex, f"scores 3000 Gaussians batch {batch}", bound, **c)
    assert r["scored"] > 200


@pytest.mark.parametrize("variant", ["spatial", "temporal", "first_derivative", "sigma_t"])
@pytest.mark.parametrize("batch", [1, 8])
def test_score_variants_match_oracle(fd, variant, batch):
    """The score variants of the paper's ablation (Table 4 b-e) through
    fdgs_variation_score_variant, per render (batch 1) and batched (8), against the oracle's
    variants at 1e-4 relative."""
    s = scenes.make_scene(3000, 6, sh_degree=3, lt_short=(-4.0, 0.5), lt_long=(-2.0, 0.5),
                          short_frac=0.7)
    cams = [scenes.arc_camera(th, 96, 72) for th in (-10.0, 0.0, 10.0)]
    ts = [0.1, 0.5, 0.77]
    got, lists = _scores_and_lists(fd, s, cams, ts, batch, variant)
    want = oracle.variation_scores(s, cams, [parity.f32(t) for t in ts], "R1",
                                  variant=variant)
    if variant == "temporal":
        ex, bound, c = np.zeros(s.n, bool), None, {}
    else:
        ex, bound, c = _score_exemptions(s, cams, ts, want, lists, variant)
    r = _compare_scores(got, want, ex, f"score variant {variant} batch {batch}", bound, **c)
    assert r["scored"] > 200


def test_variation_score_at_fifty_thousand_gaussians(fd):
    """A larger score parity case: 50,000 Gaussians of the unpruned lifespan mix, 2 times x 2
    views at 320x240 through the batched pipeline, every tile's weights from the oracle."""
    s = scenes.make_scene(50_000, 61, sh_degree=3, lt_short=(-4.0, 0.5), lt_long=(-2.0, 0.5),
                          short_frac=0.7)
    cams = [scenes.arc_camera(th, 320, 240) for th in (-7.0, 7.0)]
    ts = [0.3, 0.65]
    got, lists = _scores_and_lists(fd, s, cams, ts, 4)
    want = oracle.variation_scores(s, cams, [parity.f32(t) for t in ts], "R1")
    ex, bound, c = _score_exemptions(s, cams, ts, want, lists)
    try:
        r = _compare_scores(got, want, ex, "scores 50000 Gaussians 2 x 2 renders 320x240",
                            bound, **c)
    except AssertionError:
        # per render, the spatial score (the blend weight sums) of the worst Gaussians on both
        # sides, to tell a weight difference from a factor difference
        tol = np.maximum(1e-4 * want, bound)
        worst = np.argsort(-np.where(~ex, np.abs(got - want) / np.maximum(tol, 1e-300), 0))[:4]
        sc = fd.Scene.from_host(s)
        P = oracle.Params.from_scene(s)
        rows = []
        for t in ts:
            for cam in cams:
                gw = parity.to_np(sc.variation_score([cam], [t], batch=1, variant="spatial"))
                ow = oracle.render(P, cam, parity.f32(t), weights=True)["w_sum"].numpy()
                rows.append([(int(i), float(gw[i]), float(ow[i])) for i in worst])
        sc.close()
        parity.report("scores 50000 diagnosis", worst=[int(i) for i in worst],
                      got=[float(got[i]) for i in worst], want=[float(want[i]) for i in worst],
                      per_render_weights=rows)
        raise
    assert r["scored"] > 3000


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
    lists = {(t, k): _gpu_lists(sc, cam, t) for t in ts for k, cam in enumerate(cams)}
    sc.close()
    want_s = oracle.variation_scores(s, cams, [parity.f32(t) for t in ts])
    want = oracle.keep_set(want_s, 0.8)
    order = np.lexsort((np.arange(s.n), want_s))
    cut = want_s[order[int(math.floor(0.8 * s.n))]]
    near = np.abs(want_s - cut) <= 1e-4 * max(cut, 1e-30)
    ex, _, _ = _score_exemptions(s, cams, ts, want_s, lists)
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


def test_score_pass_in_parts_and_resumed_equals_the_whole_pass(fd, tmp_path):
    """fdgs_variation_score_add: a pass split into parts adds up to the whole pass; a pass
    interrupted after its first part and resumed from its checkpoint gives the same scores
    (up to the order of the float sums)."""
    from paper_2503_16422_gb300 import checkpoint
    s = scenes.make_scene(3000, 9, sh_degree=3, lt_short=(-4.0, 0.5), lt_long=(-2.0, 0.5),
                          short_frac=0.7, name="ck")
    sc = fd.Scene.from_host(s)
    cams = [scenes.arc_camera(a, 96, 72) for a in (-8.0, 0.0, 8.0)]
    ts = [0.05, 0.3, 0.55, 0.8, 0.95]
    for batch in (1, 4):
        want = sc.variation_score(cams, ts, batch=batch).cpu().numpy()
        acc = torch.zeros(s.n, dtype=torch.float32, device="cuda")
        for part in checkpoint.parts_of(ts, 2):
            sc.variation_score(cams, part, batch=batch, out=acc, accumulate=True)
        got = acc.cpu().numpy()
        assert np.allclose(got, want, rtol=1e-5, atol=1e-7 * float(want.max()))
    # interrupted after one part (the stand-in raises), then resumed by the library's pass
    path = str(tmp_path / "score.npz")
    parts = checkpoint.parts_of(ts, 2)
    key = checkpoint.pass_key(s.n, cams, ts, "full", 4)

    def first_only(i, scores):
        if i > 0:
            raise RuntimeError("interrupted")
        acc = torch.as_tensor(scores).cuda()
        sc.variation_score(cams, parts[i], batch=4, out=acc, accumulate=True)
        return acc.cpu().numpy()
    with pytest.raises(RuntimeError):
        checkpoint.resumable_pass(path, key, s.n, parts, first_only)
    assert checkpoint.describe(path)["done"] == 1
    got = checkpoint.variation_score_resumable(sc, cams, ts, path, per_part=2, batch=4)
    want = sc.variation_score(cams, ts, batch=4).cpu().numpy()
    assert np.allclose(got.cpu().numpy(), want, rtol=1e-5, atol=1e-7 * float(want.max()))
    assert checkpoint.describe(path)["done"] == len(parts)
    with pytest.raises(ValueError):
        sc.variation_score(cams, ts, accumulate=True)
    sc.close()
