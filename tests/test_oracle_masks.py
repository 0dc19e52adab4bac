"""Pins of the oracle's key-frame masks (Sec. 4.2.2) and active-set metrics (Sec. 4.1), CPU.

The visibility mask of a view is pinned against brute-force per-pixel compositing, and the
key-frame masks against the property that defines them: at a key-frame time, rendering any
training view through the filter gives the unfiltered image (up to the summation order of the
vectorised compositing), and dropping one marked Gaussian changes it."""
import numpy as np
import torch

import brute
import oracle
from paper_2503_16422_gb300 import scenes


def _scene():
    # large, overlapping Gaussians: many pixels saturate, so the stop rule is exercised
    return scenes.make_scene(400, 21, sh_degree=1, lxyz=(-1.2, 0.3), lt_long=(-1.0, 0.3))


def _cams():
    return [scenes.arc_camera(-8.0, 48, 40), scenes.arc_camera(9.0, 40, 48)]


def test_visibility_mask_matches_brute_force_blended_set():
    s = _scene()
    P = oracle.Params.from_scene(s)
    for cam, t in zip(_cams(), (0.3, 0.7)):
        got = oracle.contributing(P, cam, t)
        pre = oracle.preprocess(P, cam, t)
        blended, stoppers = set(), set()
        brute.composite_pixels(
            pre["mean2d"].detach().numpy(), pre["conic"].detach().numpy(),
            pre["a"].detach().numpy(), pre["rgb"].detach().numpy(),
            pre["depth"].detach().numpy(), pre["radius"].numpy(), pre["visible"].numpy(),
            cam.width, cam.height, blended=blended, stoppers=stoppers)
        assert set(np.nonzero(got)[0]) == blended | stoppers
        assert 10 < len(blended) < s.n     # neither vacuous nor everything
        assert stoppers                    # the stop rule is exercised


def _uniform_layers(opacity_logits, depths_z):
    """Isotropic Gaussians far larger than the view (G ~ 1 on every pixel), one per layer,
    centred on the optical axis at the given world z, with a long lifespan around t = 0.5."""
    n = len(depths_z)
    mean4 = np.array([[0.0, 0.0, z, 0.5] for z in depths_z])
    ls = np.tile([np.log(60.0)] * 3 + [np.log(5.0)], (n, 1))
    ident = np.tile([1.0, 0, 0, 0], (n, 1))
    sh = np.full((1, 3, n), 0.3)
    return scenes.Scene(mean4, ls, ident, ident, np.asarray(opacity_logits, np.float64), sh, 0)


def test_a_gaussian_that_only_stops_pixels_is_marked():
    """Front layer blended everywhere at alpha 0.99; the middle layer (alpha 0.99) takes T
    below 1e-4 on every pixel, so it stops each pixel without being blended; the back layer
    (alpha 0.5) is never reached. The mask holds the first two; without the middle one the
    back layer would be blended and the image would change."""
    s = _uniform_layers([9.0, 9.0, 0.0], [1.0, 0.0, -1.0])   # camera at z = 4
    cam = scenes.tiny_camera(32, 32)
    P = oracle.Params.from_scene(s)
    pre = oracle.preprocess(P, cam, 0.5)
    blended, stoppers = set(), set()
    brute.composite_pixels(
        pre["mean2d"].detach().numpy(), pre["conic"].detach().numpy(),
        pre["a"].detach().numpy(), pre["rgb"].detach().numpy(), pre["depth"].detach().numpy(),
        pre["radius"].numpy(), pre["visible"].numpy(), cam.width, cam.height,
        blended=blended, stoppers=stoppers)
    assert blended == {0} and stoppers == {1}
    assert oracle.contributing(P, cam, 0.5).tolist() == [True, True, False]
    masks = oracle.build_keyframe_masks(s, [cam], [0.5])
    assert oracle.mask_row_bools(masks[0], 3).tolist() == [True, True, False]
    full = oracle.render_image(P, cam, 0.5)[0]
    keep = oracle.render_image(P, cam, 0.5, active=np.array([1, 1, 0], bool))[0]
    drop = oracle.render_image(P, cam, 0.5, active=np.array([1, 0, 1], bool))[0]
    assert (keep - full).abs().max() < 1e-12
    assert (drop - full).abs().max() > 1e-6


def test_keyframe_masks_leave_training_views_unchanged_at_key_times():
    s = _scene()
    P = oracle.Params.from_scene(s)
    cams = _cams()
    kt = np.array([0.25, 0.5, 0.75])
    masks = oracle.build_keyframe_masks(s, cams, kt)
    assert masks.shape == (3, (s.n + 7) // 8) and masks.dtype == np.uint8
    for i, t in enumerate(kt):
        union = np.zeros(s.n, bool)
        for cam in cams:
            union |= oracle.contributing(P, cam, t)
        assert np.array_equal(oracle.mask_row_bools(masks[i], s.n), union)
        active = oracle.active_from_masks(masks, kt, float(t), s.n)
        for cam in cams:
            full, _ = oracle.render_image(P, cam, float(t))
            filt, _ = oracle.render_image(P, cam, float(t), active=active)
            # equal up to the summation order of the vectorised compositing (~1e-16)
            assert (full - filt).abs().max() < 1e-12
    # the masks are not vacuous: without one marked Gaussian some training view changes
    t = float(kt[1])
    m = oracle.active_from_masks(masks, kt, t, s.n)
    marked = np.nonzero(oracle.mask_row_bools(masks[1], s.n))[0]
    drop = m.copy()
    drop[marked[len(marked) // 2]] = False
    changed = max(float((oracle.render_image(P, c, t)[0]
                         - oracle.render_image(P, c, t, active=drop)[0]).abs().max())
                  for c in cams)
    assert changed > 1e-9


def test_active_ratio_and_activation_iou():
    n = 37
    a = np.zeros(n, bool)
    a[[0, 3, 8, 9, 36]] = True
    b = np.zeros(n, bool)
    b[[3, 9, 20]] = True
    pa, pb = np.packbits(a, bitorder="little"), np.packbits(b, bitorder="little")
    pz = np.zeros_like(pa)
    assert oracle.active_ratio(pa, n) == 5 / 37
    assert oracle.activation_iou(pa, pa, n) == 1.0
    assert oracle.activation_iou(pa, pz, n) == 0.0
    assert oracle.activation_iou(pz, pz, n) == 1.0
    assert oracle.activation_iou(pa, pb, n) == oracle.activation_iou(pb, pa, n) == 2 / 6
