"""Pins of the oracle's key-frame masks (Sec. 4.2.2) and active-set metrics (Sec. 4.1), CPU.

The visibility mask of a view is pinned against brute-force per-pixel compositing, and the
key-frame masks against the property that defines them: at a key-frame time, rendering any
training view through the filter gives exactly the unfiltered image, and dropping one marked
Gaussian changes it."""
import numpy as np
import torch

import brute
import oracle
from paper_2503_16422_gb300 import scenes


def _scene():
    return scenes.make_scene(120, 21, sh_degree=1, lxyz=(-2.4, 0.4), lt_long=(-1.6, 0.4))


def _cams():
    return [scenes.arc_camera(-8.0, 48, 40), scenes.arc_camera(9.0, 40, 48)]


def test_visibility_mask_matches_brute_force_blended_set():
    s = _scene()
    P = oracle.Params.from_scene(s)
    for cam, t in zip(_cams(), (0.3, 0.7)):
        got = oracle.contributing(P, cam, t)
        pre = oracle.preprocess(P, cam, t)
        want = set()
        brute.composite_pixels(
            pre["mean2d"].detach().numpy(), pre["conic"].detach().numpy(),
            pre["a"].detach().numpy(), pre["rgb"].detach().numpy(),
            pre["depth"].detach().numpy(), pre["radius"].numpy(), pre["visible"].numpy(),
            cam.width, cam.height, blended=want)
        assert set(np.nonzero(got)[0]) == want
        assert 10 < len(want) < s.n        # neither vacuous nor everything


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
            assert torch.equal(full, filt)
    # the masks are not vacuous: without one marked Gaussian some training view changes
    t = float(kt[1])
    m = oracle.active_from_masks(masks, kt, t, s.n)
    marked = np.nonzero(oracle.mask_row_bools(masks[1], s.n))[0]
    drop = m.copy()
    drop[marked[len(marked) // 2]] = False
    changed = any(not torch.equal(oracle.render_image(P, c, t)[0],
                                  oracle.render_image(P, c, t, active=drop)[0]) for c in cams)
    assert changed


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
