"""Key-frame masks built on the GPU (Sec. 4.2.2) against the oracle, and the property that
defines them, through the C ABI."""
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


def _bools(rows, n):
    return np.unpackbits(np.asarray(rows, np.uint8), axis=1, bitorder="little")[:, :n] > 0


def test_keyframe_masks_match_oracle(fd):
    s = scenes.make_scene(700, 31, sh_degree=1, lxyz=(-2.4, 0.4), lt_long=(-1.6, 0.4))
    cams = [scenes.arc_camera(-7.0, 72, 60), scenes.arc_camera(8.0, 60, 72)]
    kt = np.array([0.3, 0.6], np.float32)
    sc = fd.Scene.from_host(s)
    gpu = _bools(sc.build_keyframe_masks(cams, kt).cpu().numpy(), s.n)
    P = oracle.Params.from_scene(s)
    want = np.zeros_like(gpu)
    ex = np.zeros_like(gpu)
    for k, t in enumerate(kt):
        for cam in cams:
            m, e = parity.contribution_exempt(P, cam, parity.f32(t))
            want[k] |= m
            ex[k] |= e | parity.exempt_gaussians(oracle.preprocess(P, cam, parity.f32(t)), cam,
                                                   s.mean4)
    bad = (gpu != want) & ~ex
    print(f"marked {int(want.sum())}, exempt {int(ex.sum())}, mismatches {int((gpu != want).sum())}")
    assert not bad.any(), np.argwhere(bad)[:10]
    assert want.sum() > 50
    sc.close()


def test_filtered_training_views_equal_unfiltered_at_key_times(fd):
    """With the masks built from the training views, a training view rendered at a key-frame
    time through the filter is the unfiltered image, bit for bit (full-size pruned scene)."""
    s = scenes.pruned_scene()
    sc = fd.Scene.from_host(s)
    cams = [scenes.arc_camera(th, 1352, 1014) for th in (-10.0, -3.0, 4.0, 10.0)]
    kt = scenes.keyframe_times(300, 6)
    masks = sc.build_keyframe_masks(cams, kt)
    sc.set_active_mask(masks, kt)
    rows = _bools(masks.cpu().numpy(), s.n)
    ratio = rows.mean(axis=1)
    print(f"active ratio min/median/max {ratio.min():.3f}/{np.median(ratio):.3f}/{ratio.max():.3f}")
    assert 0.0 < ratio.min() and ratio.max() < 1.0
    for k in (0, 17, 49):
        t = float(kt[k])
        for cam in cams:
            full = sc.render(cam, t, use_mask=False)
            filt = sc.render(cam, t, use_mask=True)
            assert torch.equal(full, filt), (k, cam.width)
    sc.close()


def test_batched_masks_equal_one_render_at_a_time(fd):
    """Several key-frames and views go through the batched pipeline (16 renders a batch, the
    last one partial); one key-frame and one view at a time through the per-frame path. The
    blend decisions are the same, so the masks are equal bit for bit."""
    s = scenes.make_scene(5000, 33, sh_degree=1, lxyz=(-2.6, 0.4), lt_long=(-1.4, 0.4))
    cams = [scenes.arc_camera(th, w, h) for th, w, h in ((-9.0, 96, 80), (-1.0, 130, 70),
                                                         (7.0, 64, 112))]
    kt = np.linspace(0.0, 1.0, 7).astype(np.float32)
    sc = fd.Scene.from_host(s)
    batched = sc.build_keyframe_masks(cams, kt).cpu().numpy()
    single = np.zeros_like(batched)
    for k in range(len(kt)):
        for cam in cams:
            single[k] |= sc.build_keyframe_masks([cam], kt[k:k + 1]).cpu().numpy()[0]
    assert np.array_equal(batched, single)
    assert _bools(batched, s.n).sum() > 100
    sc.close()
