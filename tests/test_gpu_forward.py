"""Forward parity: CUDA path (through the C ABI) vs the FP64 oracle."""
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


def _run(fd, scene, cam, t, masks=None, key_times=None, use_mask=False, temporal_cull=True):
    sc = fd.Scene.from_host(scene)
    if masks is not None:
        sc.set_active_mask(torch.as_tensor(masks).cuda(), key_times)
    img, fr = sc.render(cam, t, use_mask=use_mask, keep_frame=True, temporal_cull=temporal_cull)
    ex = fr.export()
    torch.cuda.synchronize()
    out = {k: parity.to_np(v) if isinstance(v, torch.Tensor) else v for k, v in ex.items()}
    out["image"] = parity.to_np(img)
    fr.release()
    sc.close()
    return out


def _check_frame(g, scene, cam, t, active=None, strict_image=True, temporal_cull=True):
    P = oracle.Params.from_scene(scene)
    ref = oracle.render(P, cam, t, active, temporal_cull=temporal_cull)
    pre = ref["pre"]
    ex = parity.exempt_gaussians(pre, cam)
    nbad, nex, bad_ids = parity.compare_flags(g["flags"], pre, ex)
    assert nbad == 0, f"{nbad} non-exempt flag mismatches, ids {bad_ids[:10]}"
    st = g["stats"]
    assert st["n_visible"] == int(((g["flags"] & parity.FLAG_VISIBLE) > 0).sum())
    lists = parity.compare_tile_lists(g["tile_ranges"], g["tile_ids"], ref["lists"], pre, ex)
    assert not lists["bad_tiles"], lists["bad_tiles"][:10]
    # records of visible Gaussians
    vis = pre["visible"].numpy() & ~ex
    rec = g["records"][vis]
    m2 = pre["mean2d"].detach().numpy()[vis]
    con = pre["conic"].detach().numpy()[vis]
    assert np.abs(rec[:, 0:2] - m2).max() < 2e-3
    assert np.allclose(rec[:, 2:5], con, rtol=2e-3, atol=1e-6)
    assert np.allclose(rec[:, 5], pre["a"].detach().numpy()[vis], rtol=1e-4, atol=1e-7)
    assert np.allclose(rec[:, 6:9], pre["rgb"].detach().numpy()[vis], rtol=1e-4, atol=1e-5)
    assert np.allclose(rec[:, 9], pre["depth"].detach().numpy()[vis], rtol=1e-5)
    assert np.array_equal(rec[:, 10], pre["radius"].numpy()[vis])
    # image
    im = parity.image_metrics(g["image"], ref["image"].numpy())
    assert im["frac_bad"] <= 1e-4 and im["psnr"] >= 60.0, im
    tf = parity.image_metrics(g["T_final"], ref["T_final"].numpy())
    assert tf["frac_bad"] <= 1e-4, tf
    nc_eq = (g["n_contrib"] == ref["n_contrib"].numpy()).mean()
    assert nc_eq >= 0.999, nc_eq
    return dict(exempt=nex, image=im, nc_eq=float(nc_eq))


@pytest.mark.parametrize("wh", [(128, 128), (100, 75), (37, 200)])
def test_tiny_render_matches_oracle(fd, wh):
    s = scenes.tiny_scene()
    cam = scenes.tiny_camera(*wh)
    g = _run(fd, s, cam, 0.5)
    info = _check_frame(g, s, cam, 0.5)
    assert g["stats"]["n_keys"] > 100
    print("tiny", wh, info)


@pytest.mark.parametrize("t", [0.0, 0.31, 1.0])
def test_degree3_timestamps_and_off_centre_camera(fd, t):
    s = scenes.make_scene(3000, 7, sh_degree=3, lt_long=(-1.0, 0.5))
    cam = scenes.arc_camera(8.0, 160, 120)
    g = _run(fd, s, cam, t)
    _check_frame(g, s, cam, t)


def test_masked_render_gate_is_bit_exact(fd):
    s = scenes.make_scene(4000, 9, sh_degree=1, lt_short=(-4.0, 0.5), lt_long=(-2.0, 0.5),
                          short_frac=0.7)
    kt = scenes.keyframe_times(300, 6)
    masks = scenes.keyframe_masks(s, kt)
    cam = scenes.tiny_camera(96, 80)
    for t in (0.0, 0.5, 0.8, 1.0):
        active = oracle.active_from_masks(masks, kt, t, s.n)
        g = _run(fd, s, cam, t, masks, kt, use_mask=True)
        assert np.array_equal((g["flags"] & parity.FLAG_MASK) > 0, active)
        assert g["stats"]["n_active"] == int(active.sum())
        l, r = oracle.keyframe_pair(kt, t)
        assert (g["stats"]["key_l"], g["stats"]["key_r"]) == (l, r)
        _check_frame(g, s, cam, t, active)


def test_all_ones_mask_equals_unmasked_and_all_zeros_is_black(fd):
    s = scenes.tiny_scene()
    cam = scenes.tiny_camera(64, 64)
    ones = np.stack([scenes.pack_bits(np.ones(s.n, bool))] * 3)
    zeros = np.stack([scenes.pack_bits(np.zeros(s.n, bool))] * 3)
    kt = [0.0, 0.5, 1.0]
    g0 = _run(fd, s, cam, 0.5)
    g1 = _run(fd, s, cam, 0.5, ones, kt, use_mask=True)
    assert np.array_equal(g0["image"], g1["image"])
    assert np.array_equal(g0["n_contrib"], g1["n_contrib"])
    gz = _run(fd, s, cam, 0.5, zeros, kt, use_mask=True)
    assert np.abs(gz["image"]).max() == 0.0
    assert gz["stats"]["n_keys"] == 0 and gz["stats"]["n_active"] == 0
    assert np.all(gz["T_final"] == 1.0)


def test_no_temporal_cull_gives_the_same_image_with_longer_lists(fd):
    """Without the exact a < 1/255 cull (the comparison renderer of the paper's speed-up) the
    lists carry the Gaussians the cull would drop; the image and transmittance are the same
    bit for bit, and flags and lists match the oracle run the same way."""
    s = scenes.make_scene(4000, 9, sh_degree=1, lt_short=(-4.0, 0.5), lt_long=(-2.0, 0.5),
                          short_frac=0.7)
    cam = scenes.tiny_camera(96, 80)
    on = _run(fd, s, cam, 0.5)
    off = _run(fd, s, cam, 0.5, temporal_cull=False)
    assert np.array_equal(on["image"], off["image"])
    assert np.array_equal(on["T_final"], off["T_final"])
    assert off["stats"]["n_visible"] > on["stats"]["n_visible"]
    assert off["stats"]["n_keys"] > on["stats"]["n_keys"]
    _check_frame(off, s, cam, 0.5, temporal_cull=False)


def test_empty_and_fully_culled_scenes(fd):
    s = scenes.tiny_scene().subset(np.arange(0))
    cam = scenes.tiny_camera(40, 30)
    g = _run(fd, s, cam, 0.5)
    assert np.abs(g["image"]).max() == 0.0 and g["stats"]["n_keys"] == 0
    # camera looking away from the scene: everything behind the near plane
    s = scenes.tiny_scene()
    cam = scenes.look_at_camera((0.0, 0.0, 4.0), 48, 48, target=(0.0, 0.0, 8.0))
    g = _run(fd, s, cam, 0.5)
    assert g["stats"]["n_visible"] == 0 and np.abs(g["image"]).max() == 0.0


def test_background_colour(fd):
    s = scenes.tiny_scene()
    cam = scenes.tiny_camera(64, 48)
    sc = fd.Scene.from_host(s)
    bg = (0.2, 0.5, 1.0)
    img0 = sc.render(cam, 0.5)
    img1, fr = sc.render(cam, 0.5, bg=bg, keep_frame=True)
    ex = fr.export()
    Tf = ex["T_final"]
    want = img0 + Tf[None] * torch.tensor(bg, device="cuda")[:, None, None]
    assert torch.allclose(img1, want, atol=1e-6)
    fr.release()
    sc.close()


@pytest.mark.parametrize("builder,shape", [(1, 0), (1, 2), (1, 3), (1, 4), (1, 5), (2, 0),
                                           (2, 1), (2, 2), (2, 3)])
def test_list_builders_and_blend_shapes_give_identical_frames(fd, builder, shape):
    """Bitmask vs sort tile lists, and the six launch shapes of the blend (warp footprints
    with their ballot culling, one, two or four pixels per lane), must all give the same lists
    and bit-identical images, transmittances and n_contrib."""
    s = scenes.make_scene(6000, 17, sh_degree=1, lt_long=(-1.0, 0.5))
    cam = scenes.arc_camera(4.0, 200, 150)
    fd.set_list_builder(1)
    fd.set_blend_shape(1)   # one pixel per lane, 8x4 footprint: the reference shape
    try:
        ref = _run(fd, s, cam, 0.4)
        fd.set_list_builder(builder)
        fd.set_blend_shape(shape)
        g = _run(fd, s, cam, 0.4)
    finally:
        fd.set_list_builder(0)
        fd.set_blend_shape(fd.DEFAULT_BLEND_SHAPE)
    assert ref["stats"]["list_builder"] == 1 and g["stats"]["list_builder"] == builder
    for k in ("image", "T_final", "n_contrib", "tile_ranges", "tile_ids"):
        assert np.array_equal(g[k], ref[k]), k


@pytest.mark.slow
def test_full_size_pruned_masked_frame_sampled_tiles(fd):
    """The benchmark workload (200k pruned scene, 1352x1014, masked, degree-3 SH): full
    frame on the GPU, oracle on sampled tiles (corners, ragged edges, centre, random)."""
    s = scenes.pruned_scene()
    kt = scenes.keyframe_times()
    masks = scenes.keyframe_masks(s, kt)
    cam = scenes.arc_camera(scenes.frame_theta(150))
    t = float(scenes.frame_times()[150])
    g = _run(fd, s, cam, t, masks, kt, use_mask=True)
    active = oracle.active_from_masks(masks, kt, t, s.n)
    P = oracle.Params.from_scene(s)
    pre = oracle.preprocess(P, cam, t, active)
    gx, gy = pre["grid"]
    rng = np.random.default_rng(0)
    tiles = sorted(set([0, gx - 1, gx * (gy - 1), gx * gy - 1, (gy // 2) * gx + gx // 2,
                        (gy // 2) * gx + gx - 1, (gy - 1) * gx + gx // 2] +
                       rng.choice(gx * gy, 5, replace=False).tolist()))
    ref = oracle.render(P, cam, t, active, tiles=tiles, pre=pre)
    ex = parity.exempt_gaussians(pre, cam)
    nbad, nex, _ = parity.compare_flags(g["flags"], pre, ex)
    assert nbad == 0
    lists = parity.compare_tile_lists(g["tile_ranges"], g["tile_ids"], ref["lists"], pre, ex)
    assert not lists["bad_tiles"], lists["bad_tiles"]
    im = parity.image_metrics(g["image"], ref["image"].numpy())
    assert im["frac_bad"] <= 1e-4 and im["psnr"] >= 60.0, im
    print("full-size sampled:", dict(exempt=nex, keys_checked=lists["keys"], **im))
