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


def _check_frame(g, scene, cam, t, active=None, temporal_cull=True, name="frame", tiles=None,
                 pre=None, tile_sets="square"):
    """GPU frame (flags, records, lists, image, T_final, n_contrib) against the oracle, with
    the float32 exemptions of parity.py; reports the counts and returns them."""
    P = oracle.Params.from_scene(scene)
    t = parity.f32(t)                  # the time the GPU received
    if pre is None:
        pre = oracle.preprocess(P, cam, t, active, tile_sets, temporal_cull)
    ref = oracle.render(P, cam, t, active, tiles=tiles, pre=pre)
    ex, why = parity.exempt_gaussians(pre, cam, scene.mean4, detail=True)
    nbad, nex, bad_ids, nex_diff = parity.compare_flags(g["flags"], pre, ex)
    assert nbad == 0, f"{nbad} non-exempt flag mismatches, ids {bad_ids[:10]}"
    st = g["stats"]
    assert st["n_visible"] == int(((g["flags"] & parity.FLAG_VISIBLE) > 0).sum())
    # records of visible Gaussians within their float32 bounds
    b = parity.f32_bounds(pre, cam, scene.mean4)
    vis = pre["visible"].numpy() & ((g["flags"] & parity.FLAG_VISIBLE) > 0)
    rec = g["records"].astype(np.float64)
    m2 = pre["mean2d"].detach().numpy()
    con = pre["conic"].detach().numpy()
    a = pre["a"].detach().numpy()
    z = pre["depth"].detach().numpy()
    ru = np.abs(rec[vis, 0] - m2[vis, 0]) / b["u"][vis]
    rv = np.abs(rec[vis, 1] - m2[vis, 1]) / b["v"][vis]
    # a relative to its bound where it is a normal float32 number with room to spare;
    # below that (no temporal cull: p(t) underflows) the GPU's a must be as small
    av, rav = a[vis], rec[vis, 5]
    big = av >= 1e-30
    ra = np.where(big, np.abs(rav / np.where(big, av, 1.0) - 1) / b["a"][vis],
                  np.where(np.abs(rav) <= 2e-30, 0.0, np.inf))
    rz = np.abs(rec[vis, 9] - z[vis]) / b["z"][vis]
    assert ru.max() <= 1 and rv.max() <= 1 and ra.max() <= 1 and rz.max() <= 1, \
        (ru.max(), rv.max(), ra.max(), rz.max())
    scale = np.sqrt(con[vis, 0] * con[vis, 2])
    cerr = max(np.abs(rec[vis, 2] / con[vis, 0] - 1).max(), np.abs(rec[vis, 4] / con[vis, 2] - 1).max(),
               (np.abs(rec[vis, 3] - con[vis, 1]) / scale).max())
    assert cerr <= parity.CONIC_REL, cerr
    assert np.allclose(rec[vis, 6:9], pre["rgb"].detach().numpy()[vis], rtol=1e-4, atol=1e-5)
    okr = vis & ~ex
    assert np.array_equal(rec[okr, 10], pre["radius"].numpy()[okr])
    # lists: sets and (depth, id) order
    gpu_depth = np.where(vis, rec[:, 9], np.nan)
    lists = parity.compare_tile_lists(g["tile_ranges"], g["tile_ids"], ref["lists"], pre, ex,
                                      gpu_depth, b["z"])
    assert not lists["bad_tiles"], lists["bad_tiles"][:10]
    # image and transmittance
    im = parity.image_metrics(g["image"], ref["image"].numpy())
    assert im["frac_bad"] <= 1e-4 and im["psnr"] >= 60.0, im
    tf = parity.image_metrics(g["T_final"], ref["T_final"].numpy())
    assert tf["frac_bad"] <= 1e-4, tf
    # the last composited entry of every pixel, exactly, outside the exempt pixels
    done = list(ref["lists"].keys())
    gl = {tid: g["tile_ids"][int(g["tile_ranges"][tid, 0]):int(g["tile_ranges"][tid, 1])]
          for tid in done}
    pex, pwhy = parity.pixel_exemptions(pre, ref["lists"], cam, ex, gl, b, detail=True,
                                        rec=(rec, vis))
    lg = parity.last_blended(g["tile_ranges"], g["tile_ids"], g["n_contrib"], done, cam)
    lo = parity.last_blended(None, ref["lists"], ref["n_contrib"].numpy(), done, cam)
    checked = lo != -2
    nc_bad = checked & ~pex & (lg != lo)
    n_pix = int(checked.sum())
    n_act = max(int(pre["pass_mask"].sum()), 1)
    counts = dict(active=n_act, visible=int(pre["visible"].sum()), exempt_gaussians=nex,
                  exempt_by_reason=why, exempt_with_flag_difference=nex_diff,
                  keys_checked=lists["keys"], tiles_checked=lists["tiles"],
                  depth_tie_pairs=lists["tie_pairs"], pixels_checked=n_pix,
                  exempt_pixels=int(pex.sum()), exempt_pixels_by_reason=pwhy,
                  last_entry_differs_on_exempt_pixels=int((checked & pex & (lg != lo)).sum()),
                  max_err_over_f32_bound=dict(u=float(ru.max()), v=float(rv.max()),
                                              a=float(ra.max()), z=float(rz.max())),
                  conic_rel_err=float(cerr), image=im,
                  last_entry_mismatches=int(nc_bad.sum()))
    parity.report(name, **counts)
    assert int(nc_bad.sum()) == 0, (int(nc_bad.sum()), np.argwhere(nc_bad)[:5])
    assert nex <= 0.02 * n_act + 5, (nex, n_act)
    assert int(pex.sum()) <= 0.02 * n_pix + 16, (int(pex.sum()), n_pix)
    return counts


@pytest.mark.parametrize("wh", [(128, 128), (100, 75), (37, 200)])
def test_tiny_render_matches_oracle(fd, wh):
    s = scenes.tiny_scene()
    cam = scenes.tiny_camera(*wh)
    g = _run(fd, s, cam, 0.5)
    _check_frame(g, s, cam, 0.5, name=f"forward tiny {wh[0]}x{wh[1]}")
    assert g["stats"]["n_keys"] > 100


@pytest.mark.parametrize("t", [0.0, 0.31, 1.0])
def test_degree3_timestamps_and_off_centre_camera(fd, t):
    s = scenes.make_scene(3000, 7, sh_degree=3, lt_long=(-1.0, 0.5))
    cam = scenes.arc_camera(8.0, 160, 120)
    g = _run(fd, s, cam, t)
    _check_frame(g, s, cam, t, name=f"forward degree-3 t={t}")


def test_masked_render_gate_is_bit_exact(fd):
    s = scenes.make_scene(4000, 9, sh_degree=1, lt_short=(-4.0, 0.5), lt_long=(-2.0, 0.5),
                          short_frac=0.7)
    kt = scenes.keyframe_times(300, 6)
    masks = scenes.keyframe_masks(s, kt)
    cam = scenes.tiny_camera(96, 80)
    for t in (0.0, 0.5, 0.8, 1.0):
        active = oracle.active_from_masks(masks, [parity.f32(k) for k in kt], parity.f32(t), s.n)
        g = _run(fd, s, cam, t, masks, kt, use_mask=True)
        assert np.array_equal((g["flags"] & parity.FLAG_MASK) > 0, active)
        assert g["stats"]["n_active"] == int(active.sum())
        l, r = oracle.keyframe_pair([parity.f32(k) for k in kt], parity.f32(t))
        assert (g["stats"]["key_l"], g["stats"]["key_r"]) == (l, r)
        _check_frame(g, s, cam, t, active, name=f"forward masked t={t}")


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
    _check_frame(off, s, cam, 0.5, temporal_cull=False, name="forward no temporal cull")


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


@pytest.mark.parametrize("builder,shape", [(1, 0), (1, 2), (1, 3), (1, 4), (1, 5), (1, 6),
                                           (2, 0), (2, 1), (2, 2), (2, 3), (2, 6)])
def test_list_builders_and_blend_shapes_give_identical_frames(fd, builder, shape):
    """Bitmask vs sort tile lists, and the seven launch shapes of the blend (warp footprints
    with their ballot culling, one, two, four or eight pixels per lane), must all give the same lists
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
        fd.set_blend_shape(None)
    assert ref["stats"]["list_builder"] == 1 and g["stats"]["list_builder"] == builder
    for k in ("image", "T_final", "n_contrib", "tile_ranges", "tile_ids"):
        assert np.array_equal(g[k], ref[k]), k


def test_forward_only_blend_equals_the_frame_render(fd):
    """A render that keeps no frame (black background) runs the forward-only blend (T = 0
    stop encoding, paired FP32 evaluation, no transmittance or n_contrib written): for every
    launch shape its image equals, bit for bit, the render that keeps a frame."""
    s = scenes.make_scene(6000, 18, sh_degree=3, lt_long=(-1.0, 0.5))
    sc = fd.Scene.from_host(s)
    try:
        for cam in (scenes.arc_camera(3.0, 200, 150), scenes.tiny_camera(37, 61)):
            ref, fr = sc.render(cam, 0.45, keep_frame=True)
            ref = ref.clone()
            fr.release()
            for shape in range(7):
                fd.set_blend_shape(shape)
                got = sc.render(cam, 0.45)
                assert torch.equal(got, ref), (cam.width, shape)
    finally:
        fd.set_blend_shape(None)
    sc.close()


@pytest.mark.slow
def test_full_size_pruned_masked_frame_sampled_tiles(fd):
    """The benchmark workload (200k pruned scene, 1352x1014, masked, degree-3 SH): full
    frame on the GPU, every Gaussian's flags and record against the oracle, tiles sampled
    (corners, ragged edges, centre, random) for lists, image and last entries."""
    s = scenes.pruned_scene()
    kt = scenes.keyframe_times()
    masks = scenes.keyframe_masks(s, kt)
    cam = scenes.arc_camera(scenes.frame_theta(150))
    t = float(scenes.frame_times()[150])
    g = _run(fd, s, cam, t, masks, kt, use_mask=True)
    active = oracle.active_from_masks(masks, [parity.f32(k) for k in kt], parity.f32(t), s.n)
    P = oracle.Params.from_scene(s)
    pre = oracle.preprocess(P, cam, parity.f32(t), active)
    gx, gy = pre["grid"]
    rng = np.random.default_rng(0)
    tiles = sorted(set([0, gx - 1, gx * (gy - 1), gx * gy - 1, (gy // 2) * gx + gx // 2,
                        (gy // 2) * gx + gx - 1, (gy - 1) * gx + gx // 2] +
                       rng.choice(gx * gy, 5, replace=False).tolist()))
    c = _check_frame(g, s, cam, t, active, name="forward full size 1352x1014 (bench frame)",
                     tiles=tiles, pre=pre)
    assert c["visible"] > 100_000 and c["keys_checked"] > 10_000
