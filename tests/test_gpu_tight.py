"""Alpha-tight tile sets through the per-frame C ABI (fdgs_render_opts.tile_sets = 1): lists
match the oracle's tight lists, images equal the 3-sigma-square renders bit for bit, and
gradients equal them up to the order of the atomic accumulation."""
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


@pytest.mark.parametrize("wh", [(128, 128), (100, 75)])
def test_tight_lists_match_oracle_and_images_equal_square(fd, wh):
    s = scenes.tiny_scene()
    cam = scenes.tiny_camera(*wh)
    sc = fd.Scene.from_host(s)
    sq = sc.render(cam, 0.5, use_mask=False)
    img, fr = sc.render(cam, 0.5, use_mask=False, keep_frame=True, tight=True)
    ex = {k: parity.to_np(v) if isinstance(v, torch.Tensor) else v for k, v in fr.export().items()}
    fr.release()
    assert torch.equal(img, sq)
    P = oracle.Params.from_scene(s)
    ref = oracle.render(P, cam, 0.5, tile_sets="tight")
    pre = ref["pre"]
    exempt, why = parity.exempt_gaussians(pre, cam, s.mean4, detail=True)
    b = parity.f32_bounds(pre, cam, s.mean4)
    vis = (ex["flags"] & parity.FLAG_VISIBLE) > 0
    depth = np.where(vis, ex["records"][:, 9].astype(np.float64), np.nan)
    lists = parity.compare_tile_lists(ex["tile_ranges"], ex["tile_ids"], ref["lists"], pre,
                                      exempt, depth, b["z"])
    assert not lists["bad_tiles"], lists["bad_tiles"][:10]
    assert int(exempt.sum()) <= 0.02 * s.n + 5
    parity.report(f"tight lists {wh[0]}x{wh[1]}", exempt_gaussians=int(exempt.sum()),
                  exempt_by_reason=why, keys_checked=lists["keys"],
                  depth_tie_pairs=lists["tie_pairs"])
    n_sq = sum(len(v) for v in oracle.render(P, cam, 0.5)["lists"].values())
    assert ex["stats"]["n_keys"] < n_sq
    sc.close()


@pytest.mark.parametrize("builder", [1, 2])
def test_tight_full_size_images_equal_square(fd, builder):
    s = scenes.pruned_scene()
    sc = fd.Scene.from_host(s)
    kt = scenes.keyframe_times(300, 6)
    sc.set_active_mask(torch.as_tensor(scenes.keyframe_masks(s, kt)).cuda(), kt)
    ts = scenes.frame_times()
    fd.set_list_builder(builder)
    try:
        for k, masked in ((20, True), (150, False)):
            cam = scenes.arc_camera(scenes.frame_theta(k), 1352, 1014)
            a, fa = sc.render(cam, float(ts[k]), use_mask=masked, keep_frame=True)
            b, fb = sc.render(cam, float(ts[k]), use_mask=masked, keep_frame=True, tight=True)
            assert torch.equal(a, b), (k, builder)
            ka, kb = fa.stats()["n_keys"], fb.stats()["n_keys"]
            assert kb < 0.6 * ka, (ka, kb)
            fa.release()
            fb.release()
    finally:
        fd.set_list_builder(0)
    sc.close()


def test_tight_gradients_equal_square(fd):
    s = scenes.pruned_scene(20_000, 7)
    sc = fd.Scene.from_host(s)
    cam = scenes.arc_camera(3.0, 256, 192)
    target = torch.rand(3, 192, 256, device="cuda")
    grads = []
    for tight in (False, True):
        img, fr = sc.render(cam, 0.4, use_mask=False, keep_frame=True, tight=tight)
        dL = torch.sign(img - target) / img.numel()
        g = sc.render_backward(fr, dL)
        fr.release()
        grads.append([x.clone() for x in g.list()])
    for a, b in zip(*grads):
        scale = float(a.abs().max())
        assert scale > 0
        assert float((a - b).abs().max()) <= 1e-5 * scale + 1e-12
    sc.close()
