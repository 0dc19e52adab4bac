"""Batched rendering (one device-driven pass, CUDA-graph replay, persistent longest-first
blend) must give exactly the images of per-request fdgs_render calls."""
import numpy as np
import pytest
import torch

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


def _requests(seed, n, resolutions):
    rng = np.random.default_rng(seed)
    cams, ts = [], []
    for i in range(n):
        w, h = resolutions[i % len(resolutions)]
        cams.append(scenes.arc_camera(float(rng.uniform(-10, 10)), w, h))
        ts.append(float(rng.uniform(0, 1)))
    return cams, ts


def _scene_gpu(fd, masked, n=20_000, seed=41):
    s = scenes.make_scene(n, seed, sh_degree=3, lt_short=(-3.0, 0.5), lt_long=(-1.0, 0.5),
                          short_frac=0.5)
    sc = fd.Scene.from_host(s)
    if masked:
        kt = scenes.keyframe_times(300, 6)
        sc.set_active_mask(torch.as_tensor(scenes.keyframe_masks(s, kt)).cuda(), kt)
    return s, sc


@pytest.mark.parametrize("masked", [True, False])
def test_batch_matches_sequential_renders_and_replays(fd, masked):
    _, sc = _scene_gpu(fd, masked)
    res = [(512, 512), (200, 150), (1352, 1014), (37, 61), (800, 800), (1014, 1352), (16, 16)]
    for call, seed in enumerate((1, 2)):           # second call replays the captured graph
        cams, ts = _requests(seed, 7, res)
        outs = sc.render_batch(cams, ts, use_mask=masked)
        torch.cuda.synchronize()
        for i, (c, t) in enumerate(zip(cams, ts)):
            ref = sc.render(c, t, use_mask=masked)
            assert torch.equal(outs[i], ref), (call, i)
        info = sc.batch_info(7)
        lat = np.array(info["latency_ms"])
        assert np.all(lat > 0) and np.all(lat < 10_000)
    sc.close()


def test_batch_autotune_and_background(fd):
    _, sc = _scene_gpu(fd, True, n=8000, seed=43)
    cams, ts = _requests(3, 5, [(320, 240), (240, 320)])
    bg = (0.1, 0.2, 0.3)
    outs = sc.batch_autotune(cams, ts, bg=bg)
    info = sc.batch_info(5)
    assert info["footprint"] in range(7) and info["ctas_per_sm"] >= 1
    outs2 = sc.render_batch(cams, ts, bg=bg)
    for i, (c, t) in enumerate(zip(cams, ts)):
        ref = sc.render(c, t, bg=bg)
        assert torch.equal(outs[i], ref) and torch.equal(outs2[i], ref), i
    sc.close()


def test_batch_autotune_cache(fd, tmp_path):
    """The autotune cache: a miss searches and stores the pick under the batch's key; a hit
    (another scene of a size in the same power-of-two bucket) sets that shape without a
    search, and both give the per-request images."""
    path = str(tmp_path / "shapes.json")
    cams, ts = _requests(5, 4, [(320, 240), (250, 200)])
    _, sc = _scene_gpu(fd, True, n=7000, seed=45)
    try:
        outs = sc.batch_autotune(cams, ts, cache=path)
        assert not sc.autotune_from_cache
        picked = sc.batch_info(4)
        entries = fd.read_autotune_cache(path)
        assert len(entries) == 1
        (key, entry), = entries.items()
        assert entry == {"footprint": picked["footprint"], "ctas_per_sm": picked["ctas_per_sm"]}
        for i, (c, t) in enumerate(zip(cams, ts)):
            assert torch.equal(outs[i], sc.render(c, t)), i
        sc.close()
        _, sc = _scene_gpu(fd, True, n=8000, seed=46)
        sc.set_batch_shape(6 if entry["footprint"] != 6 else 5, 1)
        outs = sc.batch_autotune(cams, ts, cache=path)
        assert sc.autotune_from_cache
        info = sc.batch_info(4)
        assert (info["footprint"], info["ctas_per_sm"]) == (entry["footprint"],
                                                            entry["ctas_per_sm"])
        for i, (c, t) in enumerate(zip(cams, ts)):
            assert torch.equal(outs[i], sc.render(c, t)), i
        sc.batch_autotune(cams, ts, use_mask=False, cache=path)   # another key: a search
        assert not sc.autotune_from_cache
        assert len(fd.read_autotune_cache(path)) == 2
    finally:
        sc.set_batch_shape(6, 0)
        sc.close()


def test_every_batch_shape_gives_the_per_request_images(fd):
    """Each of the seven launch shapes of the batched blend (fdgs_set_batch_shape), at the
    occupancy limit and at a quarter of it, with a black background (the black-only kernel)
    and a coloured one: the images equal the per-request renders, eagerly and on graph
    replay."""
    _, sc = _scene_gpu(fd, True, n=8000, seed=49)
    res = [(200, 150), (33, 17), (96, 96)]
    cams, ts = _requests(14, len(res), res)
    try:
        for bg in ((0.0, 0.0, 0.0), (0.1, 0.2, 0.3)):
            want = [sc.render(c, t, bg=bg).clone() for c, t in zip(cams, ts)]
            for shape in range(7):
                for quarter in (False, True):
                    ctas = 0
                    if quarter:
                        sc.set_batch_shape(shape, 0)
                        sc.render_batch(cams, ts, bg=bg)
                        ctas = max(1, sc.batch_info(len(cams))["ctas_per_sm"] // 4)
                    sc.set_batch_shape(shape, ctas)
                    for call in range(2):        # eager run and capture, then replay
                        outs = sc.render_batch(cams, ts, bg=bg)
                        for i in range(len(cams)):
                            assert torch.equal(outs[i], want[i]), (bg, shape, ctas, call, i)
    finally:
        sc.set_batch_shape(6, 0)
    sc.close()


def test_batch_of_one_and_empty_view(fd):
    _, sc = _scene_gpu(fd, False, n=3000, seed=44)
    away = scenes.look_at_camera((0.0, 0.0, 4.0), 64, 48, target=(0.0, 0.0, 8.0))
    cams = [scenes.arc_camera(2.0, 96, 64), away]
    ts = [0.3, 0.6]
    outs = sc.render_batch(cams, ts, use_mask=False)
    assert torch.equal(outs[0], sc.render(cams[0], 0.3, use_mask=False))
    assert float(outs[1].abs().max()) == 0.0
    one = sc.render_batch(cams[:1], ts[:1], use_mask=False)
    assert torch.equal(one[0], outs[0])
    sc.close()


def _assert_lists_equal_tight_frame(sc, req, cam, t):
    """The batch's tile lists of request ``req`` equal the per-frame alpha-tight lists (the
    same tile rectangles, so the same entries in the same depth order) bit for bit."""
    ranges, ids = sc.batch_tile_lists(req)
    _, fr = sc.render(cam, t, use_mask=True, keep_frame=True, tight=True)
    ex = fr.export()
    torch.cuda.synchronize()
    want_r = ex["tile_ranges"].cpu().numpy().astype(np.uint32)
    want_i = ex["tile_ids"].cpu().numpy().astype(np.uint32)
    fr.release()
    assert ranges.shape == want_r.shape and np.array_equal(ranges, want_r), req
    assert np.array_equal(ids, want_i), req


def test_batch_lists_equal_per_frame_tight_lists_at_ragged_sizes(fd):
    """Mixed resolutions whose tile grids are not multiples of the 4x4 list blocks (and one
    smaller than a block): every request's lists equal its per-frame alpha-tight lists."""
    _, sc = _scene_gpu(fd, True, n=6000, seed=46)
    res = [(200, 150), (33, 17), (64, 48), (250, 130), (40, 40)]
    cams, ts = _requests(11, len(res), res)
    outs = sc.render_batch(cams, ts, use_mask=True)
    for i in range(len(res)):
        assert torch.equal(outs[i], sc.render(cams[i], ts[i], use_mask=True)), i
        _assert_lists_equal_tight_frame(sc, i, cams[i], ts[i])
    with pytest.raises(fd.FdgsError):
        sc.batch_tile_lists(len(res))
    sc.close()


def test_batch_full_size_dense_tiles_match_sequential(fd):
    """200k-Gaussian pruned scene at 1352x1014: tiles hold thousands of entries and the 4x4
    tile blocks of the list builder tens of thousands (rounds of 64 bitmask words overflow
    the per-warp queue and are queued in parts); many tiles stop early. The images must
    equal the per-request renders and the lists the per-frame alpha-tight lists."""
    s = scenes.pruned_scene()
    sc = fd.Scene.from_host(s)
    kt = scenes.keyframe_times(300, 6)
    sc.set_active_mask(torch.as_tensor(scenes.keyframe_masks(s, kt)).cuda(), kt)
    ts = scenes.frame_times()
    ks = (0, 77, 150, 299)
    cams = [scenes.arc_camera(scenes.frame_theta(k), 1352, 1014) for k in ks]
    tt = [float(ts[k]) for k in ks]
    outs = sc.render_batch(cams, tt, use_mask=True)
    counts = sc.batch_counts()
    nv = nk = 0
    for i, (c, t) in enumerate(zip(cams, tt)):
        img, fr = sc.render(c, t, use_mask=True, keep_frame=True)
        assert torch.equal(outs[i], img), i
        st = fr.stats()
        nv += st["n_visible"]
        nk += st["n_keys"]
        fr.release()
        if i < 2:
            _assert_lists_equal_tight_frame(sc, i, c, t)
    # same visibility decisions; the batch's alpha-tight tile sets are subsets of the squares
    assert counts["n_visible"] == nv
    assert 0 < counts["n_keys"] <= nk
    print(f"batch keys {counts['n_keys']} vs per-request 3-sigma keys {nk}")
    sc.close()


def test_batch_of_128_requests_and_the_limit(fd):
    _, sc = _scene_gpu(fd, True, n=6000, seed=45)
    res = [(64, 48), (48, 64), (33, 17), (96, 96)]
    cams, ts = _requests(7, 128, res)
    outs = sc.render_batch(cams, ts, use_mask=True)
    for i in range(0, 128, 9):
        assert torch.equal(outs[i], sc.render(cams[i], ts[i], use_mask=True)), i
    assert len(sc.batch_info(128)["latency_ms"]) == 128
    with pytest.raises(fd.FdgsError):
        sc.render_batch(cams + cams[:1], ts + ts[:1], use_mask=True)
    sc.close()


def test_batch_list_capacity_overflow_regrows_and_reruns(fd):
    """A batch whose block lists exceed the capacity is detected on the device, the lists
    grow and the batch reruns inside the call: images and lists are those of a batch that
    fit (twice: the capacity is reset to 1024 entries before each call)."""
    _, sc = _scene_gpu(fd, True, n=8000, seed=47)
    res = [(200, 150), (96, 96), (250, 130)]
    cams, ts = _requests(12, 6, res)
    want = sc.render_batch(cams, ts, use_mask=True)
    lists = [sc.batch_tile_lists(i) for i in range(len(cams))]
    for attempt in range(2):
        sc.set_batch_list_capacity(1024)
        outs = sc.render_batch(cams, ts, use_mask=True)
        for i in range(len(cams)):
            assert torch.equal(outs[i], want[i]), (attempt, i)
            r, ids = sc.batch_tile_lists(i)
            assert np.array_equal(r, lists[i][0]) and np.array_equal(ids, lists[i][1])
    sc.set_batch_list_capacity(0)
    sc.close()


def test_large_scene_batch_matches_sequential(fd):
    """300k degree-3 Gaussians (78 MB of attributes, more than half of L2): the batched
    preprocess runs partition-major; images still equal the per-request renders."""
    s = scenes.make_scene(300_000, 48, sh_degree=3, lt_short=(-3.0, 0.5), lt_long=(-1.0, 0.5),
                          short_frac=0.5)
    sc = fd.Scene.from_host(s)
    kt = scenes.keyframe_times(300, 6)
    sc.set_active_mask(torch.as_tensor(scenes.keyframe_masks(s, kt)).cuda(), kt)
    cams, ts = _requests(13, 5, [(160, 120), (96, 128), (200, 90)])
    outs = sc.render_batch(cams, ts, use_mask=True)
    for i in range(len(cams)):
        assert torch.equal(outs[i], sc.render(cams[i], ts[i], use_mask=True)), i
    sc.close()


@pytest.mark.slow
def test_bench_batch_configuration_matches_oracle_on_sampled_tiles(fd):
    """The configuration the benchmark times: the pruned 200k scene with the key-frame masks,
    one batch of 64 frames of the 300-frame sequence at 1352x1014 (its stride-7 walk), the
    autotuned launch shape, graph replay. The FP64 oracle renders sampled tiles (corners, the
    centre, random) of three of the 64 frames."""
    import oracle
    import parity
    s = scenes.pruned_scene()
    kt = scenes.keyframe_times()
    masks = scenes.keyframe_masks(s, kt)
    sc = fd.Scene.from_host(s)
    sc.set_active_mask(torch.as_tensor(masks).cuda(), kt)
    ts = scenes.frame_times()
    frames = [(7 * i) % 300 for i in range(64)]
    cams = [scenes.arc_camera(scenes.frame_theta(k), 1352, 1014) for k in frames]
    tt = [float(ts[k]) for k in frames]
    outs = [torch.empty((3, 1014, 1352), dtype=torch.float32, device="cuda") for _ in frames]
    sc.batch_autotune(cams, tt, outs=outs)
    for o in outs:
        o.fill_(float("nan"))
    sc.render_batch(cams, tt, outs=outs)          # replay of the tuned graph
    torch.cuda.synchronize()
    P = oracle.Params.from_scene(s)
    rng = np.random.default_rng(5)
    for i in (0, 31, 63):
        ti = parity.f32(tt[i])
        active = oracle.active_from_masks(masks, [parity.f32(k) for k in kt], ti, s.n)
        pre = oracle.preprocess(P, cams[i], ti, active)
        gx, gy = pre["grid"]
        tiles = sorted(set([0, gx - 1, gx * gy - 1, (gy // 2) * gx + gx // 2] +
                           rng.choice(gx * gy, 3, replace=False).tolist()))
        ref = oracle.render(P, cams[i], ti, active, tiles=tiles, pre=pre)
        im = parity.image_metrics(outs[i].cpu().numpy(), ref["image"].numpy())
        assert im["n"] >= 3 * 48 * len(tiles)     # every sampled tile has at least 8x6 pixels
        assert im["frac_bad"] <= 1e-4 and im["psnr"] >= 60.0, (frames[i], im)
        parity.report(f"batch bench configuration frame {frames[i]}", tiles=len(tiles), **im)
    sc.close()
