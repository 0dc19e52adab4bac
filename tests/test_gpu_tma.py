"""Record staging of the batched blend by TMA (cp.async.bulk.tensor tile::gather4 into
mbarrier-completed buffers) against the per-thread cp.async staging: the same images bit for
bit, the same per-request renders, the same counts, and scores equal up to the order of
their float sums."""
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
    yield fdgs
    fdgs.set_batch_staging(fdgs.STAGING_CP_ASYNC)


def _requests(seed, n, resolutions):
    rng = np.random.default_rng(seed)
    cams, ts = [], []
    for i in range(n):
        w, h = resolutions[i % len(resolutions)]
        cams.append(scenes.arc_camera(float(rng.uniform(-10, 10)), w, h))
        ts.append(float(rng.uniform(0, 1)))
    return cams, ts


def _masked_scene(fd, n, seed):
    s = scenes.make_scene(n, seed, sh_degree=3, lt_short=(-3.0, 0.5), lt_long=(-1.0, 0.5),
                          short_frac=0.5)
    sc = fd.Scene.from_host(s)
    sc.set_batch_shape(5, 0)     # the gather4 staging is built for four pixels a lane
    kt = scenes.keyframe_times(300, 6)
    sc.set_active_mask(torch.as_tensor(scenes.keyframe_masks(s, kt)).cuda(), kt)
    return s, sc


def _batch(fd, sc, mode, cams, ts, **kw):
    fd.set_batch_staging(mode)
    outs = sc.render_batch(cams, ts, **kw)
    torch.cuda.synchronize()
    return [o.clone() for o in outs]


def test_gather4_staging_equals_cp_async_and_per_request_renders(fd):
    """Mixed and ragged resolutions (tile grids that are not multiples of the 4x4 list
    blocks, lists shorter than a stage and many stages long), masked, black background (the
    T = 0 blend) and a coloured one; twice each (the second call replays the graph, which
    was re-captured for the new staging)."""
    _, sc = _masked_scene(fd, 20_000, 51)
    res = [(512, 512), (200, 150), (1352, 1014), (37, 61), (800, 800), (16, 16)]
    cams, ts = _requests(5, len(res), res)
    for shape in (4, 5):
        sc.set_batch_shape(shape, 0)
        for bg in ((0.0, 0.0, 0.0), (0.2, 0.1, 0.05)):
            want = _batch(fd, sc, fd.STAGING_CP_ASYNC, cams, ts, bg=bg)
            for call in range(2):
                got = _batch(fd, sc, fd.STAGING_TMA, cams, ts, bg=bg)
                for i in range(len(cams)):
                    assert torch.equal(got[i], want[i]), (shape, bg, call, i)
        for i, (c, t) in enumerate(zip(cams, ts)):
            assert torch.equal(want[i], sc.render(c, t, bg=bg)), (bg, i)
    sc.status_sync()
    sc.close()


def test_gather4_staging_on_the_full_size_scene(fd):
    """The 200k pruned scene at 1352x1014 (thousands of entries per tile, many stages per
    tile, early exits of saturated tiles with a stage in flight), four frames, through shape 5
    and through the autotuned shape (which may be one without TMA staging); the counting
    variant of the kernel gives the same evaluation counts under either staging."""
    s = scenes.pruned_scene()
    sc = fd.Scene.from_host(s)
    sc.set_batch_shape(5, 0)
    kt = scenes.keyframe_times(300, 6)
    sc.set_active_mask(torch.as_tensor(scenes.keyframe_masks(s, kt)).cuda(), kt)
    ft = scenes.frame_times()
    ks = (0, 90, 181, 299)
    cams = [scenes.arc_camera(scenes.frame_theta(k), 1352, 1014) for k in ks]
    ts = [float(ft[k]) for k in ks]
    want = _batch(fd, sc, fd.STAGING_CP_ASYNC, cams, ts)
    got = _batch(fd, sc, fd.STAGING_TMA, cams, ts)
    for i in range(len(cams)):
        assert torch.equal(got[i], want[i]), i
    counts = {}
    for mode in (fd.STAGING_CP_ASYNC, fd.STAGING_TMA):
        fd.set_batch_staging(mode)
        sc.profile(2)
        sc.render_batch(cams, ts)
        counts[mode] = sc.blend_counts()
        sc.profile(0)
    assert counts[fd.STAGING_CP_ASYNC] == counts[fd.STAGING_TMA], counts
    fd.set_batch_staging(fd.STAGING_TMA)
    tuned = sc.batch_autotune(cams, ts)
    shape = sc.batch_info(len(cams))["footprint"]
    for i in range(len(cams)):
        assert torch.equal(tuned[i], want[i]), (shape, i)
    sc.status_sync()
    sc.close()


def test_gather4_staging_in_the_weighted_passes(fd):
    """The score pass and the key-frame mask pass run the weighted variant of the blend:
    with TMA staging the masks are bit-identical and the scores equal to 1e-5 relative
    (float sums in another order)."""
    s, sc = _masked_scene(fd, 6000, 52)
    cams = [scenes.arc_camera(th, 120, 88) for th in (-8.0, 3.0)]
    ts = [0.2, 0.55, 0.9]
    kt = [0.0, 0.4, 0.8]
    fd.set_batch_staging(fd.STAGING_CP_ASYNC)
    s0 = sc.variation_score(cams, ts, batch=3).cpu().numpy().astype(np.float64)
    m0 = sc.build_keyframe_masks(cams, kt).cpu().numpy()
    fd.set_batch_staging(fd.STAGING_TMA)
    s1 = sc.variation_score(cams, ts, batch=3).cpu().numpy().astype(np.float64)
    m1 = sc.build_keyframe_masks(cams, kt).cpu().numpy()
    sc.status_sync()
    sig = s0 > 1e-6 * s0.max()
    assert int(sig.sum()) > 100
    assert float((np.abs(s1 - s0)[sig] / s0[sig]).max()) <= 1e-5
    assert np.all(np.abs(s1[~sig] - s0[~sig]) <= 1e-6 * s0.max())
    assert np.array_equal(m0, m1)
    sc.close()
