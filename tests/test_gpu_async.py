"""Renders without host synchronisation (fdgs_render_async) against fdgs_render.

The call enqueues every stage and returns; its tile lists are the coverage-bitmask lists,
built into a capacity fixed before the launch. Images must equal the synchronised render's
bit for bit (the synchronised render is the one checked against the FP64 oracle), queued
back to back, replayed from a captured CUDA graph, and after a capacity overflow, which
leaves the background and is reported (FDGS_ERR_CAPACITY) by the next status_sync, after
which the capacity fits.
"""
import numpy as np
import pytest
import torch

from paper_2503_16422_gb300 import scenes

pytestmark = pytest.mark.gpu

FDGS_ERR_CAPACITY = -4


@pytest.fixture(scope="module")
def fd():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2503_16422_gb300 import build, fdgs
    build.build()
    fdgs.lib()
    return fdgs


@pytest.fixture(scope="module")
def masked_scene(fd):
    """A 30k-Gaussian degree-3 scene with key-frame masks, and frames on the arc at 480x360
    (ragged tiles at both edges)."""
    s = scenes.make_scene(30_000, 21, sh_degree=3, lt_long=(-1.5, 0.5), name="async")
    kt = scenes.keyframe_times()
    masks = scenes.keyframe_masks(s, kt)
    sc = fd.Scene.from_host(s)
    sc.set_active_mask(torch.as_tensor(masks).cuda(), kt)
    times = scenes.frame_times()
    frames = [(scenes.arc_camera(scenes.frame_theta(k), 480, 360), float(times[k]))
              for k in (0, 37, 150, 233, 299)]
    yield sc, frames
    sc.close()


def fit(fd, sc, frames, **kw):
    """Renders every frame once without host synchronisation, repeating the pass while the
    status reports a list-capacity overflow (each report grows the capacity to fit)."""
    for _ in range(4):
        for c, t in frames:
            sc.render_async(c, t, **kw)
        try:
            sc.status_sync()
            return
        except fd.FdgsError as e:
            assert e.code == FDGS_ERR_CAPACITY
    raise AssertionError("the list capacity kept overflowing")


@pytest.mark.parametrize("use_mask,bg,tight", [(True, (0.0, 0.0, 0.0), False),
                                               (False, (0.0, 0.0, 0.0), False),
                                               (True, (0.2, 0.5, 1.0), False),
                                               (True, (0.0, 0.0, 0.0), True)])
def test_async_renders_equal_synchronised_renders(fd, masked_scene, use_mask, bg, tight):
    sc, frames = masked_scene
    want = [sc.render(c, t, use_mask=use_mask, bg=bg, tight=tight).clone() for c, t in frames]
    fit(fd, sc, frames, use_mask=use_mask, bg=bg, tight=tight)
    # queued back to back on one stream, no host synchronisation between them
    outs = [sc.render_async(c, t, use_mask=use_mask, bg=bg, tight=tight) for c, t in frames]
    sc.status_sync()
    for k, (o, w) in enumerate(zip(outs, want)):
        assert torch.equal(o, w), f"frame {k}: async render differs"


def test_async_render_replays_from_a_cuda_graph(fd, masked_scene):
    sc, frames = masked_scene
    want = [sc.render(c, t).clone() for c, t in frames]
    outs = [torch.zeros((3, 360, 480), dtype=torch.float32, device="cuda") for _ in frames]
    fit(fd, sc, frames)                               # sized outside the capture
    for o in outs:
        o.zero_()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for (c, t), o in zip(frames, outs):
            sc.render_async(c, t, out=o)
    for o in outs:
        o.fill_(7.0)
    torch.cuda.synchronize()
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        sc.status_sync()
        for k, (o, w) in enumerate(zip(outs, want)):
            assert torch.equal(o, w), f"frame {k}: graph replay differs"


def test_async_capacity_overflow_is_reported_and_the_retry_fits(fd, masked_scene):
    sc, frames = masked_scene
    cam, t = frames[2]
    want = sc.render(cam, t).clone()
    sc.reserve_render_lists(1000)                    # far below the frame's list length
    got = sc.render_async(cam, t)
    with pytest.raises(fd.FdgsError) as ei:
        sc.status_sync()
    assert ei.value.code == FDGS_ERR_CAPACITY
    # the overflowing frame composited nothing: background only, nothing out of bounds
    assert float(got.abs().max()) == 0.0
    sc.status_sync()                                 # the status word was cleared
    got = sc.render_async(cam, t)
    sc.status_sync()
    assert torch.equal(got, want)
    # other frames of the sequence fit the grown capacity as well, or grow it once more
    for c, tt in frames:
        w = sc.render(c, tt)
        g = sc.render_async(c, tt)
        try:
            sc.status_sync()
        except fd.FdgsError as e:
            assert e.code == FDGS_ERR_CAPACITY
            g = sc.render_async(c, tt)
            sc.status_sync()
        assert torch.equal(g, w)


def test_async_render_refuses_the_sort_list_builder(fd, masked_scene):
    sc, frames = masked_scene
    fd.set_list_builder(1)
    try:
        with pytest.raises(fd.FdgsError) as ei:
            sc.render_async(*frames[0])
        assert ei.value.code == -1 and "bitmask" in str(ei.value)
    finally:
        fd.set_list_builder(0)
    assert np.isfinite(sc.render_async(*frames[0]).cpu().numpy()).all()
    sc.status_sync()
