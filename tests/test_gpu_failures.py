"""Failure detection in the forms this library uses, made without faulting or hanging the GPU:
a device spin-wait that gives up after a short limit (a look-back publish withheld on the
host's request) and reports FDGS_ERR_TIMEOUT, and a device allocation refused on the host
(FDGS_ERR_OOM). After each failure the next call on the same scene must work."""
import numpy as np
import pytest
import torch

import oracle
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
    fdgs.debug_inject(fdgs.INJECT_NONE)


def _scores(n, seed):
    rng = np.random.default_rng(seed)
    return rng.gamma(0.6, 1.0, n).astype(np.float32)


def test_lookback_timeout_is_reported_and_the_next_call_works(fd):
    sc = fd.Scene.from_host(scenes.tiny_scene())
    n = 100_000                                    # 25 sort partitions of 4096 keys
    s32 = _scores(n, 1)
    scores = torch.as_tensor(s32).cuda()
    want = oracle.keep_set(s32.astype(np.float64), float(np.float32(0.8)))
    # a short spin limit and a partition that never publishes: its successors give up
    fd.debug_inject(fd.INJECT_SPIN_LIMIT, 2000)
    fd.debug_inject(fd.INJECT_WITHHOLD_PUBLISH, 3)
    sc.select_keep(scores, 0.8)
    with pytest.raises(fd.FdgsError) as ei:
        sc.status_sync()
    assert ei.value.code == -5
    # the status word was read and cleared; the withheld publish was one-shot
    sc.status_sync()
    keep = sc.select_keep(scores, 0.8).cpu().numpy().astype(bool)
    sc.status_sync()
    assert np.array_equal(keep, want)
    fd.debug_inject(fd.INJECT_NONE)
    keep = sc.select_keep(scores, 0.8).cpu().numpy().astype(bool)
    sc.status_sync()
    assert np.array_equal(keep, want)
    sc.close()


def test_refused_allocation_returns_oom_and_the_next_render_works(fd):
    s = scenes.tiny_scene()
    cam = scenes.tiny_camera(64, 48)
    ref = fd.Scene.from_host(s)
    want = ref.render(cam, 0.5).clone()
    ref.close()
    sc = fd.Scene.from_host(s)                     # a fresh scene: its workspaces must grow
    fd.debug_inject(fd.INJECT_FAIL_ALLOCS, 1)
    with pytest.raises(fd.FdgsError) as ei:
        sc.render(cam, 0.5)
    assert ei.value.code == -3 and "injected" in str(ei.value)
    got = sc.render(cam, 0.5)
    assert torch.equal(got, want)
    # the batched path: its plan's first buffer is refused, then the batch renders
    cams = [scenes.arc_camera(-4.0, 48, 40), cam]
    fd.debug_inject(fd.INJECT_FAIL_ALLOCS, 1)
    with pytest.raises(fd.FdgsError) as ei:
        sc.render_batch(cams, [0.3, 0.5], use_mask=False)
    assert ei.value.code == -3
    outs = sc.render_batch(cams, [0.3, 0.5], use_mask=False)
    for c, t, o in zip(cams, [0.3, 0.5], outs):
        assert torch.equal(o, sc.render(c, t, use_mask=False))
    sc.close()


def test_tma_stage_wait_timeout_is_reported_and_the_next_batch_works(fd):
    """TMA record staging with one arrival withheld on every stage barrier of one batch: the
    blend's stage waits give up after their poll limit, the missing arrival is supplied so the
    copies in flight land before the CTAs leave, the call reports FDGS_ERR_TIMEOUT, and the
    next batch (graph replay) renders the same images as before the failure."""
    s = scenes.make_scene(6000, 53, sh_degree=1, lt_short=(-3.0, 0.5), lt_long=(-1.0, 0.5),
                          short_frac=0.5)
    sc = fd.Scene.from_host(s)
    cams = [scenes.arc_camera(th, 96, 72) for th in (-5.0, 2.0, 8.0)]
    ts = [0.2, 0.5, 0.8]
    try:
        fd.set_batch_staging(fd.STAGING_TMA)
        sc.set_batch_shape(5, 0)            # a four-pixels-a-lane shape: TMA staging applies
        want = [o.clone() for o in sc.render_batch(cams, ts, use_mask=False)]
        fd.debug_inject(fd.INJECT_TMA_MISSING_ARRIVAL, 0)
        with pytest.raises(fd.FdgsError) as ei:
            sc.render_batch(cams, ts, use_mask=False)
        assert ei.value.code == -5
        got = sc.render_batch(cams, ts, use_mask=False)
        sc.status_sync()
        for i in range(len(cams)):
            assert torch.equal(got[i], want[i]), i
    finally:
        fd.set_batch_staging(fd.STAGING_CP_ASYNC)
        fd.debug_inject(fd.INJECT_NONE)
    sc.close()
