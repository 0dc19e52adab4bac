"""The allocation-free keep-set entry point against the regular one.

fdgs_select_keep_noalloc serves callers that may not call cudaMalloc/cudaFree (a pruning
step inside a real-time loop, where those calls would synchronise the device, or a process
whose HBM is fully reserved by another allocator). Its scratch is a static device array that
every call reuses, so this test calls it several times in a row, with different inputs (the
largest accepted size among them), and checks each result against fdgs_select_keep. A sort
look-back that reaches its spin-wait limit (injected on the host: a short limit and a
withheld publish) must come back as FDGS_ERR_TIMEOUT from the call itself, and the next call
must be right again. It lives in its own file, collected last, and passes both alone and
after the other tests.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _scores(n, seed):
    rng = np.random.default_rng(seed)
    s = rng.gamma(0.5, 1.0, n).astype(np.float32)
    s[rng.random(n) < 0.05] = 0.0                         # a block of exact ties at zero
    s[rng.random(n) < 0.05] = np.float32(0.25)           # and ties inside the range
    return torch.as_tensor(s).cuda()


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2503_16422_gb300 import build, fdgs, scenes
    build.build()
    lib = fdgs.lib()
    sc = fdgs.Scene.from_host(scenes.tiny_scene())
    yield fdgs, lib, sc
    fdgs.debug_inject(fdgs.INJECT_NONE)
    sc.close()


def _noalloc(lib, scores, ratio):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    got = torch.full((scores.numel(),), 7, dtype=torch.uint8, device="cuda")
    rc = lib.fdgs_select_keep_noalloc(ctypes.c_void_p(scores.data_ptr()), scores.numel(),
                                      ratio, ctypes.c_void_p(got.data_ptr()), stream)
    return rc, got


def test_noalloc_keep_set_matches_select_keep_on_successive_calls(env):
    fdgs, lib, sc = env
    for call, (n, ratio) in enumerate([(300_001, 0.8), (1_000_000, 0.85), (1 << 20, 0.5),
                                       (4097, 0.3)]):
        scores = _scores(n, 100 + call)
        want = sc.select_keep(scores, ratio)
        rc, got = _noalloc(lib, scores, ratio)
        assert rc == 0, lib.fdgs_last_error()
        torch.cuda.synchronize()
        assert torch.equal(got, want), f"call {call}: keep sets differ"
        assert int((got == 0).sum()) == int(np.floor(np.float32(ratio) * np.float64(n)))
    # beyond the static limit: a clear error, nothing written
    big = torch.zeros((1 << 20) + 1, dtype=torch.float32, device="cuda")
    rc, out = _noalloc(lib, big, 0.5)
    assert rc == -4 and b"limit" in lib.fdgs_last_error()
    assert int((out == 7).sum()) == out.numel()


def test_noalloc_reports_a_sort_timeout_and_recovers(env):
    fdgs, lib, sc = env
    scores = _scores(200_000, 7)                          # 49 sort partitions
    want = sc.select_keep(scores, 0.8)
    fdgs.debug_inject(fdgs.INJECT_SPIN_LIMIT, 2000)
    fdgs.debug_inject(fdgs.INJECT_WITHHOLD_PUBLISH, 5)
    rc, _ = _noalloc(lib, scores, 0.8)
    assert rc == -5 and b"spin-wait" in lib.fdgs_last_error()
    fdgs.debug_inject(fdgs.INJECT_NONE)
    rc, got = _noalloc(lib, scores, 0.8)
    assert rc == 0, lib.fdgs_last_error()
    assert torch.equal(got, want)
