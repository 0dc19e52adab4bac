"""The allocation-free keep-set entry point against the regular one.

fdgs_select_keep_noalloc serves callers that may not call cudaMalloc/cudaFree (a pruning
step inside a real-time loop, where those calls would synchronise the device, or a process
whose HBM is fully reserved by another allocator). Its scratch is a static device array that
every call reuses, so this test calls it twice in a row, with different inputs, and checks
each result against fdgs_select_keep. It lives in its own file, collected last, and passes
both alone and after the other tests.
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


def test_noalloc_keep_set_matches_select_keep_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2503_16422_gb300 import build, fdgs, scenes
    build.build()
    lib = fdgs.lib()
    sc = fdgs.Scene.from_host(scenes.tiny_scene())
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, (n, ratio) in enumerate([(300_001, 0.8), (1_000_000, 0.85)]):
        scores = _scores(n, 100 + call)
        want = sc.select_keep(scores, ratio)
        got = torch.full((n,), 7, dtype=torch.uint8, device="cuda")
        rc = lib.fdgs_select_keep_noalloc(ctypes.c_void_p(scores.data_ptr()), n, ratio,
                                          ctypes.c_void_p(got.data_ptr()), stream)
        assert rc == 0, lib.fdgs_last_error()
        torch.cuda.synchronize()
        assert torch.equal(got, want), f"call {call}: keep sets differ"
        assert int((got == 0).sum()) == int(np.floor(ratio * n))
    # beyond the static limit: a clear error, nothing written
    big = torch.zeros((1 << 20) + 1, dtype=torch.float32, device="cuda")
    out = torch.zeros_like(big, dtype=torch.uint8)
    rc = lib.fdgs_select_keep_noalloc(ctypes.c_void_p(big.data_ptr()), big.numel(), 0.5,
                                      ctypes.c_void_p(out.data_ptr()), stream)
    assert rc == -4 and b"limit" in lib.fdgs_last_error()
    sc.close()
