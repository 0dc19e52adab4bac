"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/*.h declares (no GPU needed: no compute call is made)."""
import ctypes
import glob
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(fdgs_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    if not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")):
        pytest.skip("nvcc not available")
    from paper_2503_16422_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("fdgs_create_scene", "fdgs_set_active_mask", "fdgs_render",
                 "fdgs_render_backward", "fdgs_variation_score", "fdgs_render_batch",
                 "fdgs_select_keep", "fdgs_status_sync", "fdgs_last_error"):
        assert want in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header(libpath):
    from paper_2503_16422_gb300 import fdgs
    lib = fdgs.lib()
    declared = set(declared_functions())
    bound = set(fdgs._SIGNATURES) | {"fdgs_last_error", "fdgs_version"}
    assert declared <= bound, declared - bound
    assert lib.fdgs_version().decode().startswith("fdgs")


def test_invalid_arguments_fail_without_a_gpu(libpath):
    """Argument validation happens on the host before any CUDA call."""
    from paper_2503_16422_gb300 import fdgs
    lib = fdgs.lib()
    h = ctypes.c_void_p()
    rc = lib.fdgs_create_scene(None, ctypes.byref(h))
    assert rc == -1 and b"null" in lib.fdgs_last_error()
    d = fdgs.fdgs_scene_desc()
    d.n, d.sh_degree = 10, 5
    assert lib.fdgs_create_scene(ctypes.byref(d), ctypes.byref(h)) == -1
    assert b"sh_degree" in lib.fdgs_last_error()
    d.sh_degree = 0
    assert lib.fdgs_create_scene(ctypes.byref(d), ctypes.byref(h)) == -1   # null pointers
    assert lib.fdgs_render(None, None, 0.0, None, None, None, None) == -1
    assert lib.fdgs_destroy_scene(None) == 0
    assert lib.fdgs_frame_release(None) == 0


def test_batch_marshalling_matches_the_c_structs():
    """The binding marshals a batch's cameras, times and output pointers through numpy; the
    bytes must be exactly those of the ctypes fdgs_camera array the header describes."""
    import numpy as np

    from paper_2503_16422_gb300 import fdgs, scenes
    cams = [scenes.arc_camera(th, w, h) for th, w, h in ((-9.5, 1352, 1014), (0.0, 33, 17),
                                                         (7.25, 512, 512))]
    arr, ptr = fdgs.make_cameras(cams)
    ref = (fdgs.fdgs_camera * len(cams))(*[fdgs.make_camera(c) for c in cams])
    assert arr.tobytes() == bytes(ref)
    assert ctypes.addressof(ptr.contents) == arr.ctypes.data
    ts = [0.0, 0.5, 1.0]
    ta, tp = fdgs._times(ts)
    assert ta.dtype == np.float32 and list(ta) == ts
    assert ctypes.addressof(tp.contents) == ta.ctypes.data
    empty, _ = fdgs.make_cameras([])
    assert empty.shape == (1,)


def test_failure_injection_arguments_are_checked_on_the_host(libpath):
    """fdgs_debug_inject is a host-side setter: bad kinds and values are refused, and
    clearing restores the defaults (no GPU needed)."""
    from paper_2503_16422_gb300 import fdgs
    lib = fdgs.lib()
    assert lib.fdgs_debug_inject(99, 0) == -1 and b"unknown" in lib.fdgs_last_error()
    assert lib.fdgs_debug_inject(fdgs.INJECT_SPIN_LIMIT, -1) == -1
    assert lib.fdgs_debug_inject(fdgs.INJECT_SPIN_LIMIT, 1 << 21) == -1
    assert lib.fdgs_debug_inject(fdgs.INJECT_WITHHOLD_PUBLISH, -2) == -1
    assert lib.fdgs_debug_inject(fdgs.INJECT_FAIL_ALLOCS, -1) == -1
    assert lib.fdgs_debug_inject(fdgs.INJECT_SPIN_LIMIT, 1000) == 0
    assert lib.fdgs_debug_inject(fdgs.INJECT_FAIL_ALLOCS, 2) == 0
    assert lib.fdgs_debug_inject(fdgs.INJECT_NONE, 0) == 0
