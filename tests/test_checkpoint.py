"""Checkpoint helpers on the host (no GPU): a scene written and read back, and the
bookkeeping of a resumable score pass, interrupted and resumed, against an uninterrupted one
(the per-part work is a stand-in that adds fixed values, so any lost or repeated part shows)."""
import numpy as np
import pytest

from paper_2503_16422_gb300 import checkpoint, scenes


def test_scene_roundtrip(tmp_path):
    s = scenes.make_scene(500, 7, sh_degree=3, name="ck")
    path = str(tmp_path / "scene.npz")
    checkpoint.save_scene(path, s)
    r = checkpoint.load_scene(path)
    assert r.sh_degree == 3 and r.n == 500
    for f in checkpoint.SCENE_FIELDS:
        assert np.array_equal(getattr(r, f), getattr(s, f)), f
    assert checkpoint.load_masks(path) is None
    kt = scenes.keyframe_times()
    bits = scenes.keyframe_masks(s, kt)
    checkpoint.save_scene(path, s, masks=bits, key_times=kt)
    got_bits, got_kt = checkpoint.load_masks(path)
    assert np.array_equal(got_bits, bits) and np.array_equal(got_kt, kt.astype(np.float32))
    assert np.array_equal(checkpoint.load_scene(path).sh, s.sh)


def _part_adder(n, fail_at=None):
    calls = []

    def run_part(i, scores):
        if fail_at is not None and i == fail_at:
            raise RuntimeError("interrupted")
        calls.append(i)
        out = scores.copy()
        out[i::5] += np.float32(i + 1)       # a part's own, distinguishable contribution
        return out
    return run_part, calls


def test_resumable_pass_resumes_after_an_interruption(tmp_path):
    n, parts = 23, [[0.1], [0.2], [0.3], [0.4], [0.5], [0.6]]
    path = str(tmp_path / "score.npz")
    want, _ = checkpoint.resumable_pass(str(tmp_path / "whole.npz"), "k", n, parts,
                                        _part_adder(n)[0])
    run, calls = _part_adder(n, fail_at=3)
    with pytest.raises(RuntimeError):
        checkpoint.resumable_pass(path, "k", n, parts, run)
    assert calls == [0, 1, 2] and checkpoint.describe(path)["done"] == 3
    run2, calls2 = _part_adder(n)
    got, ran = checkpoint.resumable_pass(path, "k", n, parts, run2)
    assert calls2 == [3, 4, 5] and ran == 3
    assert np.array_equal(got, want)
    # a finished pass is not run again
    got2, ran2 = checkpoint.resumable_pass(path, "k", n, parts, _part_adder(n)[0])
    assert ran2 == 0 and np.array_equal(got2, want)


def test_resumable_pass_ignores_a_checkpoint_of_another_pass(tmp_path):
    n, parts = 11, [[0.1], [0.2], [0.3]]
    path = str(tmp_path / "score.npz")
    checkpoint.resumable_pass(path, "other", n, parts, _part_adder(n)[0])
    got, ran = checkpoint.resumable_pass(path, "k", n, parts, _part_adder(n)[0])
    assert ran == 3
    want, _ = checkpoint.resumable_pass(str(tmp_path / "w.npz"), "k", n, parts,
                                        _part_adder(n)[0])
    assert np.array_equal(got, want)


def test_pass_key_depends_on_the_arguments():
    cams = [scenes.arc_camera(0.0, 64, 48), scenes.arc_camera(5.0, 64, 48)]
    k = checkpoint.pass_key(100, cams, [0.1, 0.2], "full", 8)
    assert k == checkpoint.pass_key(100, cams, [0.1, 0.2], "full", 8)
    assert k != checkpoint.pass_key(100, cams, [0.1, 0.3], "full", 8)
    assert k != checkpoint.pass_key(100, cams[:1], [0.1, 0.2], "full", 8)
    assert k != checkpoint.pass_key(100, cams, [0.1, 0.2], "spatial", 8)
    assert checkpoint.parts_of([1, 2, 3, 4, 5], 2) == [[1, 2], [3, 4], [5]]
