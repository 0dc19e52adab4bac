"""Checkpoints: a scene's attributes on disk, and a Spatial-Temporal Variation Score pass that
survives an interruption.

A score pass over many (t, camera) renders (1M Gaussians x 200 renders in the paper's
pruning step, Sec. 4.2.1) is split into parts of a few timestamps; after each part the
partial scores and the number of parts done are written to the checkpoint file (atomically:
a temporary file renamed over the old one), and a pass started again with the same
arguments continues after the last part written. Every part adds its renders' scores into
the same array (``fdgs_variation_score_add``), so the resumed pass gives the scores of an
uninterrupted one, up to the order of the float additions.
"""
from __future__ import annotations

import hashlib
import os

import numpy as np

from .scenes import Scene

SCENE_FIELDS = ("mean4", "logscale4", "q_left", "q_right", "opacity_logit", "sh")


def _atomic_savez(path, **arrays):
    tmp = path + ".tmp.npz"
    np.savez(tmp, **arrays)
    os.replace(tmp, path)


def _host(a):
    if hasattr(a, "detach"):                # a torch tensor on any device
        a = a.detach().cpu().numpy()
    return np.asarray(a)


def save_scene(path, scene, masks=None, key_times=None) -> None:
    """Write a scene's attribute arrays (host Scene, or device SceneTensors) to ``path``
    (.npz), with its key-frame active masks when given: the packed bits [n_key][ceil(n/8)]
    (LSB-first, the layout of fdgs_set_active_mask) and the key-frame times."""
    arrays = {f: np.ascontiguousarray(_host(getattr(scene, f)), np.float32) for f in SCENE_FIELDS}
    arrays["sh_degree"] = np.array(int(scene.sh_degree), np.int64)
    if masks is not None:
        arrays["mask_bits"] = np.ascontiguousarray(_host(masks), np.uint8)
        arrays["key_times"] = np.ascontiguousarray(_host(key_times), np.float32)
    _atomic_savez(path, **arrays)


def load_scene(path, name="") -> Scene:
    """Read a scene written by save_scene (host arrays)."""
    with np.load(path) as z:
        return Scene(*(z[f].copy() for f in SCENE_FIELDS), int(z["sh_degree"]), name)


def load_masks(path):
    """The key-frame masks saved with a scene: (bits, key_times), or None if it has none."""
    with np.load(path) as z:
        if "mask_bits" not in z.files:
            return None
        return z["mask_bits"].copy(), z["key_times"].copy()


def pass_key(n, cams, ts, variant, batch) -> str:
    """Identity of a score pass: resuming is allowed only for the same arguments."""
    h = hashlib.sha256()
    h.update(np.asarray([n, batch], np.int64).tobytes())
    h.update(variant.encode())
    h.update(np.asarray(ts, np.float32).tobytes())
    for c in cams:
        h.update(np.asarray(c.viewmat, np.float32).tobytes())
        h.update(np.asarray([c.fx, c.fy, c.cx, c.cy, c.znear], np.float32).tobytes())
        h.update(np.asarray([c.width, c.height], np.int64).tobytes())
    return h.hexdigest()[:32]


def parts_of(ts, per_part):
    """The timestamps split into consecutive parts of at most per_part."""
    ts = list(ts)
    return [ts[i:i + per_part] for i in range(0, len(ts), per_part)]


def resumable_pass(path, key, n, parts, run_part, load=np.load, save=_atomic_savez):
    """Host side of a resumable pass. run_part(i, scores) adds part i's contribution into the
    float32 array ``scores`` [n] and returns it; after each part the scores and the count of
    parts done are saved to ``path`` under ``key``. A checkpoint found at ``path`` with the
    same key and n resumes the pass after its last part; one with another key is ignored and
    overwritten. Returns (scores, parts run by this call)."""
    scores = np.zeros(n, np.float32)
    start = 0
    if os.path.exists(path):
        with load(path) as z:
            if str(z["key"]) == key and int(z["n"]) == n:
                scores = z["scores"].astype(np.float32).copy()
                start = int(z["done"])
    ran = 0
    for i in range(start, len(parts)):
        scores = run_part(i, scores)
        ran += 1
        save(path, key=np.array(key), n=np.array(n, np.int64), done=np.array(i + 1, np.int64),
             scores=scores)
    return scores, ran


def variation_score_resumable(scene, cams, ts, path, per_part=5, batch=8, variant="full"):
    """The score pass of fdgs.Scene ``scene`` over timestamps ``ts`` and cameras ``cams``,
    checkpointed to ``path`` after every part of ``per_part`` timestamps. Returns the scores
    as a device tensor [n]."""
    import torch

    parts = parts_of(ts, per_part)
    key = pass_key(scene.n, cams, ts, variant, batch)

    def run_part(i, scores):
        acc = torch.as_tensor(scores).to(scene.device)
        scene.variation_score(cams, parts[i], batch=batch, out=acc, variant=variant,
                              accumulate=True)
        return acc.cpu().numpy()

    scores, _ = resumable_pass(path, key, scene.n, parts, run_part)
    return torch.as_tensor(scores).to(scene.device)


def describe(path) -> dict:
    """What a score checkpoint holds (for logs): its key, n and parts done."""
    with np.load(path) as z:
        return {"key": str(z["key"]), "n": int(z["n"]), "done": int(z["done"])}
