"""GPU-vs-oracle comparison helpers.

Decisions the GPU takes in float32 (temporal cull, near plane, tile rectangle edges, the
integer radius) may legitimately differ from the FP64 oracle when the oracle's value sits
within float32 rounding of the threshold. Such Gaussians are *exempt*: counted, reported and
left out of the bit-exact comparisons. Bands (relative to the oracle's value):
  a = sigmoid(o) p(t) vs 1/255 ............ 2e-5 relative
  camera depth vs znear ................... 1e-5 absolute
  rectangle edge quantities vs 16 k ....... 1e-3 px (float32 error of u, v at 1352 px is ~1e-4)
  3 sqrt(lambda_max) vs an integer ........ 5e-5 relative
Per-tile lists are compared as sets after removing exempt Gaussians, and the GPU order must
follow the oracle depth up to a relative 2e-6 (equal-depth groups compared as sets).
"""
import math

import numpy as np
import torch

import oracle

FLAG_MASK, FLAG_TEMPORAL, FLAG_NEAR, FLAG_DET, FLAG_VISIBLE = 1, 2, 4, 8, 16


def oracle_flags(pre):
    f = np.zeros(len(pre["active"]), np.uint8)
    f |= np.where(pre["pass_mask"].numpy(), FLAG_MASK, 0).astype(np.uint8)
    f |= np.where(pre["pass_temporal"].numpy(), FLAG_TEMPORAL, 0).astype(np.uint8)
    f |= np.where(pre["pass_near"].numpy(), FLAG_NEAR, 0).astype(np.uint8)
    f |= np.where(pre["pass_det"].numpy(), FLAG_DET, 0).astype(np.uint8)
    f |= np.where(pre["visible"].numpy(), FLAG_VISIBLE, 0).astype(np.uint8)
    return f


def _near_multiple(x, m, band):
    r = np.mod(x, m)
    return np.minimum(r, m - r) <= band


def exempt_gaussians(pre, cam, edge_band=1e-3, a_rel=2e-5, z_band=1e-5, r_rel=5e-5):
    """Boolean [N]: Gaussians whose decisions sit within float32 reach of a threshold."""
    a = pre["a"].detach().numpy()
    z = pre["depth"].detach().numpy()
    amin = oracle.ALPHA_MIN
    ex = np.abs(a - amin) <= a_rel * amin
    ex |= np.abs(z - cam.znear) <= z_band
    live = pre["pass_near"].numpy()
    edges = pre["rect_edges"].detach().numpy()
    r3 = pre["r3"].numpy()
    W, H = cam.width, cam.height
    near_edge = np.zeros(len(a), bool)
    for k, lim in ((0, W), (1, H), (2, W + 15), (3, H + 15)):
        x = edges[:, k]
        inside = (x > -16) & (x < lim + 16)
        near_edge |= inside & _near_multiple(x, 16.0, edge_band)
    near_r = np.abs(r3 - np.round(r3)) <= r_rel * np.maximum(r3, 1.0)
    ex |= live & (near_edge | near_r)
    if pre.get("tight_edges") is not None:
        # alpha-tight tile sets: the ellipse box edges against tile boundaries; the float32
        # half-widths carry a relative error ~1e-6 on top of the u, v error
        te = pre["tight_edges"].detach().numpy()
        half = np.maximum(np.abs(te[:, 2] - te[:, 0]), np.abs(te[:, 3] - te[:, 1])) * 0.5
        band = edge_band + 1e-5 * half
        near_t = np.zeros(len(a), bool)
        for k, lim in ((0, W), (1, H), (2, W), (3, H)):
            x = te[:, k]
            inside = (x > -16) & (x < lim + 16)
            r = np.mod(x, 16.0)
            near_t |= inside & (np.minimum(r, 16.0 - r) <= band)
        ex |= live & near_t
    return ex


def compare_flags(gpu_flags, pre, exempt):
    """Returns (number of non-exempt mismatches, number of exempt Gaussians)."""
    want = oracle_flags(pre)
    got = np.asarray(gpu_flags, np.uint8)
    bad = (want != got) & ~exempt
    return int(bad.sum()), int(exempt.sum()), np.nonzero(bad)[0]


def compare_tile_lists(gpu_ranges, gpu_ids, oracle_lists, pre, exempt, rel_tie=2e-6):
    """Compare per-tile lists. gpu_ranges [tiles,2], gpu_ids [K] (numpy). oracle_lists:
    {tile: ids}. Returns dict with counts of mismatching tiles and checked keys."""
    depth = pre["depth"].detach().numpy()
    bad_tiles = []
    keys = 0
    for tid, want in oracle_lists.items():
        s, e = int(gpu_ranges[tid, 0]), int(gpu_ranges[tid, 1])
        got = np.asarray(gpu_ids[s:e]) if e > s else np.zeros(0, np.int64)
        w = np.asarray(want)
        w = w[~exempt[w]]
        g = got[~exempt[got]] if len(got) else got
        keys += len(w)
        if len(w) != len(g) or set(w.tolist()) != set(g.tolist()):
            bad_tiles.append((tid, "set"))
            continue
        if len(g) > 1:
            d = depth[g]
            if np.any(d[1:] < d[:-1] * (1 - rel_tie)):
                bad_tiles.append((tid, "order"))
    return dict(bad_tiles=bad_tiles, keys=keys, tiles=len(oracle_lists))


def image_metrics(gpu, ref, tol=1e-3):
    """max-abs, fraction of values above tol, PSNR (peak 1) over the finite reference
    entries."""
    g = np.asarray(gpu, np.float64)
    r = np.asarray(ref, np.float64)
    m = np.isfinite(r)
    d = np.abs(g[m] - r[m])
    mse = float(np.mean(d * d)) if d.size else 0.0
    psnr = float("inf") if mse == 0 else 10 * math.log10(1.0 / mse)
    return dict(max_abs=float(d.max()) if d.size else 0.0,
                frac_bad=float((d > tol).mean()) if d.size else 0.0, psnr=psnr, n=int(d.size))


def to_np(t):
    return t.detach().cpu().numpy() if isinstance(t, torch.Tensor) else np.asarray(t)


def contribution_exempt(P, cam, t, eps=1e-4):
    """The oracle's visibility mask of one view and the Gaussians whose blended-somewhere
    status flips when the alpha floor or the stop threshold moves by eps (relative): cases a
    float32 renderer may decide either way. Returns (mask [N], exempt [N])."""
    import oracle.fdgs_oracle as om
    base = oracle.contributing(P, cam, t)
    ex = np.zeros_like(base)
    a0, t0 = om.ALPHA_MIN, om.T_STOP
    try:
        for fa in (1 - eps, 1 + eps):
            for ft in (1 - eps, 1 + eps):
                om.ALPHA_MIN, om.T_STOP = a0 * fa, t0 * ft
                ex |= oracle.contributing(P, cam, t) != base
    finally:
        om.ALPHA_MIN, om.T_STOP = a0, t0
    return base, ex
