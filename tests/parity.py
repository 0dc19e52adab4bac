"""GPU-vs-oracle comparison helpers.

Decisions the GPU takes in float32 (temporal cull, near plane, tile-rectangle edges, the
integer radius, the alpha floor and the stop rule of the blend) may legitimately differ from
the FP64 oracle when the oracle's value sits within float32 reach of the threshold. Such
Gaussians and pixels are *exempt*: counted, reported (one ``PARITY {json}`` line per check,
also appended to the file named by FDGS_PARITY_LOG), bounded, and left out of the exact
comparisons. The contract's bands are 1e-4 px at a tile edge, 1e-4 at an integer radius and
1e-6 relative at a cull threshold; where float32 cannot meet one, the band is the float32
error bound of that quantity (``f32_bounds``), never less than the contract's band:

  u, v  eps (f/|z| (1 + |x/z|) (32 |D| + 8 (|mu| + |t_v|)) + 2 |u|)   px
  a     eps (16 + 64 |ln p|)                                          relative
  z     eps (32 |D| + 16 (|mu| + |t_v|))                              absolute
  r3    64 eps r3                                                     absolute

with eps = 2^-24, D = mu_xyz|t - mu_xyz the conditional shift of Eq. 1, mu the spatial mean,
t_v the camera translation, p the temporal weight of Eq. 3. Each is a first-order count of the
float32 roundings on the way to the quantity (the 4D frame, Eq. 1's shift and the view
transform), each bounded by eps times the magnitude it rounds; the constants carry a margin,
and ``test_gpu_forward`` measures the GPU's actual error against them on every visible
Gaussian.
"""
import json
import math
import os

import numpy as np
import torch

import oracle

FLAG_MASK, FLAG_TEMPORAL, FLAG_NEAR, FLAG_DET, FLAG_VISIBLE = 1, 2, 4, 8, 16
EPS32 = 2.0 ** -24
EDGE_BAND = 1e-4          # px, tile edges (contract)
RADIUS_BAND = 1e-4        # 3 sqrt(lambda) against an integer (contract)
CULL_REL = 1e-6           # relative, cull thresholds a = 1/255 and z = znear (contract)
CONIC_REL = 1e-5          # relative error of the GPU's conic (asserted on every record)


def f32(x):
    """The float32 value the C ABI receives for a time or key time x, as a Python float: the
    oracle is evaluated at the same inputs as the GPU (near an inflection of p(t) the score
    factor moves by 0.2% between 0.65 and float32(0.65))."""
    return float(np.float32(x))


def report(name, **counts):
    """One machine-readable line of counts for a parity check."""
    line = json.dumps({"check": name, **counts}, sort_keys=True, default=float)
    print("PARITY " + line)
    path = os.environ.get("FDGS_PARITY_LOG")
    if path:
        with open(path, "a") as f:
            f.write(line + "\n")
    return line


def oracle_flags(pre):
    f = np.zeros(len(pre["active"]), np.uint8)
    f |= np.where(pre["pass_mask"].numpy(), FLAG_MASK, 0).astype(np.uint8)
    f |= np.where(pre["pass_temporal"].numpy(), FLAG_TEMPORAL, 0).astype(np.uint8)
    f |= np.where(pre["pass_near"].numpy(), FLAG_NEAR, 0).astype(np.uint8)
    f |= np.where(pre["pass_det"].numpy(), FLAG_DET, 0).astype(np.uint8)
    f |= np.where(pre["visible"].numpy(), FLAG_VISIBLE, 0).astype(np.uint8)
    return f


def f32_bounds(pre, cam, mean4):
    """Per-Gaussian float32 error bounds (see the module docstring) of u, v (px), a
    (relative), z (absolute) and 3 sqrt(lambda) (absolute)."""
    xc = pre["xc"].detach().numpy()
    z = np.abs(xc[:, 2]) + 1e-30
    mu = np.asarray(mean4, np.float64)[:, :3]
    shift = np.linalg.norm(pre["mu3"].detach().numpy() - mu, axis=1)
    tv = float(np.linalg.norm(np.asarray(cam.viewmat, np.float64)[:3, 3]))
    mag = np.linalg.norm(mu, axis=1) + tv
    m2 = pre["mean2d"].detach().numpy()
    base = 32.0 * shift + 8.0 * mag
    bu = EPS32 * (cam.fx / z * (1 + np.abs(xc[:, 0]) / z) * base + 2 * np.abs(m2[:, 0]))
    bv = EPS32 * (cam.fy / z * (1 + np.abs(xc[:, 1]) / z) * base + 2 * np.abs(m2[:, 1]))
    lnp = np.abs(np.log(np.maximum(pre["p"].detach().numpy(), 1e-300)))
    ba = EPS32 * (16.0 + 64.0 * lnp)
    bz = EPS32 * (32.0 * shift + 16.0 * mag)
    br = 64.0 * EPS32 * pre["r3"].numpy()
    return dict(u=bu, v=bv, a=ba, z=bz, r3=br)


def _near_multiple(x, m, band):
    r = np.mod(x, m)
    return np.minimum(r, m - r) <= band


def exempt_gaussians(pre, cam, mean4, detail=False):
    """Boolean [N]: Gaussians whose float32 decisions may differ from the oracle's (value
    within max(contract band, float32 bound) of a threshold). With detail, also the counts
    per reason."""
    b = f32_bounds(pre, cam, mean4)
    a = pre["a"].detach().numpy()
    z = pre["depth"].detach().numpy()
    amin = oracle.ALPHA_MIN
    ex_a = np.abs(a - amin) <= np.maximum(CULL_REL, b["a"]) * amin
    ex_z = np.abs(z - cam.znear) <= np.maximum(CULL_REL * cam.znear, b["z"])
    live = pre["pass_near"].numpy()
    edges = pre["rect_edges"].detach().numpy()
    r3 = pre["r3"].numpy()
    W, H = cam.width, cam.height
    near_edge = np.zeros(len(a), bool)
    for k, lim, bb in ((0, W, b["u"]), (1, H, b["v"]), (2, W + 15, b["u"]),
                       (3, H + 15, b["v"])):
        x = edges[:, k]
        inside = (x > -16) & (x < lim + 16)
        near_edge |= inside & _near_multiple(x, 16.0, np.maximum(EDGE_BAND, bb))
    near_r = np.abs(r3 - np.round(r3)) <= np.maximum(RADIUS_BAND, b["r3"])
    near_t = np.zeros(len(a), bool)
    if pre.get("tight_edges") is not None:
        # alpha-tight tile sets: the ellipse box edges against tile boundaries (half-widths
        # carry a relative float32 error on top of u, v; the box is widened by 0.1% + 0.1 in
        # both renderers, so only the u, v error and that rounding matter)
        te = pre["tight_edges"].detach().numpy()
        half = np.maximum(np.abs(te[:, 2] - te[:, 0]), np.abs(te[:, 3] - te[:, 1])) * 0.5
        for k, lim, bb in ((0, W, b["u"]), (1, H, b["v"]), (2, W, b["u"]), (3, H, b["v"])):
            x = te[:, k]
            inside = (x > -16) & (x < lim + 16)
            band = np.maximum(EDGE_BAND, bb + 64 * EPS32 * half)
            near_t |= inside & _near_multiple(x, 16.0, band)
    ex = ex_a | ex_z | (live & (near_edge | near_r | near_t))
    if detail:
        return ex, dict(alpha_cull=int(ex_a.sum()), near_plane=int(ex_z.sum()),
                        tile_edge=int((live & near_edge).sum()),
                        radius=int((live & near_r).sum()), tight_edge=int((live & near_t).sum()))
    return ex


def compare_flags(gpu_flags, pre, exempt):
    """Returns (number of non-exempt mismatches, number of exempt Gaussians, their ids, number
    of exempt Gaussians whose flags differ)."""
    want = oracle_flags(pre)
    got = np.asarray(gpu_flags, np.uint8)
    diff = want != got
    bad = diff & ~exempt
    return int(bad.sum()), int(exempt.sum()), np.nonzero(bad)[0], int((diff & exempt).sum())


def compare_tile_lists(gpu_ranges, gpu_ids, oracle_lists, pre, exempt, gpu_depth, z_bound):
    """Per-tile lists. Sets: equal after removing exempt Gaussians. Order: the GPU's list is
    exactly ascending in (its float32 depth bits, id); against the oracle, two entries must
    be in the oracle's (depth, id) order unless their oracle depths are within the sum of
    their float32 depth bounds (such ties are compared as sets). gpu_depth [N]: the GPU's
    record depths (NaN where not visible); z_bound [N]: float32 depth bounds."""
    depth = pre["depth"].detach().numpy()
    bad_tiles = []
    keys = ties = 0
    for tid, want in oracle_lists.items():
        s, e = int(gpu_ranges[tid, 0]), int(gpu_ranges[tid, 1])
        got = np.asarray(gpu_ids[s:e], np.int64) if e > s else np.zeros(0, np.int64)
        w = np.asarray(want)
        w = w[~exempt[w]]
        g = got[~exempt[got]] if len(got) else got
        keys += len(w)
        if len(w) != len(g) or set(w.tolist()) != set(g.tolist()):
            bad_tiles.append((tid, "set"))
            continue
        if len(got) > 1:
            gd = gpu_depth[got].astype(np.float32).view(np.uint32).astype(np.int64)
            key = gd * (1 << 32) + got
            if np.any(np.diff(key) <= 0):
                bad_tiles.append((tid, "gpu order"))
                continue
        if len(g) > 1:
            d = depth[g]
            zb = z_bound[g]
            # no entry may come after one whose oracle depth exceeds its own by more than the
            # pair's float32 bounds: max over earlier i of (d_i - zb_i) <= d_j + zb_j
            lo = np.maximum.accumulate(d - zb)
            if np.any(lo[:-1] > d[1:] + zb[1:]):
                bad_tiles.append((tid, "order"))
                continue
            ties += int(np.sum(np.abs(np.diff(d)) <= zb[1:] + zb[:-1]))
    return dict(bad_tiles=bad_tiles, keys=keys, tiles=len(oracle_lists), tie_pairs=ties)


def _tile_alpha(pre, ids, px, py, bounds=None, rec=None):
    """power and alpha = min(0.99, a exp(power)) of the entries ``ids`` at pixels (px, py);
    with ``bounds`` (``f32_bounds``), also [lo, hi], an interval holding the GPU's float32
    alpha, and r = max(hi / alpha - 1, 1 - lo / alpha) (inf where alpha is 0). ``rec`` =
    (records [N, >=6], valid [N]) are the GPU's own records of the view (u, v, A, B, C, a):
    the interval is then spanned by the oracle's alpha and the alpha of the GPU's record,
    evaluated in float64; without them (or where not valid) it is the oracle's alpha widened
    by the first-order bound of the record error (u, v within b_u, b_v, the conic within
    CONIC_REL, a within b_a): CONIC_REL |power| + |A dx + B dy| b_u + |B dx + C dy| b_v + b_a.
    Either way it is widened by twice the evaluation's own rounding (four roundings of the
    log2 exponent and the ex2 approximation), 16 eps (1 + |power| + |log2 a|), relative."""
    m2 = pre["mean2d"].detach().numpy()
    con = pre["conic"].detach().numpy()
    a = pre["a"].detach().numpy()
    dx = m2[None, ids, 0] - px[:, None]
    dy = m2[None, ids, 1] - py[:, None]
    A, B, C = con[None, ids, 0], con[None, ids, 1], con[None, ids, 2]
    power = -0.5 * (A * dx * dx + C * dy * dy) - B * dx * dy
    raw = a[None, ids] * np.exp(power)
    alpha = np.minimum(raw, oracle.ALPHA_MAX)
    if bounds is None:
        return power, alpha
    la = np.abs(np.log2(np.maximum(a[None, ids], 1e-300)))
    re = 32.0 * EPS32 * (1.0 + np.abs(power) + la)
    rb = (CONIC_REL * np.abs(power) + np.abs(A * dx + B * dy) * bounds["u"][None, ids]
          + np.abs(B * dx + C * dy) * bounds["v"][None, ids] + bounds["a"][None, ids])
    lo, hi = raw * (1.0 - rb), raw * (1.0 + rb)
    if rec is not None:
        R, ok = rec
        g = R[ids].astype(np.float64)
        gdx = g[None, :, 0] - px[:, None]
        gdy = g[None, :, 1] - py[:, None]
        gpow = -0.5 * (g[None, :, 2] * gdx * gdx + g[None, :, 4] * gdy * gdy) \
            - g[None, :, 3] * gdx * gdy
        with np.errstate(over="ignore", invalid="ignore"):
            graw = g[None, :, 5] * np.exp(np.minimum(gpow, 0.0))
        use = ok[None, ids] & np.isfinite(graw)
        lo = np.where(use, np.minimum(raw, graw), lo)
        hi = np.where(use, np.maximum(raw, graw), hi)
    lo = np.minimum(lo * (1.0 - re), oracle.ALPHA_MAX)
    hi = np.minimum(hi * (1.0 + re), oracle.ALPHA_MAX)
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(alpha > 0, np.maximum(hi / alpha - 1.0, 1.0 - lo / alpha), np.inf)
    return power, alpha, lo, hi, r


def _order_suspects(ids, gpu_ids, pre, z_bound):
    """Pairs of entries of a tile list whose order may differ between the renderers: with the
    GPU's list, the common pairs in inverted order; without it, the pairs within runs of
    adjacent oracle entries whose depths lie within their float32 bounds. Returns [P, 2]."""
    none = np.zeros((0, 2), np.int64)
    if gpu_ids is not None:
        common = np.intersect1d(ids, gpu_ids)
        if len(common) < 2:
            return none
        o = ids[np.isin(ids, common)]
        g = gpu_ids[np.isin(gpu_ids, common)]
        if np.array_equal(o, g):
            return none
        rank = {int(x): k for k, x in enumerate(o)}
        seq = np.array([rank[int(x)] for x in g])
        pairs = [(int(g[k]), int(g[l])) for k in range(len(g)) for l in range(k + 1, len(g))
                 if seq[k] > seq[l]]
        return np.asarray(pairs, np.int64).reshape(-1, 2)
    if z_bound is None or len(ids) < 2:
        return none
    d = pre["depth"].detach().numpy()[ids]
    zb = z_bound[ids]
    tie = np.abs(np.diff(d)) <= zb[1:] + zb[:-1]
    pairs = []
    k = 0
    while k < len(tie):
        if not tie[k]:
            k += 1
            continue
        e = k
        while e < len(tie) and tie[e]:
            e += 1
        run = ids[k:e + 1]                      # entries k..e form one run of ties
        pairs += [(int(run[i]), int(run[j])) for i in range(len(run))
                  for j in range(i + 1, len(run))]
        k = e
    return np.asarray(pairs, np.int64).reshape(-1, 2)


def _membership_suspects(pre, ids, tid, gx, exempt, gpu_ids):
    """Exempt Gaussians whose membership in tile ``tid`` may differ between the renderers:
    with the GPU's list, the symmetric difference of the two lists; without it, the exempt
    Gaussians with valid geometry whose 3-sigma rectangle, grown by one tile, covers it."""
    if gpu_ids is not None:
        return np.setxor1d(ids, gpu_ids)
    tx, ty = tid % gx, tid // gx
    r = pre["rect_square"].numpy()
    ok = exempt & pre["pass_near"].numpy() & (pre["det"].detach().numpy() > 0)
    near = ok & (r[:, 0] - 1 <= tx) & (tx <= r[:, 2]) & (r[:, 1] - 1 <= ty) & (ty <= r[:, 3])
    return np.nonzero(near)[0]


def _tile_flags(pre, ids, tid, gx, px, py, exempt, gid, bounds, last_entry=False, rec=None):
    """The per-pixel decisions of one tile that float32 may take differently (see
    ``pixel_exemptions``). Returns (flags {reason: [P] bool}, detail) where detail holds the
    oracle's blend weights ignoring the stop rule [P, L] (alpha T over the entries that pass
    the floor), the relative float32 error bound of each such weight [P, L], the entry flags
    of the alpha and stop reasons [P, L], each pixel's stop position [P], and the list-position
    span [P, 2] a membership or order difference may touch (-1 where none)."""
    L = len(ids)
    P_ = len(px)
    amin = oracle.ALPHA_MIN
    flags = {}
    span = np.full((P_, 2), -1, np.int64)
    if L:
        power, alpha, lo, hi, r = _tile_alpha(pre, ids, px, py, bounds, rec)
        used = (power <= 0) & (alpha >= amin)
        au = np.where(used, alpha, 0.0)
        T_after = np.cumprod(1.0 - au, axis=1)
        T_before = np.concatenate([np.ones((P_, 1)), T_after[:, :-1]], 1)
        # relative error of T after each entry: its alpha's error through 1 - alpha, and the
        # rounding of T - alpha T (eps / (1 - alpha): the subtraction cancels)
        step = np.where(used, au / (1.0 - au) * np.where(used, r, 0.0)
                        + 2.0 * EPS32 / (1.0 - au), 0.0)
        rT_after = np.cumsum(step, axis=1)
        rT_before = np.concatenate([np.zeros((P_, 1)), rT_after[:, :-1]], 1)
        pos = np.arange(L)[None, :]
        first = np.where(T_after < oracle.T_STOP, pos, L).min(axis=1)
        live = pos <= first[:, None]
        near_a = live & (lo <= amin) & (hi >= amin)
        near_t = live & used & (np.abs(T_after - oracle.T_STOP)
                                <= 2.0 * rT_after * T_after + 4 * EPS32 * oracle.T_STOP)
        flags["alpha"] = near_a.any(axis=1)
        flags["stop"] = near_t.any(axis=1)
        w = np.where(hi >= amin, alpha * T_before, 0.0)
        rw = np.where(hi >= amin, r, 0.0) + rT_before + EPS32
        last_used = np.where(used & live & (pos < first[:, None]), pos, -1).max(axis=1)
    else:
        w = rw = near_a = near_t = np.zeros((P_, 0))
        first = np.zeros(P_, np.int64)
        last_used = np.full(P_, -1)

    def reaches(g):
        return _tile_alpha(pre, g, px, py, bounds, rec)[3] >= amin

    mem = _membership_suspects(pre, ids, tid, gx, exempt, gid)
    if len(mem):
        m = np.any(reaches(mem), axis=1)
        flags["member"] = m
        span[m] = (0, max(L - 1, 0))            # an entry added or removed anywhere
    pairs = _order_suspects(ids, gid, pre, bounds["z"])
    if len(pairs):
        u, inv = np.unique(pairs, return_inverse=True)
        hit = reaches(u)                                        # [P, unique]
        inv = inv.reshape(-1, 2)
        both = hit[:, inv[:, 0]] & hit[:, inv[:, 1]]            # [P, pairs]
        where = {int(g): k for k, g in enumerate(ids)}
        pp = np.array([[where.get(int(a), -1), where.get(int(b), -1)] for a, b in pairs])
        plo = np.minimum(pp[:, 0], pp[:, 1])[None, :]
        phi = np.maximum(pp[:, 0], pp[:, 1])[None, :]
        if last_entry:
            # a swap of entries that both precede the pixel's last composited entry, or both
            # follow its stop, leaves both unchanged (the transmittance after the pair is the
            # same product)
            both = both & (phi >= last_used[:, None]) & (plo <= first[:, None])
        o = both.any(axis=1)
        flags["order"] = o
        lo = np.where(both, plo, L).min(axis=1)
        hi = np.where(both, phi, -1).max(axis=1)
        sel = o & ~flags.get("member", np.zeros(P_, bool))
        span[sel] = np.stack([lo[sel], hi[sel]], 1)
    return flags, dict(w=w, rw=rw, near_a=near_a, near_t=near_t, first=first, span=span)


def pixel_exemptions(pre, lists, cam, exempt, gpu_lists, bounds, detail=False,
                     last_entry=True, rec=None):
    """Boolean [H, W] of the pixels whose float32 compositing decisions may legitimately
    differ from the oracle's, over the tiles in ``lists`` (the oracle's {tile: ids}; other
    pixels False). ``bounds``: ``f32_bounds`` of the frame. Reasons:
      alpha   an entry reached before the pixel's stop has alpha within twice its float32
              error bound (``_tile_alpha``) of 1/255;
      stop    a composited entry leaves a transmittance within twice its float32 error
              bound (the alpha bounds of the entries so far, through 1 - alpha) of 1e-4;
      member  a Gaussian whose membership in the tile may differ (``_membership_suspects``)
              reaches alpha >= 1/255 (within its bound) there;
      order   two entries whose order may differ (``_order_suspects``) both reach it (with
              ``last_entry``: and the pair touches the pixel's last composited entry or its
              stop, the only way a swap changes them).
    ``gpu_lists`` ({tile: ids}) makes member and order exact; None bounds them from the
    oracle's side (exempt Gaussians near the tile; depth ties within the depth bounds).
    ``rec``: the GPU's records of the view, see ``_tile_alpha``. With ``detail``, also the
    pixel counts per reason."""
    W, H = cam.width, cam.height
    gx = (W + oracle.TILE - 1) // oracle.TILE
    out = np.zeros((H, W), bool)
    why = dict(alpha=0, stop=0, member=0, order=0)
    for tid, ids in lists.items():
        ids = np.asarray(ids, np.int64)
        px, py = oracle.tile_pixels(int(tid), gx, W, H)
        px, py = px.numpy(), py.numpy()
        gid = None
        if gpu_lists is not None and tid in gpu_lists:
            gid = np.asarray(gpu_lists[tid], np.int64)
        flags, _ = _tile_flags(pre, ids, int(tid), gx, px.astype(np.float64),
                               py.astype(np.float64), exempt, gid, bounds, last_entry, rec)
        flag = np.zeros(len(px), bool)
        for k, f in flags.items():
            why[k] += int(f.sum())
            flag |= f
        out[py, px] = flag
    return (out, why) if detail else out


def score_pixel_weights(P, cam, t, gpu_lists=None, rec=None, active=None):
    """For one render, per Gaussian: the oracle's exemption, a bound on how much of its blend
    weight (Eq. 4) the float32 decisions at the render's exempt pixels (``pixel_exemptions``)
    can change, and a first-order bound on the float32 error of its weight elsewhere.
    Decision bounds:
      alpha   the entry near the floor and the entry at the stop, all of their weight; every
              later entry reached, 0.4% of its weight (its transmittance moves by 1 - alpha,
              alpha ~ 1/255);
      stop    the entry near the stop, all of its weight (the other renderer stops at the
              next entry with alpha >= 1/255 either way);
      member  every entry, all of its weight; order: the entries between the pair, all.
    "All of its weight" is alpha T with T the transmittance ignoring the stop rule. The
    rounding bound sums alpha T (r_alpha + r_T) over the pixels (``_tile_flags``; ``rec``:
    the GPU's records of the view, see ``_tile_alpha``). Returns (exempt [N], decision bound
    [N], rounding bound [N], counts)."""
    pre = oracle.preprocess(P, cam, f32(t), active)
    n = P.mean4.shape[0]
    mean4 = P.mean4.detach().numpy()
    ex = exempt_gaussians(pre, cam, mean4)
    bounds = f32_bounds(pre, cam, mean4)
    offs, all_ids = oracle.tile_lists(pre)
    gx, gy = pre["grid"]
    W, H = cam.width, cam.height
    dec = np.zeros(n)
    rnd = np.zeros(n)
    why = dict(alpha=0, stop=0, member=0, order=0)
    nex = 0
    for tid in range(gx * gy):
        ids = np.asarray(all_ids[offs[tid]:offs[tid + 1]], np.int64)
        if not len(ids):
            continue
        px, py = oracle.tile_pixels(int(tid), gx, W, H)
        px, py = px.numpy().astype(np.float64), py.numpy().astype(np.float64)
        gid = None
        if gpu_lists is not None and tid in gpu_lists:
            gid = np.asarray(gpu_lists[tid], np.int64)
        flags, d = _tile_flags(pre, ids, tid, gx, px, py, ex, gid, bounds, False, rec)
        w = d["w"]                                           # [P, L]
        L = len(ids)
        pos = np.arange(L)[None, :]
        live = pos <= d["first"][:, None]
        np.add.at(rnd, ids, np.where(live, w * d["rw"], 0.0).sum(0))
        anyf = np.zeros(len(px), bool)
        for k, f in flags.items():
            why[k] += int(f.sum())
            anyf |= f
        nex += int(anyf.sum())
        if not anyf.any():
            continue
        aff = np.zeros_like(w)
        if "alpha" in flags:
            fa = flags["alpha"]
            k0 = np.where(d["near_a"], pos, L).min(axis=1)    # first entry near the floor
            after = fa[:, None] & (pos > k0[:, None])
            aff += np.where(after, 0.004 * w, 0.0)
            at_k = fa[:, None] & (d["near_a"] | (pos == np.minimum(d["first"], L - 1)[:, None]))
            aff = np.where(at_k, w, aff)
        if "stop" in flags:
            aff = np.where(d["near_t"], w, aff)
        sp = d["span"]
        has = sp[:, 0] >= 0
        if has.any():
            inside = has[:, None] & (pos >= sp[:, :1]) & (pos <= sp[:, 1:])
            aff = np.where(inside, w, aff)
        np.add.at(dec, ids, aff.sum(0))
    return ex, dec, rnd, dict(exempt_pixels=nex, pixels=W * H, **why)


def last_blended(ranges, ids, n_contrib, tiles, cam):
    """The Gaussian id of each pixel's last composited entry (-1 for none): entry
    n_contrib - 1 of its tile's list. ranges [tiles, 2] and ids [K] in the export layout, or
    ranges None with ``ids`` a {tile: ids} dict."""
    W, H = cam.width, cam.height
    gx = (W + oracle.TILE - 1) // oracle.TILE
    out = np.full((H, W), -2, np.int64)
    for tid in tiles:
        px, py = oracle.tile_pixels(int(tid), gx, W, H)
        px, py = px.numpy(), py.numpy()
        lst = np.asarray(ids[tid] if ranges is None
                         else ids[int(ranges[tid, 0]):int(ranges[tid, 1])], np.int64)
        nc = np.asarray(n_contrib)[py, px].astype(np.int64)
        ok = (nc >= 1) & (nc <= len(lst))
        val = np.full(len(px), -1, np.int64)
        val[ok] = lst[nc[ok] - 1]
        val[(nc > len(lst))] = -3
        out[py, px] = val
    return out


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
