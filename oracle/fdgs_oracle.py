"""FP64 CPU oracle of the masked 4D Gaussian rasterizer (4DGS-1K, arXiv 2503.16422).

TEST INFRASTRUCTURE. Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import this module. The CUDA library never calls it and shares no code
with it; the only thing both sides share is the seeded input generator.

Everything is plain PyTorch CPU arithmetic in float64, written in the order the method states
it, with no blocking or fusion. Gradients come from autograd through this same forward.

Method steps and where they come from:
  * key-frame selection and mask gate ........ Sec. 4.2.2 ("Filter based Rendering")
  * 4D covariance from scales and the left/right quaternion pair ... Sec. 3 (Preliminary)
  * conditional 3D Gaussian at time t ........ Sec. 3, Eq. 1
  * marginal temporal weight p_i(t), alpha ... Sec. 3, Eq. 3
  * depth-sorted front-to-back compositing ... Sec. 3, Eq. 2
  * spatial score, temporal variation score, pruning ... Sec. 4.2.1, Eqs. 4-7
  * key-frame masks from the training views .. Sec. 4.2.2 ("Key-frame based Temporal
    Filtering"); active ratio and activation IoU ... Sec. 4.1 ("Inactive Gaussians")
The paper leaves the projection, thresholds and colour model to the 3DGS/4DGS renderer it
builds on; the readings used for those are listed where they are used (constants below).

Thresholds are the float32 constants promoted to double, so that the oracle's decisions sit
at the same points as a float32 renderer's.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

F64 = torch.float64
TILE = 16
ALPHA_MIN = float(np.float32(1.0 / 255.0))     # skip alpha below this (3DGS-family reading)
ALPHA_MAX = float(np.float32(0.99))            # alpha clamp
T_STOP = float(np.float32(1e-4))               # stop when transmittance would drop below
COV2D_DILATION = 0.3                           # px^2 added to the 2D covariance diagonal
CLAMP_FOV = 1.3                                # Jacobian clamp, x 1/2 tan(fov)
RADIUS_FLOOR = 0.1                             # floor of the eigenvalue discriminant
SH_C0 = 0.28209479177387814                    # 1 / (2 sqrt(pi))


# ----------------------------------------------------------------------------------------
# Temporal filter (Sec. 4.2.2)
# ----------------------------------------------------------------------------------------

def keyframe_pair(key_times, t):
    """The two nearest key-frames of t: l = last key-frame with t_l <= t (0 if t precedes all),
    r = l + 1 clamped to the last key-frame (Sec. 4.2.2, "two nearest key-frames")."""
    kt = np.asarray(key_times, np.float64)
    n = len(kt)
    l = 0
    for i in range(n):
        if kt[i] <= t:
            l = i
    r = min(l + 1, n - 1)
    return l, r


def active_from_masks(mask_bits, key_times, t, n):
    """Active set at t: union of the masks of the two nearest key-frames (Sec. 4.2.2).
    mask_bits is [n_key, ceil(n/8)] LSB-first packed bytes. No masks -> everything active."""
    if mask_bits is None or len(key_times) == 0:
        return np.ones(n, bool)
    l, r = keyframe_pair(key_times, t)
    bits = np.asarray(mask_bits, np.uint8)
    ml = np.unpackbits(bits[l], bitorder="little")[:n].astype(bool)
    mr = np.unpackbits(bits[r], bitorder="little")[:n].astype(bool)
    return ml | mr


# ----------------------------------------------------------------------------------------
# 4D Gaussian (Sec. 3)
# ----------------------------------------------------------------------------------------

def left_quat_matrix(q):
    """Matrix of v -> q * v (Hamilton product, v as a quaternion (v0, v1, v2, v3))."""
    a, b, c, d = q.unbind(-1)
    return torch.stack([
        torch.stack([a, -b, -c, -d], -1),
        torch.stack([b, a, -d, c], -1),
        torch.stack([c, d, a, -b], -1),
        torch.stack([d, -c, b, a], -1)], -2)


def right_quat_matrix(q):
    """Matrix of v -> v * q (Hamilton product)."""
    p, q1, r, s = q.unbind(-1)
    return torch.stack([
        torch.stack([p, -q1, -r, -s], -1),
        torch.stack([q1, p, s, -r], -1),
        torch.stack([r, -s, p, q1], -1),
        torch.stack([s, r, -q1, p], -1)], -2)


def rotation_4d(q_left, q_right):
    """R_4D from the left/right quaternion pair (Sec. 3): R = L(q_l/|q_l|) R(q_r/|q_r|),
    acting on (x, y, z, t) with t the fourth coordinate."""
    ql = q_left / q_left.norm(dim=-1, keepdim=True)
    qr = q_right / q_right.norm(dim=-1, keepdim=True)
    return left_quat_matrix(ql) @ right_quat_matrix(qr)


def covariance_4d(logscale4, q_left, q_right):
    """Sigma = R S S^T R^T with S = diag(exp(logscale)) (Sec. 3)."""
    R = rotation_4d(q_left, q_right)
    s2 = torch.exp(2.0 * logscale4)
    return (R * s2[..., None, :]) @ R.transpose(-1, -2)


def condition_on_time(mean4, cov4, t):
    """Eq. 1: conditional 3D mean and covariance at time t, plus Sigma_t = Sigma_44 and the
    marginal temporal weight p(t) = exp(-(t - mu_t)^2 / (2 Sigma_t)) (Eq. 3, unnormalised,
    peak 1)."""
    s_xt = cov4[..., :3, 3]
    s_tt = cov4[..., 3, 3]
    dt = t - mean4[..., 3]
    mu3 = mean4[..., :3] + s_xt / s_tt[..., None] * dt[..., None]
    cov3 = cov4[..., :3, :3] - s_xt[..., :, None] * s_xt[..., None, :] / s_tt[..., None, None]
    p = torch.exp(-0.5 * dt * dt / s_tt)
    return mu3, cov3, s_tt, p


# ----------------------------------------------------------------------------------------
# Colour: real spherical harmonics, degree <= 3 (reading: the paper only says "colour of
# each Gaussian", Eq. 2; the standard real SH basis without the Condon-Shortley phase)
# ----------------------------------------------------------------------------------------

def sh_basis(d, degree):
    """Real SH values Y_k(d), k = l^2 + l + m, for unit directions d [N,3] -> [N,(deg+1)^2]."""
    x, y, z = d.unbind(-1)
    out = [torch.full_like(x, SH_C0)]
    if degree >= 1:
        c1 = math.sqrt(3.0 / (4.0 * math.pi))
        out += [c1 * y, c1 * z, c1 * x]
    if degree >= 2:
        c2a = 0.5 * math.sqrt(15.0 / math.pi)
        c2b = 0.25 * math.sqrt(5.0 / math.pi)
        c2c = 0.25 * math.sqrt(15.0 / math.pi)
        out += [c2a * x * y, c2a * y * z, c2b * (3.0 * z * z - 1.0), c2a * x * z,
                c2c * (x * x - y * y)]
    if degree >= 3:
        c3a = 0.25 * math.sqrt(35.0 / (2.0 * math.pi))
        c3b = 0.5 * math.sqrt(105.0 / math.pi)
        c3c = 0.25 * math.sqrt(21.0 / (2.0 * math.pi))
        c3d = 0.25 * math.sqrt(7.0 / math.pi)
        c3e = 0.25 * math.sqrt(105.0 / math.pi)
        out += [c3a * y * (3.0 * x * x - y * y), c3b * x * y * z,
                c3c * y * (5.0 * z * z - 1.0), c3d * z * (5.0 * z * z - 3.0),
                c3c * x * (5.0 * z * z - 1.0), c3e * z * (x * x - y * y),
                c3a * x * (x * x - 3.0 * y * y)]
    return torch.stack(out, -1)


# ----------------------------------------------------------------------------------------
# Scene / camera containers (float64 torch views of the generator's arrays)
# ----------------------------------------------------------------------------------------

@dataclass
class Params:
    mean4: torch.Tensor
    logscale4: torch.Tensor
    q_left: torch.Tensor
    q_right: torch.Tensor
    opacity_logit: torch.Tensor
    sh: torch.Tensor          # [K,3,N]
    sh_degree: int

    @staticmethod
    def from_scene(scene, requires_grad=False):
        def t(a):
            x = torch.as_tensor(np.asarray(a, np.float64), dtype=F64).clone()
            return x.requires_grad_(requires_grad)
        return Params(t(scene.mean4), t(scene.logscale4), t(scene.q_left), t(scene.q_right),
                      t(scene.opacity_logit), t(scene.sh), int(scene.sh_degree))

    def tensors(self):
        return [self.mean4, self.logscale4, self.q_left, self.q_right, self.opacity_logit,
                self.sh]


def camera_f64(cam):
    V = torch.as_tensor(np.asarray(cam.viewmat, np.float64), dtype=F64)
    return V


# ----------------------------------------------------------------------------------------
# Per-Gaussian stage: gate, slice, cull, project (EWA), colour, tile rectangle
# ----------------------------------------------------------------------------------------

def tight_tile_rect(mean2d, conic, a, rect):
    """The alpha-tight tile set (the per-frame option and the batched path): the 3-sigma
    rectangle ``rect`` [N,4] (xmin, ymin, xmax, ymax) intersected with the tiles of the
    bounding box of the ellipse d^T Sigma^-1 d <= Q', Q' = 1.001 * 2 ln(255 a) + 0.1, the
    region where a pixel can take alpha >= 1/255 from the Gaussian, widened for a float32
    renderer. Half-widths sqrt(Q' Sigma_xx), sqrt(Q' Sigma_yy) with Sigma = conic^-1. An empty
    result is (0, 0, 0, 0); a degenerate conic keeps the rectangle. Returns (rect, the four
    box edges in pixels)."""
    A, B, C = conic.unbind(-1)
    dc = A * C - B * B
    Q = 2.0 * torch.log(255.0 * a) * 1.001 + 0.1
    ok = dc > 0
    dcs = torch.where(ok, dc, torch.ones_like(dc))
    Qp = torch.clamp(Q, min=0.0)
    hx = torch.sqrt(Qp * C / dcs)
    hy = torch.sqrt(Qp * A / dcs)
    u, v = mean2d.unbind(-1)
    edges = torch.stack([u - hx, v - hy, u + hx, v + hy], -1)
    box = torch.stack([torch.floor(edges[:, 0] / TILE), torch.floor(edges[:, 1] / TILE),
                       torch.floor(edges[:, 2] / TILE) + 1, torch.floor(edges[:, 3] / TILE) + 1],
                      -1).long()
    lo = torch.maximum(rect[:, :2], box[:, :2])
    hi = torch.minimum(rect[:, 2:], box[:, 2:])
    out = torch.where(ok[:, None], torch.cat([lo, hi], -1), rect)
    empty = (Q <= 0) | (out[:, 2] <= out[:, 0]) | (out[:, 3] <= out[:, 1])
    return torch.where(empty[:, None], torch.zeros_like(out), out), edges


def preprocess(P: Params, cam, t, active=None, tile_sets="square", temporal_cull=True):
    """Per-Gaussian preparation for one (camera, t). Returns a dict of float64 tensors
    (differentiable where the method is) and boolean/int decisions (detached).
    ``tile_sets``: "square" (the 3DGS-family 3-sigma rectangle, the reference) or "tight"
    (that rectangle cut to the tiles the alpha >= 1/255 ellipse can reach, see
    tight_tile_rect; the image is the same, the lists shorter).

    Order (Sec. 3 and 4.2.2): mask gate -> 4D covariance -> Eq. 1 slice and p(t) (Eq. 3) ->
    a = sigmoid(o) p(t), culled when a < 1/255 (then alpha < 1/255 everywhere) -> camera
    transform, near-plane cull z <= znear -> EWA 2D covariance + 0.3 px^2 -> conic ->
    radius ceil(3 sqrt(lambda_max)) -> tile rectangle -> SH colour.
    ``temporal_cull=False`` skips the a < 1/255 cull (a renderer without it: such Gaussians
    are projected and binned but reach alpha >= 1/255 at no pixel); ``pass_temporal`` still
    records a >= 1/255.
    """
    n = P.mean4.shape[0]
    t = float(t)
    act = torch.ones(n, dtype=torch.bool) if active is None else torch.as_tensor(active)
    cov4 = covariance_4d(P.logscale4, P.q_left, P.q_right)
    mu3, cov3, s_tt, p = condition_on_time(P.mean4, cov4, t)
    sigma = torch.sigmoid(P.opacity_logit)
    a = sigma * p
    V = camera_f64(cam)
    Rv, tv = V[:3, :3], V[:3, 3]
    xc = mu3 @ Rv.T + tv
    x, y, z = xc.unbind(-1)
    W, H = cam.width, cam.height
    fx, fy = float(cam.fx), float(cam.fy)
    cx, cy = float(cam.cx), float(cam.cy)
    zsafe = torch.where(z > cam.znear, z, torch.ones_like(z))
    limx = CLAMP_FOV * (W / (2.0 * fx))
    limy = CLAMP_FOV * (H / (2.0 * fy))
    xz = torch.clamp(x / zsafe, -limx, limx)
    yz = torch.clamp(y / zsafe, -limy, limy)
    zero = torch.zeros_like(z)
    J = torch.stack([torch.stack([fx / zsafe, zero, -fx * xz / zsafe], -1),
                     torch.stack([zero, fy / zsafe, -fy * yz / zsafe], -1)], -2)
    M = J @ Rv
    cov2 = M @ cov3 @ M.transpose(-1, -2)
    c00 = cov2[:, 0, 0] + COV2D_DILATION
    c01 = cov2[:, 0, 1]
    c11 = cov2[:, 1, 1] + COV2D_DILATION
    det = c00 * c11 - c01 * c01
    detsafe = torch.where(det > 0, det, torch.ones_like(det))
    conA, conB, conC = c11 / detsafe, -c01 / detsafe, c00 / detsafe
    u = fx * x / zsafe + cx
    v = fy * y / zsafe + cy
    with torch.no_grad():
        mid = 0.5 * (c00 + c11)
        lam = mid + torch.sqrt(torch.clamp(mid * mid - det, min=RADIUS_FLOOR))
        r3 = 3.0 * torch.sqrt(torch.clamp(lam, min=0.0))
        radius = torch.ceil(r3)
        gx, gy = (W + TILE - 1) // TILE, (H + TILE - 1) // TILE
        xlo_f, xhi_f = u - radius, u + radius + (TILE - 1)
        ylo_f, yhi_f = v - radius, v + radius + (TILE - 1)
        xmin = torch.clamp(torch.floor(xlo_f / TILE), 0, gx).long()
        xmax = torch.clamp(torch.floor(xhi_f / TILE), 0, gx).long()
        ymin = torch.clamp(torch.floor(ylo_f / TILE), 0, gy).long()
        ymax = torch.clamp(torch.floor(yhi_f / TILE), 0, gy).long()
        pass_mask = act.clone()
        pass_temporal = pass_mask & (a >= ALPHA_MIN)
        alive = pass_temporal if temporal_cull else pass_mask
        pass_near = alive & (z > cam.znear)
        pass_det = pass_near & (det > 0)
        visible = pass_det & (xmax > xmin) & (ymax > ymin)
        rect = torch.stack([xmin, ymin, xmax, ymax], -1)
        rect_tight, tight_edges = None, None
        if tile_sets == "tight":
            rect_tight, tight_edges = tight_tile_rect(
                torch.stack([u, v], -1).detach(),
                torch.stack([conA, conB, conC], -1).detach(), a.detach(), rect)
            rect = rect_tight
        elif tile_sets != "square":
            raise ValueError("tile_sets must be 'square' or 'tight'")
        ntiles = torch.where(visible, (rect[:, 2] - rect[:, 0]) * (rect[:, 3] - rect[:, 1]),
                             torch.zeros_like(xmax))
    # colour from SH at the view direction of the conditional mean
    eye = -Rv.T @ tv
    dvec = mu3 - eye
    dn = dvec / dvec.norm(dim=-1, keepdim=True)
    Y = sh_basis(dn, P.sh_degree)                              # [N,K]
    raw = torch.einsum("nk,kcn->nc", Y, P.sh) + 0.5
    rgb = torch.clamp(raw, min=0.0)
    return dict(active=act, cov4=cov4, mu3=mu3, cov3=cov3, s_tt=s_tt, p=p, sigma=sigma, a=a,
                xc=xc, depth=z, J=J, cov2=torch.stack([c00, c01, c11], -1), det=det,
                conic=torch.stack([conA, conB, conC], -1), mean2d=torch.stack([u, v], -1),
                lam=lam, r3=r3, radius=radius, rect=rect,
                rect_square=torch.stack([xmin, ymin, xmax, ymax], -1),
                rect_edges=torch.stack([xlo_f, ylo_f, xhi_f, yhi_f], -1),
                tight_edges=tight_edges, tile_sets=tile_sets,
                pass_mask=pass_mask, pass_temporal=pass_temporal, pass_near=pass_near,
                pass_det=pass_det, visible=visible, ntiles=ntiles, rgb=rgb, rgb_raw=raw,
                grid=(gx, gy))


# ----------------------------------------------------------------------------------------
# Binning and (tile, depth) ordering (Eq. 2: "blending visible Gaussians sorted by depth")
# ----------------------------------------------------------------------------------------

def tile_lists(pre):
    """Per-tile Gaussian lists. Each visible Gaussian is listed in every 16x16 tile of its
    rectangle; each list is ordered by (depth, Gaussian id) ascending.
    Returns (offsets [tiles+1], ids [K]) in CSR form, tiles numbered ty * gx + tx."""
    gx, gy = pre["grid"]
    vis = torch.nonzero(pre["visible"]).flatten()
    rect = pre["rect"][vis]
    cnt = ((rect[:, 2] - rect[:, 0]) * (rect[:, 3] - rect[:, 1])).numpy()
    ids = np.repeat(vis.numpy(), cnt)
    # enumerate the tiles of each rectangle
    start = np.repeat(np.cumsum(cnt) - cnt, cnt)
    j = np.arange(len(ids)) - start
    wdt = np.repeat((rect[:, 2] - rect[:, 0]).numpy(), cnt)
    tx = np.repeat(rect[:, 0].numpy(), cnt) + j % np.maximum(wdt, 1)
    ty = np.repeat(rect[:, 1].numpy(), cnt) + j // np.maximum(wdt, 1)
    tile = ty * gx + tx
    depth = pre["depth"].detach().numpy()[ids]
    order = np.lexsort((ids, depth, tile))
    tile, ids = tile[order], ids[order]
    offsets = np.zeros(gx * gy + 1, np.int64)
    np.add.at(offsets, tile + 1, 1)
    return np.cumsum(offsets), ids


def tile_list(pre, tile_id):
    """The list of one tile, computed directly from the rectangles (no global enumeration)."""
    gx, gy = pre["grid"]
    tx, ty = tile_id % gx, tile_id // gx
    r = pre["rect"]
    hit = pre["visible"] & (r[:, 0] <= tx) & (tx < r[:, 2]) & (r[:, 1] <= ty) & (ty < r[:, 3])
    ids = torch.nonzero(hit).flatten().numpy()
    depth = pre["depth"].detach().numpy()[ids]
    return ids[np.lexsort((ids, depth))]


# ----------------------------------------------------------------------------------------
# Front-to-back compositing of one tile (Eq. 2, Eq. 3)
# ----------------------------------------------------------------------------------------

def blend_tile(pre, ids, px, py, return_stop=False):
    """Composite the tile list ``ids`` at pixel coordinates (px, py) [P].

    Per pixel, entries in list order: power = -1/2 d^T Sigma_2D^-1 d with d = mean2D - pixel;
    skip when power > 0; alpha = min(0.99, a exp(power)); skip when alpha < 1/255; if
    T (1 - alpha) < 1e-4 stop before blending this entry; else C += c alpha T,
    T <- T (1 - alpha). Returns colour [P,3], T_final [P], n_contrib [P] (1 + list position
    of the last blended entry), and the blend weights alpha*T [P,L] (zero where not blended);
    with ``return_stop``, also the list position of the entry that stopped each pixel [P] (L
    where the list ran out).
    """
    P_ = px.shape[0]
    L = len(ids)
    if L == 0:
        out = (torch.zeros(P_, 3, dtype=F64), torch.ones(P_, dtype=F64),
               torch.zeros(P_, dtype=torch.long), torch.zeros(P_, 0, dtype=F64))
        return out + (torch.zeros(P_, dtype=torch.long),) if return_stop else out
    idx = torch.as_tensor(ids, dtype=torch.long)
    m2 = pre["mean2d"][idx]
    con = pre["conic"][idx]
    a = pre["a"][idx]
    rgb = pre["rgb"][idx]
    dx = m2[None, :, 0] - px[:, None]
    dy = m2[None, :, 1] - py[:, None]
    power = -0.5 * (con[None, :, 0] * dx * dx + con[None, :, 2] * dy * dy) \
        - con[None, :, 1] * dx * dy
    alpha = torch.clamp(a[None, :] * torch.exp(power), max=ALPHA_MAX)
    with torch.no_grad():
        used = (power <= 0) & (alpha >= ALPHA_MIN)
    alpha_u = torch.where(used, alpha, torch.zeros_like(alpha))
    T_after = torch.cumprod(1.0 - alpha_u, dim=1)
    with torch.no_grad():
        below = T_after < T_STOP
        pos = torch.arange(L)[None, :].expand(P_, L)
        first_stop = torch.where(below, pos, torch.full_like(pos, L)).min(dim=1).values
        blended = used & (pos < first_stop[:, None])
    T_before = torch.cat([torch.ones(P_, 1, dtype=F64), T_after[:, :-1]], dim=1)
    w = torch.where(blended, alpha_u * T_before, torch.zeros_like(alpha_u))
    color = w @ rgb
    one_minus = torch.where(blended, 1.0 - alpha_u, torch.ones_like(alpha_u))
    T_final = torch.prod(one_minus, dim=1)
    with torch.no_grad():
        last = torch.where(blended, pos + 1, torch.zeros_like(pos)).max(dim=1).values
    if return_stop:
        return color, T_final, last, w, first_stop
    return color, T_final, last, w


def tile_pixels(tile_id, gx, W, H):
    tx, ty = tile_id % gx, tile_id // gx
    xs = torch.arange(tx * TILE, min((tx + 1) * TILE, W))
    ys = torch.arange(ty * TILE, min((ty + 1) * TILE, H))
    py, px = torch.meshgrid(ys, xs, indexing="ij")
    return px.flatten(), py.flatten()


def render(P: Params, cam, t, active=None, tiles=None, bg=(0.0, 0.0, 0.0), weights=False,
           pre=None, tile_sets="square", temporal_cull=True):
    """Render one frame (or only the tiles listed in ``tiles``).

    Returns dict: image [3,H,W] (float64; NaN outside the rendered tiles when ``tiles`` is
    given), T_final [H,W], n_contrib [H,W], lists {tile: ids}, pre, and, with
    ``weights=True``, w_sum [N] = sum over the rendered pixels of alpha_i T_i (Eq. 4)."""
    if pre is None:
        pre = preprocess(P, cam, t, active, tile_sets, temporal_cull)
    gx, gy = pre["grid"]
    W, H = cam.width, cam.height
    todo = range(gx * gy) if tiles is None else tiles
    img = torch.full((3, H, W), float("nan"), dtype=F64)
    Tf = torch.full((H, W), float("nan"), dtype=F64)
    nc = torch.full((H, W), -1, dtype=torch.long)
    bgv = torch.as_tensor(bg, dtype=F64)
    wsum = torch.zeros(P.mean4.shape[0], dtype=F64) if weights else None
    lists = {}
    if tiles is None:
        offs, all_ids = tile_lists(pre)
    for tid in todo:
        ids = all_ids[offs[tid]:offs[tid + 1]] if tiles is None else tile_list(pre, tid)
        lists[int(tid)] = ids
        px, py = tile_pixels(int(tid), gx, W, H)
        col, T, last, w = blend_tile(pre, ids, px.to(F64), py.to(F64))
        img[:, py, px] = (col + T[:, None] * bgv[None, :]).T
        Tf[py, px] = T
        nc[py, px] = last
        if weights and len(ids):
            wsum.index_add_(0, torch.as_tensor(ids, dtype=torch.long), w.sum(0))
    return dict(image=img, T_final=Tf, n_contrib=nc, lists=lists, pre=pre, w_sum=wsum)


def render_image(P, cam, t, active=None, tiles=None):
    """Differentiable image [3,H,W] (float64, zero outside the rendered tiles)."""
    out = render(P, cam, t, active, tiles)
    img = out["image"]
    return torch.nan_to_num(img, nan=0.0), out


def gradients(scene, cam, t, dL_dimg, active=None, tiles=None):
    """Analytic gradient of L = sum(dL_dimg * image) with respect to the six parameter
    tensors (mean4, logscale4, q_left, q_right, opacity_logit, sh), by reverse-mode
    differentiation of this float64 forward. Decisions (culls, tile rectangles, order,
    alpha skip, 0.99 clamp, early stop, SH clamp at 0) carry no gradient."""
    P = Params.from_scene(scene, requires_grad=True)
    with torch.enable_grad():
        img, out = render_image(P, cam, t, active, tiles)
        g = torch.as_tensor(np.asarray(dL_dimg, np.float64), dtype=F64)
        loss = (img * g).sum()
        grads = torch.autograd.grad(loss, P.tensors(), allow_unused=True)
    res = []
    for x, gr in zip(P.tensors(), grads):
        res.append(np.zeros(tuple(x.shape)) if gr is None else gr.numpy())
    return res, out


# ----------------------------------------------------------------------------------------
# Spatial-Temporal Variation Score (Sec. 4.2.1)
# ----------------------------------------------------------------------------------------

def temporal_second_derivative(mean4, cov4, t):
    """p^(2)(t) = ((t - mu_t)^2 / Sigma_t^2 - 1/Sigma_t) p(t) (Eq. 5)."""
    s_tt = cov4[..., 3, 3]
    dt = t - mean4[..., 3]
    p = torch.exp(-0.5 * dt * dt / s_tt)
    return (dt * dt / (s_tt * s_tt) - 1.0 / s_tt) * p


def temporal_first_derivative(mean4, cov4, t):
    """p^(1)(t) = -((t - mu_t) / Sigma_t) p(t), the time derivative of Eq. 3's p(t): the
    quantity that replaces p^(2) in variant (d) of the score ablation (Table 4 and the
    supplement's variant settings)."""
    s_tt = cov4[..., 3, 3]
    dt = t - mean4[..., 3]
    p = torch.exp(-0.5 * dt * dt / s_tt)
    return -(dt / s_tt) * p


def variation_factor(mean4, cov4, t, derivative=2):
    """Per-timestamp term of S^TV (Eq. 6): 1 / (0.5 tanh(|p^(2)(t)|) + 0.5), in (1, 2];
    ``derivative=1`` puts p^(1) in place of p^(2) (score variant (d))."""
    if derivative == 1:
        pk = temporal_first_derivative(mean4, cov4, t)
    else:
        pk = temporal_second_derivative(mean4, cov4, t)
    return 1.0 / (0.5 * torch.tanh(torch.abs(pk)) + 0.5)


def volume_gamma(logscale4, beta=0.1, q=0.9):
    """gamma = Norm(V(S_4D)) (Sec. 4.2.1, following LightGaussian): V = product of the four
    activated scales, normalised by its 90th percentile (nearest rank over all N), clamped to
    [0, 1], raised to the power beta = 0.1 (reading of the unstated constants)."""
    V = torch.exp(logscale4.sum(-1))
    srt = torch.sort(V).values
    n = V.shape[0]
    k = max(int(math.ceil(q * n)), 1)
    p90 = srt[k - 1]
    return torch.clamp(V / p90, 0.0, 1.0) ** beta


SCORE_VARIANTS = ("full", "spatial", "temporal", "first_derivative", "sigma_t")


def variation_scores(scene, cams, ts, reading="R1", return_parts=False, variant="full"):
    """Spatial-Temporal Variation Score over renders at timestamps ``ts`` from cameras
    ``cams`` (no temporal filter: scoring precedes it).

    S^S_i(t, v) = sum over pixels of alpha_i T_i (Eq. 4); f_i(t) = 1/(0.5 tanh|p^(2)| + 0.5)
    (Eq. 6); gamma_i (Sec. 4.2.1). Reading R1 (the per-t product of Eq. 7):
    S_i = sum_{t,v} S^S_i(t,v) f_i(t) gamma_i. Reading R2 (S^T already summed over t):
    S_i = (gamma_i sum_t f_i(t)) (sum_{t,v} S^S_i(t,v)). The two agree for a single t.

    ``variant`` selects the score of one row of the ablation (Table 4; definitions in the
    supplement's "Variant Settings"), each in the per-t reading R1:
      "full"             (f, ours)  sum_{t,v} S^S_i(t,v) f_i(t) gamma_i
      "spatial"          (b)        sum_{t,v} S^S_i(t,v)
      "temporal"         (c)        sum_t f_i(t) gamma_i            (no render needed)
      "first_derivative" (d)        sum_{t,v} S^S_i(t,v) f1_i(t) gamma_i, f1 with p^(1)
      "sigma_t"          (e)        sum_{t,v} S^S_i(t,v) Sigma_t,i gamma_i
    """
    if variant not in SCORE_VARIANTS:
        raise ValueError(f"variant must be one of {SCORE_VARIANTS}")
    P = Params.from_scene(scene)
    with torch.no_grad():
        cov4 = covariance_4d(P.logscale4, P.q_left, P.q_right)
        gamma = volume_gamma(P.logscale4)
        S = torch.zeros(scene.n, dtype=F64)
        SS = torch.zeros(scene.n, dtype=F64)
        FT = torch.zeros(scene.n, dtype=F64)
        for t in ts:
            f = variation_factor(P.mean4, cov4, float(t))
            FT += f
            if variant == "temporal":
                S += f * gamma
                continue
            if variant == "spatial":
                g_t = torch.ones_like(f)
            elif variant == "first_derivative":
                g_t = variation_factor(P.mean4, cov4, float(t), derivative=1) * gamma
            elif variant == "sigma_t":
                g_t = cov4[:, 3, 3] * gamma
            else:
                g_t = f * gamma
            for cam in cams:
                w = render(P, cam, float(t), None, weights=True)["w_sum"]
                S += w * g_t
                SS += w
        if reading == "R2" and variant == "full":
            S = gamma * FT * SS
    if return_parts:
        return S.numpy(), dict(gamma=gamma.numpy(), spatial=SS.numpy(), ftsum=FT.numpy())
    return S.numpy()


# ----------------------------------------------------------------------------------------
# Key-frame masks (Sec. 4.2.2, "Key-frame based Temporal Filtering") and the active-set
# metrics of Sec. 4.1 ("Inactive Gaussians")
# ----------------------------------------------------------------------------------------

def contributing(P: Params, cam, t):
    """Visibility mask m_{i,j} of one view at time t, "obtained by Eq. 2": the Gaussians that
    take part in some pixel's compositing, i.e. blended there (alpha >= 1/255 before the
    pixel's stop; its weight alpha*T is then > 0) or the entry whose alpha would take T below
    the stop (it ends that pixel's list: without it the pixel would go on compositing).
    Rendered without the temporal filter (the masks are what the filter later reads)."""
    n = P.mean4.shape[0]
    mark = np.zeros(n, bool)
    with torch.no_grad():
        pre = preprocess(P, cam, float(t), None)
        gx, gy = pre["grid"]
        offs, ids = tile_lists(pre)
        for tid in range(gx * gy):
            tl = np.asarray(ids[offs[tid]:offs[tid + 1]])
            if len(tl) == 0:
                continue
            px, py = tile_pixels(tid, gx, cam.width, cam.height)
            _, _, _, w, stop = blend_tile(pre, tl, px.to(F64), py.to(F64), return_stop=True)
            mark[tl[(w > 0).any(dim=0).numpy()]] = True
            s_ = stop.numpy()
            mark[tl[s_[s_ < len(tl)]]] = True
    return mark


def build_keyframe_masks(scene, cams, key_times):
    """For each key-frame time t_i, the union over the training views j of m_{i,j}, packed
    LSB-first (bit g of row i is bit g % 8 of byte g // 8): uint8 [n_key][ceil(N/8)], the
    layout the mask gate reads."""
    P = Params.from_scene(scene)
    n = P.mean4.shape[0]
    rows = []
    for t in key_times:
        m = np.zeros(n, bool)
        for cam in cams:
            m |= contributing(P, cam, t)
        rows.append(np.packbits(m, bitorder="little"))
    if not rows:
        return np.zeros((0, (n + 7) // 8), np.uint8)
    return np.stack(rows)


def mask_row_bools(row, n):
    """Unpacked active flags [n] of one packed mask row."""
    return np.unpackbits(np.asarray(row, np.uint8), bitorder="little")[:n].astype(bool)


def active_ratio(row, n):
    """Active ratio (Sec. 4.1): active Gaussians over all views at one moment / all Gaussians."""
    return float(mask_row_bools(row, n).sum()) / max(n, 1)


def activation_iou(row_a, row_b, n):
    """Activation IoU (Sec. 4.1): |A and B| / |A or B| of two active sets (1 for two empty
    sets)."""
    a, b = mask_row_bools(row_a, n), mask_row_bools(row_b, n)
    union = int((a | b).sum())
    return 1.0 if union == 0 else float((a & b).sum()) / union


def keep_set(scores, prune_ratio=0.8):
    """Global pruning (Sec. 4.2.1, "Pruning"): rank all Gaussians by ascending (score, id) and
    drop the lowest floor(ratio * N). Returns a boolean keep vector."""
    s = np.asarray(scores, np.float64)
    n = len(s)
    order = np.lexsort((np.arange(n), s))
    keep = np.ones(n, bool)
    keep[order[: int(math.floor(prune_ratio * n))]] = False
    return keep
