"""Brute-force NumPy renderers used to pin the oracle (tests only).

Written independently of oracle/: plain loops over pixels and Gaussians, no tile lists, no
vectorised cumulative products. Thresholds restate the float32 constants of the blending rule
(alpha < 1/255 skipped, alpha clamped at 0.99, stop before T drops under 1e-4).
"""
import math

import numpy as np

A_MIN = float(np.float32(1.0 / 255.0))
A_MAX = float(np.float32(0.99))
T_MIN = float(np.float32(1e-4))


def tile_covered(u, r, tile_index):
    """Whether a Gaussian at image coordinate u with integer radius r reaches tile
    ``tile_index`` along one axis: the tile's first pixel 16*i must satisfy
    u - r < 16*i + 16 and 16*i + 1 <= u + r."""
    lo = 16 * tile_index
    return (u - r < lo + 16) and (lo + 1 <= u + r)


def composite_pixels(mean2d, conic, a, rgb, depth, radius, visible, W, H, blended=None,
                     stoppers=None):
    """Per-pixel front-to-back compositing over all visible Gaussians whose rectangle covers
    the pixel's tile, in (depth, id) order. Returns image [3,H,W], T [H,W], n_contrib [H,W]
    (1 + position in the candidate list of the last blended Gaussian). If ``blended`` /
    ``stoppers`` are sets, the ids blended at one pixel at least / that stopped a pixel are
    added to them."""
    n = len(a)
    img = np.zeros((3, H, W))
    Tout = np.ones((H, W))
    nc = np.zeros((H, W), np.int64)
    order = sorted([i for i in range(n) if visible[i]], key=lambda i: (depth[i], i))
    for py in range(H):
        for px in range(W):
            tx, ty = px // 16, py // 16
            T = 1.0
            C = np.zeros(3)
            pos = 0
            last = 0
            for i in order:
                if not (tile_covered(mean2d[i][0], radius[i], tx)
                        and tile_covered(mean2d[i][1], radius[i], ty)):
                    continue
                pos += 1
                dx = mean2d[i][0] - px
                dy = mean2d[i][1] - py
                A, B, Cc = conic[i]
                power = -0.5 * (A * dx * dx + Cc * dy * dy) - B * dx * dy
                if power > 0:
                    continue
                alpha = min(A_MAX, a[i] * math.exp(power))
                if alpha < A_MIN:
                    continue
                nT = T * (1.0 - alpha)
                if nT < T_MIN:
                    if stoppers is not None:
                        stoppers.add(i)
                    break
                C += np.asarray(rgb[i]) * alpha * T
                T = nT
                last = pos
                if blended is not None:
                    blended.add(i)
            img[:, py, px] = C
            Tout[py, px] = T
            nc[py, px] = last
    return img, Tout, nc


def project_static(mu3, cov3, cam):
    """EWA projection of static 3D Gaussians, one at a time (loops). Returns per Gaussian:
    (ok, depth, (u, v), conic (A,B,C), radius)."""
    V = np.asarray(cam.viewmat, np.float64)
    W, H = cam.width, cam.height
    out = []
    for i in range(len(mu3)):
        pc = V[:3, :3] @ mu3[i] + V[:3, 3]
        z = pc[2]
        if z <= cam.znear:
            out.append((False, z, (0, 0), (0, 0, 0), 0))
            continue
        tanx, tany = W / (2 * cam.fx), H / (2 * cam.fy)
        xr = min(max(pc[0] / z, -1.3 * tanx), 1.3 * tanx)
        yr = min(max(pc[1] / z, -1.3 * tany), 1.3 * tany)
        Jm = np.array([[cam.fx / z, 0.0, -cam.fx * xr / z],
                       [0.0, cam.fy / z, -cam.fy * yr / z]])
        T = Jm @ V[:3, :3]
        S2 = T @ cov3[i] @ T.T + 0.3 * np.eye(2)
        det = np.linalg.det(S2)
        if det <= 0:
            out.append((False, z, (0, 0), (0, 0, 0), 0))
            continue
        inv = np.linalg.inv(S2)
        # radius rule: ceil(3 sqrt(lambda_max)), lambda_max with the discriminant floored
        mid = 0.5 * (S2[0, 0] + S2[1, 1])
        lam = mid + math.sqrt(max(0.1, mid * mid - det))
        r = math.ceil(3.0 * math.sqrt(lam))
        u = cam.fx * pc[0] / z + cam.cx
        v = cam.fy * pc[1] / z + cam.cy
        out.append((True, z, (u, v), (inv[0, 0], inv[0, 1], inv[1, 1]), r))
    return out


def render_static(mu3, cov3, opacity, rgb, cam):
    """Static 3D Gaussian splatting image by brute force (no tile lists)."""
    proj = project_static(mu3, cov3, cam)
    n = len(mu3)
    W, H = cam.width, cam.height
    gx, gy = (W + 15) // 16, (H + 15) // 16
    vis = np.zeros(n, bool)
    for i, (ok, z, (u, v), con, r) in enumerate(proj):
        if not ok or opacity[i] < A_MIN:
            continue
        covers_x = any(tile_covered(u, r, tx) for tx in range(gx))
        covers_y = any(tile_covered(v, r, ty) for ty in range(gy))
        vis[i] = covers_x and covers_y
    mean2d = [p[2] for p in proj]
    conic = [p[3] for p in proj]
    depth = [p[1] for p in proj]
    radius = [p[4] for p in proj]
    return composite_pixels(mean2d, conic, opacity, rgb, depth, radius, vis, W, H)


def quat_mul(p, q):
    """Hamilton product of two quaternions (w, x, y, z)."""
    a1, b1, c1, d1 = p
    a2, b2, c2, d2 = q
    return np.array([a1 * a2 - b1 * b2 - c1 * c2 - d1 * d2,
                     a1 * b2 + b1 * a2 + c1 * d2 - d1 * c2,
                     a1 * c2 - b1 * d2 + c1 * a2 + d1 * b2,
                     a1 * d2 + b1 * c2 - c1 * b2 + d1 * a2])


def rotation_by_products(ql, qr):
    """4D rotation v -> ql * v * qr (unit quaternions), built column by column from Hamilton
    products of the basis quaternions."""
    ql = np.asarray(ql, np.float64) / np.linalg.norm(ql)
    qr = np.asarray(qr, np.float64) / np.linalg.norm(qr)
    cols = [quat_mul(quat_mul(ql, e), qr) for e in np.eye(4)]
    return np.stack(cols, 1)
