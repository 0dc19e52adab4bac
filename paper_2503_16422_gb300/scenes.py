"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module draws scenes, cameras, timestamps and key-frame masks. It holds none of the
rasterizer's arithmetic (no slicing, projection, sorting or blending) and imports nothing
from the CUDA binding or the oracle, so both sides can take their inputs from here.

Workload shapes follow the paper's evaluation setting: N3V frames rendered at half of
2704x2028, i.e. 1352x1014, 300 frames per sequence (Sec. 5, "Datasets"); most Gaussians of a
vanilla 4DGS scene short-lived (Sec. 4.1, Fig. 2a, ~70% with small Sigma_t); about 85% of
the Gaussians inactive in any frame (Sec. 4.1, Fig. 2b); key-frame masks packed into bits
(Sec. 5, "Implementation Details", Ours-PP). The N3V and D-NeRF datasets are not used: these
draws stand in for them.

Draw order for a scene (numpy ``default_rng(seed)``): spatial means, temporal means,
spatial log-scales, temporal log-scales (standard normals), short-lifespan flags, left
quaternions, right quaternions, opacity logits, SH coefficients.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

TILE = 16
N3V_WIDTH, N3V_HEIGHT, N3V_FRAMES = 1352, 1014, 300


@dataclass
class Scene:
    """Structure-of-arrays 4D Gaussian table, float32, host memory.

    mean4 [N,4] (x,y,z,t); logscale4 [N,4] (log of the four axis scales); q_left, q_right
    [N,4] (unnormalised left/right quaternions, (w,x,y,z)); opacity_logit [N];
    sh [K,3,N] with K = (sh_degree+1)^2 coefficients per colour channel.
    """
    mean4: np.ndarray
    logscale4: np.ndarray
    q_left: np.ndarray
    q_right: np.ndarray
    opacity_logit: np.ndarray
    sh: np.ndarray
    sh_degree: int
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.mean4.shape[0])

    def subset(self, idx) -> "Scene":
        idx = np.asarray(idx)
        return Scene(self.mean4[idx].copy(), self.logscale4[idx].copy(),
                     self.q_left[idx].copy(), self.q_right[idx].copy(),
                     self.opacity_logit[idx].copy(),
                     np.ascontiguousarray(self.sh[:, :, idx]), self.sh_degree,
                     self.name + "_sub")

    def arrays(self):
        return dict(mean4=self.mean4, logscale4=self.logscale4, q_left=self.q_left,
                    q_right=self.q_right, opacity_logit=self.opacity_logit, sh=self.sh)


@dataclass
class Camera:
    """Pinhole camera. viewmat is world->camera, row-major 4x4 rigid transform with the
    OpenCV axis convention (x right, y down, z forward). Pixel (i, j) sits at image
    coordinate (i, j); the principal point defaults to the image centre ((W-1)/2, (H-1)/2).
    """
    viewmat: np.ndarray
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    znear: float = 0.2
    eye: np.ndarray = field(default_factory=lambda: np.zeros(3))


def look_at_camera(eye, width, height, fov_x_deg=60.0, target=(0.0, 0.0, 0.0),
                   up=(0.0, 1.0, 0.0), znear=0.2) -> Camera:
    """Camera at ``eye`` looking at ``target`` with world up ``up`` (+y), horizontal FOV
    ``fov_x_deg``, square pixels."""
    eye = np.asarray(eye, np.float64)
    fwd = np.asarray(target, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.asarray(up, np.float64))
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    rot = np.stack([right, down, fwd])          # rows: camera axes in world coordinates
    view = np.eye(4)
    view[:3, :3] = rot
    view[:3, 3] = -rot @ eye
    fx = (width / 2.0) / math.tan(math.radians(fov_x_deg) / 2.0)
    return Camera(view.astype(np.float32), float(np.float32(fx)), float(np.float32(fx)),
                  (width - 1) / 2.0, (height - 1) / 2.0, int(width), int(height),
                  float(znear), eye)


def arc_camera(theta_deg, width=N3V_WIDTH, height=N3V_HEIGHT, radius=4.0) -> Camera:
    """Camera on the horizontal arc eye = r (sin theta, 0, cos theta), looking at the origin."""
    th = math.radians(theta_deg)
    return look_at_camera((radius * math.sin(th), 0.0, radius * math.cos(th)), width, height)


def frame_times(n_frames=N3V_FRAMES) -> np.ndarray:
    """t_k = k / (n_frames - 1), k = 0 .. n_frames-1 (timestamps evenly in [0, 1])."""
    return (np.arange(n_frames, dtype=np.float64) / (n_frames - 1)).astype(np.float32)


def frame_theta(k, n_frames=N3V_FRAMES, span_deg=20.0) -> float:
    """Camera angle of frame k on a span_deg arc centred on +z."""
    return -span_deg / 2.0 + span_deg * k / (n_frames - 1)


def make_scene(n, seed, sh_degree=0, lt_short=None, lt_long=(-2.0, 0.5), short_frac=0.0,
               lxyz=(-3.5, 0.5), sh_dc_std=0.5, sh_rest_std=0.1, name="") -> Scene:
    """Draw a synthetic 4D Gaussian scene.

    Spatial means U[-1,1]^3, temporal means U[0,1]; spatial log-scales N(lxyz); temporal
    log-scales N(lt_long), except a fraction ``short_frac`` drawn from N(lt_short)
    (short-lifespan Gaussians); quaternions N(0,1)^4 (normalised by the renderer);
    opacity logits N(0,1); SH DC coefficients N(0, sh_dc_std), higher bands N(0, sh_rest_std).
    """
    rng = np.random.default_rng(seed)
    n = int(n)
    mxyz = rng.uniform(-1.0, 1.0, size=(n, 3))
    mt = rng.uniform(0.0, 1.0, size=(n, 1))
    lsxyz = rng.normal(lxyz[0], lxyz[1], size=(n, 3))
    zt = rng.standard_normal(size=n)
    short = rng.random(n) < short_frac if short_frac > 0 else np.zeros(n, bool)
    lst = np.where(short, (lt_short or lt_long)[0] + (lt_short or lt_long)[1] * zt,
                   lt_long[0] + lt_long[1] * zt)
    ql = rng.standard_normal(size=(n, 4))
    qr = rng.standard_normal(size=(n, 4))
    op = rng.standard_normal(size=n)
    k = (sh_degree + 1) ** 2
    sh = np.empty((k, 3, n))
    sh[0] = rng.normal(0.0, sh_dc_std, size=(3, n))
    if k > 1:
        sh[1:] = rng.normal(0.0, sh_rest_std, size=(k - 1, 3, n))
    f32 = np.float32
    return Scene(np.concatenate([mxyz, mt], 1).astype(f32),
                 np.concatenate([lsxyz, lst[:, None]], 1).astype(f32),
                 ql.astype(f32), qr.astype(f32), op.astype(f32),
                 np.ascontiguousarray(sh.astype(f32)), int(sh_degree), name)


# ---- named workloads ------------------------------------------------------------------

def tiny_scene() -> Scene:
    """2,000 Gaussians, degree-0 SH, seed 1: the small parity workload."""
    return make_scene(2000, 1, sh_degree=0, name="tiny")


def tiny_camera(width=128, height=128) -> Camera:
    return look_at_camera((0.0, 0.0, 4.0), width, height)


def pruned_scene(n=200_000, seed=2) -> Scene:
    """Pruned (4DGS-1K-like) scene: 200k Gaussians, degree-3 SH, long lifespans N(-1, 0.5)."""
    return make_scene(n, seed, sh_degree=3, lt_long=(-1.0, 0.5), name="pruned")


def unpruned_scene(n=3_000_000, seed=3) -> Scene:
    """Vanilla-4DGS-sized scene: 3M Gaussians, degree-3 SH, 70% short-lifespan N(-4, 0.5),
    30% N(-2, 0.5)."""
    return make_scene(n, seed, sh_degree=3, lt_short=(-4.0, 0.5), lt_long=(-2.0, 0.5),
                      short_frac=0.7, name="unpruned")


def stvs_scene(n=1_000_000, seed=6) -> Scene:
    """Score-pass scene: 1M Gaussians with the unpruned lifespan mix, degree-3 SH."""
    return make_scene(n, seed, sh_degree=3, lt_short=(-4.0, 0.5), lt_long=(-2.0, 0.5),
                      short_frac=0.7, name="stvs")


def keyframe_times(n_frames=N3V_FRAMES, every=6) -> np.ndarray:
    """Key-frame timestamps: every ``every``-th frame of the sequence (k = 0, 6, ...)."""
    return frame_times(n_frames)[::every].copy()


def keyframe_masks(scene: Scene, key_times, k_sigma=3.0) -> np.ndarray:
    """Synthetic key-frame active masks, LSB-first packed bits, shape [n_key, ceil(N/8)].

    Gaussian i is marked active at key-frame t_k when |t_k - mu_t| < k_sigma * s_t with
    s_t = exp(temporal log-scale). This is an input recipe (the paper builds masks from
    training-view renders); the renderer takes whatever mask it is given.
    """
    mt = scene.mean4[:, 3].astype(np.float64)
    st = np.exp(scene.logscale4[:, 3].astype(np.float64))
    rows = []
    for tk in np.asarray(key_times, np.float64):
        rows.append(np.packbits(np.abs(tk - mt) < k_sigma * st, bitorder="little"))
    return np.stack(rows).astype(np.uint8)


def pack_bits(active_bool) -> np.ndarray:
    """Pack a boolean vector LSB-first into bytes (the mask storage format)."""
    return np.packbits(np.asarray(active_bool, bool), bitorder="little")


def random_requests(n_req, seed, resolutions=((512, 512), (800, 800), (1014, 1352),
                                               (1352, 1014))):
    """Batched-serving requests: (camera on the +-10 degree arc, t ~ U[0,1], resolution
    drawn uniformly from ``resolutions`` given as (W, H))."""
    rng = np.random.default_rng(seed)
    th = rng.uniform(-10.0, 10.0, size=n_req)
    ts = rng.uniform(0.0, 1.0, size=n_req).astype(np.float32)
    ri = rng.integers(0, len(resolutions), size=n_req)
    cams = [arc_camera(float(th[i]), *resolutions[ri[i]]) for i in range(n_req)]
    return cams, ts
