"""Vector quantisation of the spherical-harmonic colour coefficients (the post-processing of
Sec. 5, "Implementation Details": Ours-PP quantises SH into a codebook). An offline step, run
once per scene: the renderer then decodes inside its per-Gaussian kernel
(``Scene.set_sh_codebook``), reading 2 bytes of code instead of 180 bytes of higher-band
coefficients per Gaussian.

Reading (the paper gives no codebook details): the DC coefficients stay per Gaussian; the
(K-1) x 3 higher-band coefficients of each Gaussian form one vector, quantised by k-means with
n_code centroids (seeded sample initialisation, Lloyd iterations, a final assignment so every
code is a nearest centroid).
"""
from __future__ import annotations

import torch


def _assign(x: torch.Tensor, c: torch.Tensor, chunk: int = 32768) -> torch.Tensor:
    """Index of the nearest centroid (squared Euclidean) for every row of x."""
    c2 = (c * c).sum(1)
    out = torch.empty(x.shape[0], dtype=torch.long, device=x.device)
    for s in range(0, x.shape[0], chunk):
        xs = x[s:s + chunk]
        d = c2[None, :] - 2.0 * (xs @ c.T)          # + |x|^2, the same for every centroid
        out[s:s + chunk] = torch.argmin(d, dim=1)
    return out


def quantize_sh(sh: torch.Tensor, n_code: int = 4096, iters: int = 10, seed: int = 0):
    """sh [K][3][N] (K >= 4) -> (codebook float32 [n_code][K-1][3], codes [N] int16 bit
    patterns of uint16 indices). n_code is capped at N."""
    K, three, N = sh.shape
    assert three == 3 and K >= 4
    x = sh[1:].permute(2, 0, 1).reshape(N, (K - 1) * 3).float().contiguous()
    n_code = int(min(n_code, N))
    g = torch.Generator(device="cpu").manual_seed(seed)
    idx = torch.randperm(N, generator=g)[:n_code].to(x.device)
    cent = x[idx].clone()
    for _ in range(iters):
        codes = _assign(x, cent)
        sums = torch.zeros_like(cent).index_add_(0, codes, x)
        counts = torch.bincount(codes, minlength=n_code)
        nz = counts > 0
        cent[nz] = sums[nz] / counts[nz, None].to(x.dtype)
    codes = _assign(x, cent)
    codes16 = codes.to(torch.int32).to(torch.int16)      # bit pattern of the uint16 index
    return cent.reshape(n_code, K - 1, 3).contiguous(), codes16.contiguous()


def decode_sh(sh_dc: torch.Tensor, codebook: torch.Tensor, codes: torch.Tensor) -> torch.Tensor:
    """Full coefficients [K][3][N]: plane 0 from sh_dc ([1][3][N] or a full [K][3][N] array),
    planes 1..K-1 from codebook[codes]."""
    idx = codes.to(torch.int64) & 0xFFFF
    rest = codebook[idx]                                  # [N][K-1][3]
    return torch.cat([sh_dc[:1], rest.permute(1, 2, 0)], 0).contiguous()


def storage_bytes(n: int, sh_degree: int, n_code: int) -> dict:
    """Bytes of the colour coefficients: full SH vs DC + 16-bit code + the shared codebook."""
    k = (sh_degree + 1) ** 2
    return dict(full=n * k * 3 * 4, quantised=n * (3 * 4 + 2) + n_code * (k - 1) * 3 * 4)
