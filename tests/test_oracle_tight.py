"""Pins of the oracle's alpha-tight tile sets (CPU): every pixel that can take alpha >= 1/255
from a Gaussian inside its 3-sigma square keeps its tile (brute force over all pixels), the
tight lists are subsets of the square ones and shorter, and the image is unchanged."""
import math

import numpy as np
import torch

import oracle
from paper_2503_16422_gb300 import scenes


def _setup():
    s = scenes.make_scene(300, 23, sh_degree=1, lxyz=(-1.8, 0.5), lt_long=(-1.0, 0.3))
    cam = scenes.arc_camera(5.0, 72, 56)
    return s, cam, oracle.Params.from_scene(s)


def test_tight_sets_keep_every_pixel_that_can_take_alpha():
    s, cam, P = _setup()
    with torch.no_grad():
        sq = oracle.preprocess(P, cam, 0.4)
        ti = oracle.preprocess(P, cam, 0.4, tile_sets="tight")
    m2 = sq["mean2d"].numpy()
    con = sq["conic"].numpy()
    a = sq["a"].numpy()
    rs, rt = sq["rect"].numpy(), ti["rect"].numpy()
    vis = np.nonzero(sq["visible"].numpy())[0]
    py, px = np.mgrid[0:cam.height, 0:cam.width]
    kept_pairs = 0
    for i in vis:
        dx, dy = m2[i, 0] - px, m2[i, 1] - py
        power = -0.5 * (con[i, 0] * dx * dx + con[i, 2] * dy * dy) - con[i, 1] * dx * dy
        can = (power <= 0) & (a[i] * np.exp(np.minimum(power, 0)) >= oracle.ALPHA_MIN)
        tx, ty = px // 16, py // 16
        in_sq = (rs[i, 0] <= tx) & (tx < rs[i, 2]) & (rs[i, 1] <= ty) & (ty < rs[i, 3])
        in_ti = (rt[i, 0] <= tx) & (tx < rt[i, 2]) & (rt[i, 1] <= ty) & (ty < rt[i, 3])
        assert not np.any(can & in_sq & ~in_ti), i
        assert not np.any(in_ti & ~in_sq), i          # never outside the square
        kept_pairs += int((can & in_sq).sum())
    assert kept_pairs > 1000


def test_tight_lists_are_subsets_and_the_image_is_unchanged():
    s, cam, P = _setup()
    with torch.no_grad():
        sq = oracle.render(P, cam, 0.4)
        ti = oracle.render(P, cam, 0.4, tile_sets="tight")
    n_sq = sum(len(v) for v in sq["lists"].values())
    n_ti = sum(len(v) for v in ti["lists"].values())
    for tid, ids in ti["lists"].items():
        assert set(ids) <= set(sq["lists"][tid])
        # same relative order as in the square list (depth, id)
        pos = {g: k for k, g in enumerate(sq["lists"][tid])}
        assert [pos[g] for g in ids] == sorted(pos[g] for g in ids)
    assert n_ti < 0.8 * n_sq
    assert (sq["image"] - ti["image"]).abs().max() < 1e-12
    assert (sq["T_final"] - ti["T_final"]).abs().max() < 1e-12


def test_tight_rect_special_cases():
    # an opacity below 1/255 leaves nothing; a circular Gaussian's box is its alpha disc
    rect = torch.tensor([[0, 0, 10, 10], [0, 0, 10, 10]])
    m2 = torch.tensor([[80.0, 80.0], [80.0, 80.0]], dtype=torch.float64)
    con = torch.tensor([[1 / 25.0, 0.0, 1 / 25.0], [1 / 25.0, 0.0, 1 / 25.0]],
                       dtype=torch.float64)
    a = torch.tensor([1.0 / 300.0, 0.9], dtype=torch.float64)
    r, e = oracle.tight_tile_rect(m2, con, a, rect)
    assert r[0].tolist() == [0, 0, 0, 0]
    h = math.sqrt((1.001 * 2 * math.log(255 * 0.9) + 0.1) * 25.0)
    assert abs(float(e[1, 2]) - (80 + h)) < 1e-12
    lo, hi = math.floor((80 - h) / 16), math.floor((80 + h) / 16) + 1
    assert r[1].tolist() == [lo, lo, hi, hi]
