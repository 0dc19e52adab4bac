"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics (CPU only).

None of these re-types an oracle formula: each compares the oracle with an independent
construction (a matrix inverse, an optimiser, scipy's spherical harmonics, Hamilton products,
brute-force loops, finite differences) or with a closed-form special case.
"""
import math

import numpy as np
import pytest
import torch

import brute
import oracle
from paper_2503_16422_gb300 import scenes

F64 = torch.float64


def _scene64(mean4, logscale4, ql, qr, op, sh, deg=0):
    return scenes.Scene(np.asarray(mean4, np.float64), np.asarray(logscale4, np.float64),
                        np.asarray(ql, np.float64), np.asarray(qr, np.float64),
                        np.asarray(op, np.float64), np.asarray(sh, np.float64), deg)


def _rand_params(n, seed):
    rng = np.random.default_rng(seed)
    mean4 = np.concatenate([rng.uniform(-1, 1, (n, 3)), rng.uniform(0, 1, (n, 1))], 1)
    ls = rng.normal(-1.5, 0.4, (n, 4))
    ql = rng.standard_normal((n, 4))
    qr = rng.standard_normal((n, 4))
    return mean4, ls, ql, qr


# ---- Sec. 3: the 4D rotation and covariance ---------------------------------------------

def test_rotation_is_special_orthogonal():
    _, _, ql, qr = _rand_params(64, 0)
    R = oracle.rotation_4d(torch.tensor(ql), torch.tensor(qr)).numpy()
    eye = np.broadcast_to(np.eye(4), R.shape)
    assert np.abs(R @ np.swapaxes(R, -1, -2) - eye).max() < 1e-13
    assert np.abs(np.linalg.det(R) - 1.0).max() < 1e-13


def test_rotation_identity_and_hamilton_products():
    one = torch.tensor([[1.0, 0, 0, 0]], dtype=F64)
    assert torch.equal(oracle.rotation_4d(one, one)[0], torch.eye(4, dtype=F64))
    _, _, ql, qr = _rand_params(16, 1)
    R = oracle.rotation_4d(torch.tensor(ql), torch.tensor(qr)).numpy()
    for i in range(16):
        ref = brute.rotation_by_products(ql[i], qr[i])
        assert np.abs(R[i] - ref).max() < 1e-13


def test_covariance_eigen_structure():
    """Sigma = R diag(s^2) R^T: eigenvalues are the squared scales, R's columns the axes."""
    mean4, ls, ql, qr = _rand_params(16, 2)
    cov = oracle.covariance_4d(torch.tensor(ls), torch.tensor(ql), torch.tensor(qr)).numpy()
    for i in range(16):
        ev = np.sort(np.linalg.eigvalsh(cov[i]))
        assert np.allclose(ev, np.sort(np.exp(2 * ls[i])), rtol=1e-10)
        # each column of R (built here from Hamilton products) is an axis with its own scale
        R = brute.rotation_by_products(ql[i], qr[i])
        for k in range(4):
            assert np.allclose(cov[i] @ R[:, k], np.exp(2 * ls[i, k]) * R[:, k], atol=1e-12)


# ---- Eq. 1 / Eq. 3: conditional 3D Gaussian and temporal marginal ------------------------

def test_eq1_matches_precision_schur_complement():
    mean4, ls, ql, qr = _rand_params(32, 3)
    cov = oracle.covariance_4d(torch.tensor(ls), torch.tensor(ql), torch.tensor(qr))
    t = 0.37
    mu3, cov3, stt, p = oracle.condition_on_time(torch.tensor(mean4), cov, t)
    for i in range(32):
        lam = np.linalg.inv(cov[i].numpy())
        cond_cov = np.linalg.inv(lam[:3, :3])
        cond_mu = mean4[i, :3] - cond_cov @ lam[:3, 3] * (t - mean4[i, 3])
        assert np.allclose(cov3[i].numpy(), cond_cov, rtol=1e-9, atol=1e-14)
        assert np.allclose(mu3[i].numpy(), cond_mu, rtol=1e-9, atol=1e-12)
        assert math.isclose(stt[i].item(), cov[i, 3, 3].item())


def test_eq1_mean_maximises_the_4d_density():
    scipy_opt = pytest.importorskip("scipy.optimize")
    mean4, ls, ql, qr = _rand_params(6, 4)
    cov = oracle.covariance_4d(torch.tensor(ls), torch.tensor(ql), torch.tensor(qr))
    t = 0.8
    mu3, _, _, _ = oracle.condition_on_time(torch.tensor(mean4), cov, t)
    for i in range(6):
        lam = np.linalg.inv(cov[i].numpy())

        def f(x):
            d = np.concatenate([x, [t]]) - mean4[i]
            return d @ lam @ d
        res = scipy_opt.minimize(f, mean4[i, :3], method="BFGS", options={"gtol": 1e-12})
        assert np.abs(res.x - mu3[i].numpy()).max() < 1e-6


def test_temporal_marginal_and_second_derivative_by_finite_differences():
    mean4, ls, ql, qr = _rand_params(16, 5)
    cov = oracle.covariance_4d(torch.tensor(ls), torch.tensor(ql), torch.tensor(qr))
    m4 = torch.tensor(mean4)
    t, h = 0.42, 1e-4

    def p(tt):
        return oracle.condition_on_time(m4, cov, tt)[3].numpy()
    fd2 = (p(t + h) - 2 * p(t) + p(t - h)) / (h * h)
    p2 = oracle.temporal_second_derivative(m4, cov, t).numpy()
    assert np.allclose(p2, fd2, rtol=1e-5, atol=1e-6)
    # the marginal peaks at 1 at t = mu_t (unnormalised reading)
    pk = oracle.condition_on_time(m4, cov, 0.0)
    for i in range(4):
        assert math.isclose(oracle.condition_on_time(m4[i:i + 1], cov[i:i + 1],
                                                     float(mean4[i, 3]))[3].item(), 1.0)


# ---- colour: real spherical harmonics ------------------------------------------------------

def _real_sh_scipy(l, m, d):
    special = pytest.importorskip("scipy.special")
    theta = np.arccos(np.clip(d[:, 2], -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])
    if hasattr(special, "sph_harm_y"):
        Y = special.sph_harm_y(l, abs(m), theta, phi)
    else:
        Y = special.sph_harm(abs(m), l, phi, theta)
    if m == 0:
        return Y.real
    sgn = (-1) ** abs(m)
    return math.sqrt(2) * sgn * (Y.real if m > 0 else Y.imag)


def test_sh_basis_matches_scipy():
    rng = np.random.default_rng(6)
    d = rng.standard_normal((200, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    Y = oracle.sh_basis(torch.tensor(d), 3).numpy()
    for l in range(4):
        for m in range(-l, l + 1):
            assert np.abs(Y[:, l * l + l + m] - _real_sh_scipy(l, m, d)).max() < 1e-12


# ---- key-frame filter (Sec. 4.2.2) ----------------------------------------------------------

def test_keyframe_pair_cases():
    kt = [0.0, 0.2, 0.4]
    assert oracle.keyframe_pair(kt, 0.0) == (0, 1)
    assert oracle.keyframe_pair(kt, 0.1) == (0, 1)
    assert oracle.keyframe_pair(kt, 0.2) == (1, 2)
    assert oracle.keyframe_pair(kt, 0.39) == (1, 2)
    assert oracle.keyframe_pair(kt, 0.4) == (2, 2)
    assert oracle.keyframe_pair(kt, 0.9) == (2, 2)
    assert oracle.keyframe_pair(kt, -0.1) == (0, 1)
    assert oracle.keyframe_pair([0.5], 0.7) == (0, 0)


def test_mask_union_of_two_keyframes():
    n = 20
    a = np.zeros(n, bool); a[[1, 5, 19]] = True
    b = np.zeros(n, bool); b[[2, 5]] = True
    c = np.zeros(n, bool); c[[7]] = True
    bits = np.stack([scenes.pack_bits(a), scenes.pack_bits(b), scenes.pack_bits(c)])
    act = oracle.active_from_masks(bits, [0.0, 0.5, 1.0], 0.25, n)
    assert np.array_equal(act, a | b)
    act = oracle.active_from_masks(bits, [0.0, 0.5, 1.0], 1.0, n)
    assert np.array_equal(act, c)


def test_all_ones_mask_equals_unmasked_and_all_zeros_is_empty():
    s = scenes.tiny_scene()
    cam = scenes.tiny_camera(64, 48)
    P = oracle.Params.from_scene(s)
    ref = oracle.render(P, cam, 0.5)
    ones = oracle.active_from_masks(np.stack([scenes.pack_bits(np.ones(s.n, bool))] * 2),
                                    [0.0, 1.0], 0.5, s.n)
    r1 = oracle.render(P, cam, 0.5, active=ones)
    assert torch.equal(ref["image"], r1["image"])
    zeros = np.zeros(s.n, bool)
    r0 = oracle.render(P, cam, 0.5, active=zeros)
    assert float(r0["image"].abs().max()) == 0.0
    assert float(r0["T_final"].min()) == 1.0
    assert int(r0["n_contrib"].max()) == 0


# ---- tiles, order and compositing (Eq. 2) -----------------------------------------------------

def test_tile_lists_match_brute_force_coverage():
    s = scenes.tiny_scene()
    cam = scenes.tiny_camera(100, 75)                # ragged: 7 x 5 tiles
    P = oracle.Params.from_scene(s)
    pre = oracle.preprocess(P, cam, 0.5)
    offs, ids = oracle.tile_lists(pre)
    gx, gy = pre["grid"]
    m2 = pre["mean2d"].detach().numpy()
    rad = pre["radius"].numpy()
    vis = pre["visible"].numpy()
    depth = pre["depth"].detach().numpy()
    for tid in range(gx * gy):
        tx, ty = tid % gx, tid // gx
        want = [i for i in np.nonzero(vis)[0]
                if brute.tile_covered(m2[i, 0], rad[i], tx)
                and brute.tile_covered(m2[i, 1], rad[i], ty)]
        want.sort(key=lambda i: (depth[i], i))
        got = list(ids[offs[tid]:offs[tid + 1]])
        assert got == want
        assert list(oracle.tile_list(pre, tid)) == want


def test_compositing_matches_per_pixel_brute_force():
    s = scenes.make_scene(60, 11, sh_degree=1, lxyz=(-2.3, 0.4))
    cam = scenes.tiny_camera(40, 36)
    P = oracle.Params.from_scene(s)
    out = oracle.render(P, cam, 0.5)
    pre = out["pre"]
    img, T, nc = brute.composite_pixels(
        pre["mean2d"].detach().numpy(), pre["conic"].detach().numpy(),
        pre["a"].detach().numpy(), pre["rgb"].detach().numpy(), pre["depth"].detach().numpy(),
        pre["radius"].numpy(), pre["visible"].numpy(), cam.width, cam.height)
    assert np.abs(out["image"].numpy() - img).max() < 1e-12
    assert np.abs(out["T_final"].numpy() - T).max() < 1e-12
    assert np.array_equal(out["n_contrib"].numpy(), nc)
    assert int(pre["visible"].sum()) > 20


def _iso_scene(means, s, st, mu_t, op_logit, sh0):
    n = len(means)
    mean4 = np.concatenate([np.asarray(means, np.float64), np.full((n, 1), mu_t)], 1)
    ls = np.tile([math.log(s)] * 3 + [math.log(st)], (n, 1))
    ident = np.tile([1.0, 0, 0, 0], (n, 1))
    sh = np.asarray(sh0, np.float64).reshape(1, 3, n)
    return _scene64(mean4, ls, ident, ident, np.full(n, op_logit), sh, 0)


def test_single_gaussian_closed_form():
    W = H = 32
    cam = scenes.look_at_camera((0.0, 0.0, 4.0), W, H)
    s, st, mu_t, t, o = 0.3, 0.2, 0.55, 0.5, 0.3
    sc = _iso_scene([[0.0, 0.0, 0.0]], s, st, mu_t, o, [[0.7], [0.1], [-3.0]])
    out = oracle.render(oracle.Params.from_scene(sc), cam, t)
    f = cam.fx / 4.0
    var2 = f * f * s * s + 0.3
    a = 1 / (1 + math.exp(-o)) * math.exp(-0.5 * (t - mu_t) ** 2 / st ** 2)
    col = np.maximum(0.0, np.array([0.7, 0.1, -3.0]) / (2 * math.sqrt(math.pi)) + 0.5)
    yy, xx = np.mgrid[0:H, 0:W]
    d2 = (xx - 15.5) ** 2 + (yy - 15.5) ** 2
    alpha = np.minimum(float(np.float32(0.99)), a * np.exp(-0.5 * d2 / var2))
    alpha = np.where(alpha >= float(np.float32(1 / 255)), alpha, 0.0)
    want = col[:, None, None] * alpha[None]
    assert np.abs(out["image"].numpy() - want).max() < 1e-12
    assert np.abs(out["T_final"].numpy() - (1 - alpha)).max() < 1e-12
    assert col[2] == 0.0                                   # the SH clamp at zero is exercised


def test_positive_power_is_skipped():
    """Eq. 2 reading: an entry whose exponent is positive is skipped. An indefinite conic
    (A > 0, C < 0), built by hand, makes the exponent -0.25 one pixel along x and +0.25 one
    pixel along y: the first pixel blends the closed-form alpha, the second keeps T = 1."""
    pre = {"mean2d": torch.tensor([[0.0, 0.0]], dtype=F64),
           "conic": torch.tensor([[0.5, 0.0, -0.5]], dtype=F64),
           "a": torch.tensor([0.5], dtype=F64),
           "rgb": torch.tensor([[1.0, 0.5, 0.25]], dtype=F64)}
    px = torch.tensor([1.0, 0.0], dtype=F64)
    py = torch.tensor([0.0, 1.0], dtype=F64)
    colour, T, last, _ = oracle.blend_tile(pre, [0], px, py)
    alpha = 0.5 * math.exp(-0.25)
    assert abs(float(T[0]) - (1.0 - alpha)) < 1e-15
    assert np.allclose(colour[0].numpy(), alpha * np.array([1.0, 0.5, 0.25]), atol=1e-15)
    assert int(last[0]) == 1
    assert float(T[1]) == 1.0 and float(colour[1].abs().max()) == 0.0 and int(last[1]) == 0


def test_degree1_colour_follows_the_view_direction():
    """Colour reading: c = max(0, sum_k Y_k(d) f_k + 0.5) with d the unit vector from the
    camera centre to the conditional mean. With only a degree-1 coefficient set, the textbook
    real SH give Y_1^0 = sqrt(3 / 4 pi) d_z and Y_1^1 = sqrt(3 / 4 pi) d_x."""
    cam = scenes.look_at_camera((0.0, 0.0, 4.0), 32, 32)
    means = np.array([[0.0, 0.0, 0.0], [0.5, 0.0, 0.0]])
    n = len(means)
    mean4 = np.concatenate([means, np.full((n, 1), 0.5)], 1)
    ls = np.tile([math.log(0.2)] * 3 + [math.log(0.3)], (n, 1))
    ident = np.tile([1.0, 0, 0, 0], (n, 1))
    sh = np.zeros((4, 3, n))
    sh[2, :, 0] = [0.3, -0.2, 0.1]           # Y_1^0 (z) on the first Gaussian
    sh[3, :, 1] = [0.4, 0.0, -0.4]           # Y_1^1 (x) on the second
    sc = _scene64(mean4, ls, ident, ident, np.zeros(n), sh, 1)
    pre = oracle.preprocess(oracle.Params.from_scene(sc), cam, 0.5)
    c1 = math.sqrt(3.0 / (4.0 * math.pi))
    d0 = np.array([0.0, 0.0, -1.0])          # camera at (0, 0, 4) looking at the origin
    d1 = (means[1] - np.array([0.0, 0.0, 4.0])) / np.linalg.norm(means[1] - [0.0, 0.0, 4.0])
    want0 = c1 * d0[2] * np.array([0.3, -0.2, 0.1]) + 0.5
    want1 = c1 * d1[0] * np.array([0.4, 0.0, -0.4]) + 0.5
    rgb = pre["rgb"].detach().numpy()
    assert np.abs(rgb[0] - want0).max() < 1e-12
    assert np.abs(rgb[1] - want1).max() < 1e-12


def test_two_gaussians_and_the_stop_rule():
    W = H = 16
    cam = scenes.look_at_camera((0.0, 0.0, 4.0), W, H)
    # two Gaussians on the optical axis, the nearer one first in the blend
    sc = _iso_scene([[0.0, 0.0, -0.5], [0.0, 0.0, 0.5]], 0.25, 1.0, 0.5, 0.0,
                    [[1.0, -0.2], [0.0, 0.4], [0.5, 1.0]])
    out = oracle.render(oracle.Params.from_scene(sc), cam, 0.5)
    yy, xx = np.mgrid[0:H, 0:W]
    d2 = (xx - 7.5) ** 2 + (yy - 7.5) ** 2
    cols = np.maximum(0.0, np.array([[1.0, -0.2], [0.0, 0.4], [0.5, 1.0]])
                      / (2 * math.sqrt(math.pi)) + 0.5)
    al = []
    for z in (4.5, 3.5):                                   # Gaussian 0 is the farther one
        f = cam.fx / z
        x = np.minimum(0.99, 0.5 * np.exp(-0.5 * d2 / (f * f * 0.0625 + 0.3)))
        al.append(np.where(x >= float(np.float32(1 / 255)), x, 0.0))
    want = cols[:, 1, None, None] * al[1] + cols[:, 0, None, None] * al[0] * (1 - al[1])
    assert np.abs(out["image"].numpy() - want).max() < 1e-12
    # three fully opaque Gaussians: alpha clamps to 0.99f. With that float32 constant,
    # T after two of them is (1 - 0.99f)^2 = 9.99998e-5, just under the float32 stop threshold
    # 1e-4f, so the second one stops the pixel: only the first is blended, n_contrib = 1.
    a0 = float(np.float32(0.99))
    assert (1 - a0) ** 2 < float(np.float32(1e-4)) < (1 - a0)
    sc = _iso_scene([[0.0, 0.0, 0.0], [0.0, 0.0, -0.1], [0.0, 0.0, -0.2]], 3.0, 1.0, 0.5, 30.0,
                    [[1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
    out = oracle.render(oracle.Params.from_scene(sc), cam, 0.5)
    c = np.array([1.0, 0.0]) / (2 * math.sqrt(math.pi)) + 0.5
    centre = out["image"][:, 7, 7].numpy()
    want = np.array([c[0] * a0, c[1] * a0, c[1] * a0])
    assert np.abs(centre - want).max() < 1e-12
    assert int(out["n_contrib"][7, 7]) == 1
    assert abs(float(out["T_final"][7, 7]) - (1 - a0)) < 1e-15
    # two less opaque Gaussians (alpha 0.9 each: T = 0.1, 0.01) are both blended
    sc = _iso_scene([[0.0, 0.0, 0.0], [0.0, 0.0, -0.1]], 3.0, 1.0, 0.5, math.log(9.0) + 0.0,
                    [[1.0, 0.0], [0.0, 1.0], [0.0, 0.0]])
    out = oracle.render(oracle.Params.from_scene(sc), cam, 0.5)
    assert int(out["n_contrib"][7, 7]) == 2


def test_zero_space_time_correlation_is_a_static_splat():
    """With q_r = -k conj(q_l) k the 4D rotation fixes the t axis, the slice keeps the spatial
    block and the render equals a static 3D splat with opacity x exp(-(t-mu_t)^2/(2 s_t^2))."""
    rng = np.random.default_rng(12)
    n, t = 40, 0.45
    mean4 = np.concatenate([rng.uniform(-1, 1, (n, 3)), rng.uniform(0, 1, (n, 1))], 1)
    ls = np.concatenate([rng.normal(-1.6, 0.3, (n, 3)), rng.normal(-1.3, 0.3, (n, 1))], 1)
    ql = rng.standard_normal((n, 4))
    ql /= np.linalg.norm(ql, axis=1, keepdims=True)
    k = np.array([0.0, 0, 0, 1])
    qr = np.stack([-brute.quat_mul(brute.quat_mul(k, q * [1, -1, -1, -1]), k) for q in ql])
    op = rng.normal(0, 1, n)
    sh = rng.normal(0, 0.5, (1, 3, n))
    sc = _scene64(mean4, ls, ql, qr, op, sh, 0)
    cam = scenes.look_at_camera((0.0, 0.0, 4.0), 44, 30)
    out = oracle.render(oracle.Params.from_scene(sc), cam, t)
    mu3, cov3, opac, rgb = [], [], [], []
    for i in range(n):
        R = brute.rotation_by_products(ql[i], qr[i])
        assert abs(R[3, 3] - 1.0) < 1e-12
        M = R[:3, :3]
        mu3.append(mean4[i, :3])
        cov3.append(M @ np.diag(np.exp(2 * ls[i, :3])) @ M.T)
        st = math.exp(ls[i, 3])
        opac.append(1 / (1 + math.exp(-op[i])) * math.exp(-(t - mean4[i, 3]) ** 2 / (2 * st * st)))
        rgb.append(np.maximum(0, sh[0, :, i] / (2 * math.sqrt(math.pi)) + 0.5))
    img, T, nc = brute.render_static(np.array(mu3), np.array(cov3), np.array(opac),
                                     np.array(rgb), cam)
    assert np.abs(out["image"].numpy() - img).max() < 1e-10
    assert np.abs(out["T_final"].numpy() - T).max() < 1e-10
    assert float(out["image"].max()) > 0.1


def test_temporal_cull_changes_lists_not_images():
    """The exact temporal cull (a = sigmoid(o) p(t) < 1/255, Sec. 3 Eq. 3) is exact: a
    renderer without it lists more Gaussians per tile, every extra one with a < 1/255, and
    composites the same image (such an entry reaches alpha >= 1/255 at no pixel)."""
    s = scenes.make_scene(1500, 31, sh_degree=1, lt_short=(-4.0, 0.5), lt_long=(-2.0, 0.5),
                          short_frac=0.7)
    cam = scenes.tiny_camera(80, 64)
    P = oracle.Params.from_scene(s)
    on = oracle.render(P, cam, 0.4)
    off = oracle.render(P, cam, 0.4, temporal_cull=False)
    a = on["pre"]["a"].detach().numpy()
    assert np.abs(on["image"].numpy() - off["image"].numpy()).max() <= 1e-12
    assert np.abs(on["T_final"].numpy() - off["T_final"].numpy()).max() <= 1e-12
    extra = 0
    for tid, ids in on["lists"].items():
        more = np.setdiff1d(off["lists"][tid], ids)
        assert set(ids.tolist()) <= set(off["lists"][tid].tolist())
        assert np.all(a[more] < oracle.ALPHA_MIN)
        extra += len(more)
    assert extra > 100
    assert np.array_equal(on["pre"]["pass_temporal"].numpy(), off["pre"]["pass_temporal"].numpy())


# ---- gradients -------------------------------------------------------------------------------

def _decisions(P, cam, t):
    out = oracle.render(P, cam, t)
    pre = out["pre"]
    return (pre["visible"].numpy().copy(), pre["rect"].numpy().copy(),
            out["n_contrib"].numpy().copy(), (pre["rgb_raw"] > 0).detach().numpy().copy())


def test_gradients_match_central_finite_differences():
    s = scenes.make_scene(14, 21, sh_degree=1, lxyz=(-2.0, 0.4), lt_long=(-1.0, 0.3))
    s = _scene64(s.mean4, s.logscale4, s.q_left, s.q_right, s.opacity_logit, s.sh, 1)
    cam = scenes.look_at_camera((0.3, 0.2, 4.0), 24, 20)
    t = 0.5
    g = np.random.default_rng(3).standard_normal((3, 20, 24))
    grads, _ = oracle.gradients(s, cam, t, g)
    base = _decisions(oracle.Params.from_scene(s), cam, t)
    names = ["mean4", "logscale4", "q_left", "q_right", "opacity_logit", "sh"]
    rng = np.random.default_rng(4)
    h = 1e-6
    checked = 0
    for name, gr in zip(names, grads):
        arr = getattr(s, name)
        for flat in rng.choice(arr.size, size=min(arr.size, 12), replace=False):
            vals = []
            same = True
            for sgn in (1, -1):
                a2 = arr.copy().reshape(-1)
                a2[flat] += sgn * h
                s2 = scenes.Scene(**{**s.arrays(), name: a2.reshape(arr.shape)},
                                  sh_degree=1)
                P2 = oracle.Params.from_scene(s2)
                img, _ = oracle.render_image(P2, cam, t)
                vals.append(float((img.numpy() * g).sum()))
                d = _decisions(P2, cam, t)
                same &= all(np.array_equal(x, y) for x, y in zip(base, d))
            if not same:
                continue
            fd = (vals[0] - vals[1]) / (2 * h)
            an = gr.reshape(-1)[flat]
            scale = max(np.abs(gr).max(), 1e-3)
            assert abs(fd - an) <= 1e-6 * scale + 1e-5 * abs(an), (name, flat, fd, an)
            checked += 1
    assert checked > 50


def test_gradients_match_finite_differences_at_the_backward_workload_size():
    """The backward workload's check: 500 Gaussians (the densest in view of the pruned
    scene's draw, degree-3 SH) at 64x64, central differences with h = 1e-6 of
    L = sum(dL * image) with dL the L1-loss gradient against a target rendered from means
    perturbed by N(0, 0.01). Components whose +-h moves a decision (visibility, rectangle,
    n_contrib, SH clamp) are skipped and counted; a sample of every parameter tensor is
    checked."""
    full = scenes.pruned_scene(20_000, 5)
    idx = np.argsort(np.abs(full.mean4[:, 0]) + np.abs(full.mean4[:, 1]))[:500]
    s = full.subset(np.sort(idx))
    s = _scene64(s.mean4, s.logscale4, s.q_left, s.q_right, s.opacity_logit, s.sh, 3)
    cam = scenes.arc_camera(3.0, 64, 64)
    t = 0.45
    rng = np.random.default_rng(55)
    m = s.mean4.copy()
    m[:, :3] += rng.normal(0, 0.01, (s.n, 3))
    target = oracle.render(oracle.Params.from_scene(scenes.Scene(**{**s.arrays(), "mean4": m},
                                                                 sh_degree=3)), cam, t)["image"]
    img0 = oracle.render(oracle.Params.from_scene(s), cam, t)["image"].numpy()
    g = np.sign(img0 - target.numpy()) / img0.size
    grads, _ = oracle.gradients(s, cam, t, g)
    base = _decisions(oracle.Params.from_scene(s), cam, t)
    names = ["mean4", "logscale4", "q_left", "q_right", "opacity_logit", "sh"]
    h = 1e-6
    pick = np.random.default_rng(6)
    checked = skipped = 0
    for name, gr in zip(names, grads):
        arr = getattr(s, name)
        # sample among components with a non-zero gradient (Gaussians that reach the image)
        nz = np.flatnonzero(np.abs(gr.reshape(-1)) > 0)
        for flat in pick.choice(nz, size=min(len(nz), 24 if name == "sh" else 12),
                                replace=False):
            vals = []
            same = True
            for sgn in (1, -1):
                a2 = arr.copy().reshape(-1)
                a2[flat] += sgn * h
                s2 = scenes.Scene(**{**s.arrays(), name: a2.reshape(arr.shape)}, sh_degree=3)
                P2 = oracle.Params.from_scene(s2)
                img, _ = oracle.render_image(P2, cam, t)
                vals.append(float((img.numpy() * g).sum()))
                same &= all(np.array_equal(x, y) for x, y in zip(base, _decisions(P2, cam, t)))
            if not same:
                skipped += 1
                continue
            fd = (vals[0] - vals[1]) / (2 * h)
            an = gr.reshape(-1)[flat]
            scale = np.abs(gr).max()
            assert abs(fd - an) <= 1e-6 * abs(an) + 1e-7 * scale, (name, flat, fd, an)
            checked += 1
    assert checked >= 70 and skipped <= 10, (checked, skipped)


# ---- Sec. 4.2.1: spatial-temporal variation score ------------------------------------------

def test_blend_weights_sum_to_one_minus_final_transmittance():
    s = scenes.tiny_scene()
    cam = scenes.tiny_camera(64, 64)
    out = oracle.render(oracle.Params.from_scene(s), cam, 0.5, weights=True)
    total = float(out["w_sum"].sum())
    assert math.isclose(total, float((1 - out["T_final"]).sum()), rel_tol=1e-12)


def test_variation_factor_range_and_fixed_points():
    mean4, ls, ql, qr = _rand_params(64, 7)
    cov = oracle.covariance_4d(torch.tensor(ls), torch.tensor(ql), torch.tensor(qr))
    m4 = torch.tensor(mean4)
    for t in np.linspace(-0.5, 1.5, 9):
        f = oracle.variation_factor(m4, cov, float(t)).numpy()
        assert np.all(f >= 1.0) and np.all(f <= 2.0)      # (1, 2]; tanh rounds to 1
    # |t - mu_t| = sqrt(Sigma_t): p^(2) = 0, factor exactly 2 (up to rounding)
    stt = cov[:, 3, 3]
    f = oracle.variation_factor(m4, cov, 0.0)
    tt = (m4[:, 3] + torch.sqrt(stt))
    for i in range(8):
        fi = oracle.variation_factor(m4[i:i + 1], cov[i:i + 1], float(tt[i]))
        assert abs(float(fi) - 2.0) < 1e-9
    # far from the mean the factor tends to 2 as well (p^(2) -> 0), and at t = mu_t it is
    # 1 / (0.5 tanh(1/Sigma_t) + 0.5)
    for i in range(8):
        fi = float(oracle.variation_factor(m4[i:i + 1], cov[i:i + 1], float(m4[i, 3])))
        want = 1 / (0.5 * math.tanh(1 / float(stt[i])) + 0.5)
        assert math.isclose(fi, want, rel_tol=1e-12)


def test_volume_gamma_range_and_percentile():
    rng = np.random.default_rng(8)
    ls = torch.tensor(rng.normal(-2, 0.7, (1000, 4)))
    g = oracle.volume_gamma(ls).numpy()
    assert np.all(g >= 0) and np.all(g <= 1)
    V = np.exp(ls.numpy().sum(1))
    # exactly the Gaussians at or above the nearest-rank 90th percentile get gamma = 1
    assert int((g == 1.0).sum()) == 1000 - 900 + 1
    thr = np.sort(V)[899]
    i = np.argmin(V)
    assert math.isclose(g[i], (V[i] / thr) ** 0.1, rel_tol=1e-12)


def test_scores_permutation_invariant_and_readings_agree_at_one_t():
    s = scenes.make_scene(80, 31, sh_degree=0, lxyz=(-2.2, 0.4), lt_long=(-1.2, 0.3))
    cams = [scenes.look_at_camera((0.0, 0.0, 4.0), 32, 32),
            scenes.look_at_camera((1.0, 0.0, 3.9), 32, 32)]
    S1 = oracle.variation_scores(s, cams, [0.5], "R1")
    S2 = oracle.variation_scores(s, cams, [0.5], "R2")
    assert np.allclose(S1, S2, rtol=1e-12, atol=0)
    perm = np.random.default_rng(0).permutation(s.n)
    Sp = oracle.variation_scores(s.subset(perm), cams, [0.5], "R1")
    assert np.allclose(Sp, S1[perm], rtol=1e-10, atol=1e-14)
    Sm = oracle.variation_scores(s, cams, [0.2, 0.5, 0.9], "R1")
    assert np.all(Sm >= S1 - 1e-15) and Sm.max() > 0


def test_first_derivative_by_finite_differences_and_its_factor_range():
    """p^(1)(t) of score variant (d) (Table 4) is the time derivative of Eq. 3's p(t): central
    differences of the oracle's own marginal; the factor with p^(1) lies in (1, 2] and is
    exactly 2 at t = mu_t, where p^(1) = 0."""
    mean4, ls, ql, qr = _rand_params(16, 15)
    cov = oracle.covariance_4d(torch.tensor(ls), torch.tensor(ql), torch.tensor(qr))
    m4 = torch.tensor(mean4)
    t, h = 0.37, 1e-6

    def p(tt):
        return oracle.condition_on_time(m4, cov, tt)[3].numpy()
    fd1 = (p(t + h) - p(t - h)) / (2 * h)
    p1 = oracle.temporal_first_derivative(m4, cov, t).numpy()
    assert np.allclose(p1, fd1, rtol=1e-6, atol=1e-8)
    for tt in np.linspace(-0.5, 1.5, 9):
        f1 = oracle.variation_factor(m4, cov, float(tt), derivative=1).numpy()
        assert np.all(f1 >= 1.0) and np.all(f1 <= 2.0)
    for i in range(6):
        f1 = oracle.variation_factor(m4[i:i + 1], cov[i:i + 1], float(m4[i, 3]), derivative=1)
        assert float(f1) == 2.0


def _variant_scene():
    s = scenes.make_scene(120, 41, sh_degree=0, lxyz=(-2.2, 0.4), lt_long=(-1.2, 0.3))
    # identity quaternions for every fourth Gaussian: its 4D covariance is diag(s^2), so
    # Sigma_t = exp(2 l_t)
    ql, qr = s.q_left.copy(), s.q_right.copy()
    ql[::4] = (1.0, 0.0, 0.0, 0.0)
    qr[::4] = (1.0, 0.0, 0.0, 0.0)
    return scenes.Scene(**{**s.arrays(), "q_left": ql, "q_right": qr}, sh_degree=0)


def test_score_variants_against_the_spatial_score_and_each_other():
    """The score ablation's variants (Table 4; supplement "Variant Settings"), at one (t, view):
    every rendered variant is the spatial score S^S (variant b, the blend weights of Eq. 4)
    times its own per-Gaussian factor: f gamma (ours), f1 gamma (d), Sigma_t gamma (e), with
    Sigma_t = exp(2 l_t) where the rotation is the identity; the temporal-only score (c)
    needs no render, so it is the same for any views and adds up over disjoint time sets."""
    s = _variant_scene()
    cams = [scenes.look_at_camera((0.3, 0.1, 4.0), 40, 32)]
    t = 0.45
    P = oracle.Params.from_scene(s)
    w = oracle.render(P, cams[0], t, weights=True)["w_sum"].numpy()
    cov = oracle.covariance_4d(P.logscale4, P.q_left, P.q_right)
    gamma = oracle.volume_gamma(P.logscale4).numpy()
    f2 = oracle.variation_factor(P.mean4, cov, t).numpy()
    f1 = oracle.variation_factor(P.mean4, cov, t, derivative=1).numpy()
    sc = {v: oracle.variation_scores(s, cams, [t], variant=v) for v in oracle.SCORE_VARIANTS}
    assert np.array_equal(sc["spatial"], w) and int((w > 0).sum()) > 20
    assert np.allclose(sc["full"], w * f2 * gamma, rtol=1e-12, atol=0)
    assert np.allclose(sc["first_derivative"], w * f1 * gamma, rtol=1e-12, atol=0)
    idq = np.zeros(s.n, bool)
    idq[::4] = True
    sig_t = np.exp(2.0 * s.logscale4[:, 3].astype(np.float64))
    assert np.allclose(sc["sigma_t"][idq], (w * sig_t * gamma)[idq], rtol=1e-12, atol=0)
    assert np.allclose(sc["temporal"], f2 * gamma, rtol=1e-12, atol=0)
    # temporal only: the same with other views or none, additive over time sets
    other = [scenes.look_at_camera((-1.0, 0.0, 3.8), 24, 24)] * 3
    assert np.array_equal(oracle.variation_scores(s, other, [t], variant="temporal"),
                          sc["temporal"])
    assert np.array_equal(oracle.variation_scores(s, [], [t], variant="temporal"),
                          sc["temporal"])
    a = oracle.variation_scores(s, cams, [0.1, 0.9], variant="temporal")
    b = oracle.variation_scores(s, cams, [0.1, 0.9, t], variant="temporal")
    assert np.allclose(b, a + sc["temporal"], rtol=1e-12, atol=0)
    with pytest.raises(ValueError):
        oracle.variation_scores(s, cams, [t], variant="other")


def test_keep_set_ties_broken_by_id():
    keep = oracle.keep_set([3.0, 1.0, 1.0, 2.0, 0.0], 0.6)
    assert keep.tolist() == [True, False, False, True, False]
    keep = oracle.keep_set([1.0, 1.0, 1.0, 1.0], 0.5)
    assert keep.tolist() == [False, False, True, True]
