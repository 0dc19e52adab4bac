"""Vector-quantised SH (Ours-PP): the encoder's codes are nearest centroids and decoding is
the table look-up (CPU); on the GPU a codebook scene renders exactly as the same scene with
the decoded full coefficients, in single and batched renders."""
import numpy as np
import pytest
import torch

from paper_2503_16422_gb300 import scenes


def test_codes_are_nearest_and_decode_is_lookup():
    from paper_2503_16422_gb300 import vq
    s = scenes.make_scene(600, 5, sh_degree=3)
    sh = torch.as_tensor(s.sh, dtype=torch.float32)
    cb, codes = vq.quantize_sh(sh, n_code=40, iters=6, seed=1)
    assert cb.shape == (40, 15, 3) and codes.shape == (600,) and codes.dtype == torch.int16
    x = sh[1:].permute(2, 0, 1).reshape(600, 45).double().numpy()
    c = cb.reshape(40, 45).double().numpy()
    d = ((x[:, None, :] - c[None, :, :]) ** 2).sum(-1)
    got = d[np.arange(600), codes.numpy().astype(np.int64)]
    assert np.all(got <= d.min(1) * (1 + 1e-5) + 1e-9)
    full = vq.decode_sh(sh, cb, codes)
    assert full.shape == sh.shape and torch.equal(full[0], sh[0])
    assert torch.equal(full[1:, :, 7], cb[int(codes[7])].reshape(15, 3))


def test_one_code_per_gaussian_reproduces_the_coefficients():
    from paper_2503_16422_gb300 import vq
    s = scenes.make_scene(50, 6, sh_degree=2)
    sh = torch.as_tensor(s.sh, dtype=torch.float32)
    cb, codes = vq.quantize_sh(sh, n_code=50, iters=3)
    assert torch.equal(vq.decode_sh(sh, cb, codes), sh)


@pytest.mark.gpu
def test_codebook_scene_renders_as_decoded_scene():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2503_16422_gb300 import build, fdgs, vq
    build.build()
    s = scenes.pruned_scene(30_000, 8)
    p = fdgs.SceneTensors.from_host(s)
    cb, codes = vq.quantize_sh(p.sh, n_code=512, iters=4)
    dec = vq.decode_sh(p.sh, cb, codes)
    q = fdgs.SceneTensors(p.mean4, p.logscale4, p.q_left, p.q_right, p.opacity_logit, dec,
                          p.sh_degree)
    sc_vq = fdgs.Scene(p)                      # full sh array; only plane 0 is read
    sc_vq.set_sh_codebook(cb, codes)
    sc_dec = fdgs.Scene(q)
    cams = [scenes.arc_camera(th, 320, 240) for th in (-6.0, 2.0, 9.0)]
    ts = [0.2, 0.5, 0.8]
    for c, t in zip(cams, ts):
        assert torch.equal(sc_vq.render(c, t, use_mask=False), sc_dec.render(c, t, use_mask=False))
    a = sc_vq.render_batch(cams, ts, use_mask=False)
    b = sc_dec.render_batch(cams, ts, use_mask=False)
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    # the backward needs full coefficients
    img, fr = sc_vq.render(cams[0], ts[0], use_mask=False, keep_frame=True)
    with pytest.raises(fdgs.FdgsError):
        sc_vq.render_backward(fr, torch.ones_like(img))
    fr.release()
    # clearing the codebook restores the full-coefficient render
    sc_vq.set_sh_codebook(None, None)
    sc_full = fdgs.Scene(fdgs.SceneTensors.from_host(s))
    assert torch.equal(sc_vq.render(cams[1], ts[1], use_mask=False),
                       sc_full.render(cams[1], ts[1], use_mask=False))
    for x in (sc_vq, sc_dec, sc_full):
        x.close()
