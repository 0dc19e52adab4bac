"""Post-pruning fine-tuning (Sec. 4.2.1-4.2.2): pruning keeps the right Gaussians (CPU), and
the whole pipeline - score, prune, key-frame masks, fine-tune through the filter - lowers the
loss and raises held-out PSNR on a self-distillation target (GPU)."""
import numpy as np
import pytest
import torch

from paper_2503_16422_gb300 import scenes


def test_prune_keeps_the_marked_gaussians_in_id_order():
    from paper_2503_16422_gb300 import fdgs, finetune
    s = scenes.make_scene(50, 3, sh_degree=1)
    p = fdgs.SceneTensors.from_host(s, device="cpu")
    keep = torch.zeros(50, dtype=torch.uint8)
    keep[[1, 4, 5, 30, 49]] = 1
    q = finetune.prune(p, keep)
    idx = [1, 4, 5, 30, 49]
    assert torch.equal(q.mean4, p.mean4[idx]) and torch.equal(q.q_right, p.q_right[idx])
    assert torch.equal(q.opacity_logit, p.opacity_logit[idx])
    assert q.sh.shape == (4, 3, 5) and torch.equal(q.sh, p.sh[:, :, idx])
    assert q.sh.is_contiguous() and q.sh_degree == 1


def test_psnr():
    from paper_2503_16422_gb300 import finetune
    a = torch.zeros(3, 4, 4)
    assert finetune.psnr(a, a) == float("inf")
    assert abs(finetune.psnr(a, a + 0.1) - 20.0) < 1e-6


@pytest.mark.gpu
def test_score_prune_mask_finetune_pipeline():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2503_16422_gb300 import build, fdgs, finetune
    build.build()
    teacher = scenes.make_scene(8000, 71, sh_degree=1, lxyz=(-2.6, 0.4), lt_long=(-1.2, 0.4))
    tsc = fdgs.Scene.from_host(teacher)
    cams = [scenes.arc_camera(th, 96, 72) for th in (-10.0, -4.0, 4.0, 10.0)]
    times = [0.1, 0.3, 0.5, 0.7, 0.9]
    key_times = np.linspace(0.0, 1.0, 6)
    views = [(c, t, tsc.render(c, t, use_mask=False)) for t in times for c in cams]
    held = [(scenes.arc_camera(0.0, 96, 72), t) for t in (0.2, 0.6)]
    held = [(c, t, tsc.render(c, t, use_mask=False)) for c, t in held]
    # score over the training views, prune 80% (the paper's ratio)
    score = tsc.variation_score(cams, times)
    keep = tsc.select_keep(score, 0.8)
    student = fdgs.Scene(finetune.prune(tsc.params, keep))
    assert student.n == int(keep.sum())
    student.set_active_mask(student.build_keyframe_masks(cams, key_times), key_times)

    def held_psnr():
        with torch.no_grad():
            return np.mean([finetune.psnr(student.render(c, t, use_mask=True), ref)
                            for c, t, ref in held])

    before = held_psnr()
    losses = finetune.FineTuner(student).run(views, 300).cpu().numpy()
    after = held_psnr()
    print(f"kept {student.n}/{tsc.n}; L1 {losses[:20].mean():.5f} -> {losses[-20:].mean():.5f};"
          f" held-out PSNR {before:.2f} -> {after:.2f} dB")
    assert np.all(np.isfinite(losses))
    assert losses[-20:].mean() < 0.8 * losses[:20].mean()
    assert after > before + 2.0
    student.close()
    tsc.close()
