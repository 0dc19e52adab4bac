#!/usr/bin/env python
"""Benchmark: masked, batched 4D Gaussian rendering at 1352x1014 on one GB300.

Headline (one step = one batch): the pruned 4DGS-1K-like scene (200,000 Gaussians, degree-3
SH, temporal log-scales N(-1, 0.5)) with the key-frame temporal filter (masks every 6 frames,
|t_k - mu_t| < 3 s_t), rendered as a batch of 64 requests at 1352x1014: frames k of the
300-frame sequence (t_k = k/299, camera on a 20-degree arc) through fdgs_render_batch (one
device-driven pass replayed from a CUDA graph, one persistent longest-first blend). value =
frames per second. Inputs are synthetic (seeded), resident in HBM; L2 is flushed (256 MiB
write) before every timed step.

Beside it: the single-request masked and unmasked renders (fdgs_render), the unpruned 3M
scene, and the mixed-resolution serving batch (64 requests, resolutions from {512^2, 800^2,
1014x1352, 1352x1014}) with p50/p99 request latency against 64 sequential renders. Per-kernel
times come from CUDA events on the render stream in a profiled pass over the same frames.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--batch B] [--impl ours|reference]

With --gpus N > 1 (torchrun) every rank renders its own batches of a replica of the scene
(no collective: frames are independent), timing is the max over ranks and the value is the
total frames of all ranks per second.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FPS at 1352x1014 (masked 4DGS render, 1 GB300)"
FLUSH_BYTES = 256 << 20
E2E_COPY_STREAMS = 4   # device->host image copies run on this many streams at once
# FP32 FLOP per (Gaussian, pixel) evaluation (FMA = 2): offsets 2, exponent 7, log-opacity
# add 1, alpha clamp 1, transmittance 2, weight 1, colour 6 (plus one MUFU exp2)
EVAL_FLOP = 20
TEST_FLOP = 36        # FP32 FLOP per footprint culling test (4 edges x 9)
W_FULL, H_FULL = 1352, 1014


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the comparison workloads")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default batch launch shape (for profiling runs)")
    ap.add_argument("--only", choices=["backward", "score", "masks", "unpruned"],
                    help="run one side workload alone and print its line (for profiling runs)")
    return ap.parse_args()


def frame_list(n, offset=0):
    """Frame indices of n consecutive requests: a stride-7 walk over the 300 frames."""
    return [((offset + i) * 7) % 300 for i in range(n)]


def rank_requests(rank, steps, batch):
    """Frame indices of every timed step of one replica: each rank walks the frames from its
    own offset, so the ranks render independent request streams (weak scaling)."""
    return [frame_list(batch, rank * 1000 + s * batch) for s in range(steps)]


def job_fps(local_ms, frames_per_rank, world, reduce_max=None):
    """Whole-job throughput: the frames of all ranks over the slowest rank's time.
    reduce_max maps this rank's time to the maximum over ranks (None on one GPU)."""
    t_ms = reduce_max(local_ms) if reduce_max is not None else local_ms
    return world * frames_per_rank / (t_ms / 1e3), t_ms


def pruned_masked():
    from paper_2503_16422_gb300 import scenes
    scene = scenes.pruned_scene()
    kt = scenes.keyframe_times()
    return scene, kt, scenes.keyframe_masks(scene, kt)


def workload_config(scene, kt, batch):
    return {"workload": f"pruned scene, {scene.n} Gaussians, degree-{scene.sh_degree} SH, "
                        f"masked (key-frame masks every 6 of 300 frames, {len(kt)} rows), "
                        f"batches of {batch} frames at {W_FULL}x{H_FULL} on a 20-degree arc",
            "n_gaussians": scene.n, "width": W_FULL, "height": H_FULL, "tile": 16,
            "batch": batch, "masked": True,
            "l2": "flushed before every timed step (256 MiB write)"}


# ---- peaks -----------------------------------------------------------------------------

def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return dict(hbm=float(d["hbm_gbs"]), sm_mhz=float(d.get("sm_max_mhz", 2070.0)),
                    src="measured")
    return dict(hbm=6800.0, sm_mhz=2070.0, src="fallback")


def fp32_peak_tflops(sm_mhz, sms=152):
    # 128 FP32 lanes per SM, one FMA (2 FLOP) per lane per clock
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


# ---- clocks sampler --------------------------------------------------------------------

class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---- CPU oracle baseline ---------------------------------------------------------------

def cpu_oracle_frame(scene, kt, masks, frame=150, budget_s=12.0, min_tiles=8):
    """FP64 oracle on a bounded sample of one masked frame: the whole per-Gaussian stage,
    then the blend of randomly chosen tiles until ~budget_s of CPU work; the tile time is
    scaled to all 5,440 tiles. Returns seconds per frame, a description and the threads."""
    import torch

    import oracle
    from paper_2503_16422_gb300 import scenes
    cam = scenes.arc_camera(scenes.frame_theta(frame))
    t = float(scenes.frame_times()[frame])
    active = oracle.active_from_masks(masks, kt, t, scene.n)
    P = oracle.Params.from_scene(scene)
    t0 = time.perf_counter()
    pre = oracle.preprocess(P, cam, t, active)
    t1 = time.perf_counter()
    gx, gy = pre["grid"]
    order = np.random.default_rng(frame).permutation(gx * gy).tolist()
    done = 0
    while done < len(order) and (done < min_tiles or time.perf_counter() - t1 < budget_s):
        chunk = order[done:done + 8]
        oracle.render(P, cam, t, active, tiles=chunk, pre=pre)
        done += len(chunk)
    t2 = time.perf_counter()
    frame_s = (t1 - t0) + (t2 - t1) * (gx * gy) / done
    desc = (f"1 frame (k={frame}): per-Gaussian stage of all {scene.n} Gaussians + blend of "
            f"{done}/{gx * gy} random tiles scaled to the frame ({t2 - t0:.1f} s of CPU work)")
    return frame_s, desc, torch.get_num_threads()


# ---- helpers for our implementation ------------------------------------------------------

def stage_bytes(stats, n, deg, masked):
    """Algorithmic DRAM bytes of each HBM-bound stage of one single-request frame."""
    na, nv, K, kb = stats["n_active"], stats["n_visible"], stats["n_keys"], stats["key_bytes"]
    sh = (deg + 1) ** 2 * 3 * 4
    tiles = stats["tiles_x"] * stats["tiles_y"]
    passes = math.ceil(math.ceil(math.log2(max(tiles, 2))) / 8)
    emit = nv * 24 + K * kb if stats["list_builder"] == 1 else K * 4
    return {
        "preprocess": (2 * math.ceil(n / 32) * 4 if masked else 0) + na * 68 + nv * (sh + 48 + 8),
        "depth_sort": nv * 8 + 4 * nv * 16,
        "gather_scan": nv * (8 + 48 + 64 + 4 + 16),
        "tile_scan": (stats["tiles_x"] + 1) * (stats["tiles_y"] + 1) * 4 * 3 + tiles * 8,
        "emit": emit,
        "tile_sort": passes * K * kb * 2 if stats["list_builder"] == 1 else 0,
    }


def _flush(buf):
    buf.fill_(1.0)


def profile_single(sc, cams, times, frames, masked, out, flush, scene):
    """Per-stage CUDA-event times, frame counts and blend work counts of single renders."""
    from paper_2503_16422_gb300 import fdgs
    sc.profile(1)
    acc = {s: 0.0 for s in fdgs.PROFILE_STAGES}
    stats = []
    for k in frames:
        _flush(flush)
        _, fr = sc.render(cams[k], float(times[k]), use_mask=masked, out=out, keep_frame=True)
        ms = sc.profile_read()[0]
        for s_ in acc:
            acc[s_] += ms[s_] / len(frames)
        stats.append(fr.stats())
        fr.release()
    sc.profile(2)
    ev = te = ep = 0
    for k in frames:
        sc.render(cams[k], float(times[k]), use_mask=masked, out=out)
        e, t, p = sc.blend_counts()
        ev += e / len(frames)
        te += t / len(frames)
        ep += p / len(frames)
    sc.profile(0)
    counts = {f: float(np.mean([st[f] for st in stats])) for f in ("n_active", "n_visible",
                                                                  "n_keys")}
    counts["blend_evals"] = ev
    counts["blend_tests"] = te
    counts["blend_evals_alpha_pass"] = ep
    sb = [stage_bytes(st, scene.n, scene.sh_degree, masked) for st in stats]
    bytes_mean = {s_: float(np.mean([b[s_] for b in sb])) for s_ in sb[0]}
    return acc, counts, bytes_mean


def roofline(stage_ms, counts, bytes_mean):
    pk = peaks()
    dom = max((s_ for s_ in stage_ms if s_ != "host_sync"), key=stage_ms.get)
    if dom == "blend":
        flop = counts["blend_evals_alpha_pass"] * EVAL_FLOP
        ach = flop / (stage_ms["blend"] / 1e3) / 1e12
        peak = fp32_peak_tflops(pk["sm_mhz"])
        executed = counts["blend_evals"] * EVAL_FLOP + counts["blend_tests"] * TEST_FLOP
        return {"bound": "alu", "kernel": "k_blend", "achieved": ach, "peak": peak,
                "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
                "peak_src": f"derived: 152 SMs x 128 FP32 lanes x 2 FLOP x {pk['sm_mhz']:.0f} MHz",
                "work": "(Gaussian, pixel) evaluations reaching alpha >= 1/255 at a pixel still "
                        "compositing x 20 FLOP",
                "executed_tflops": executed / (stage_ms["blend"] / 1e3) / 1e12}
    ach = bytes_mean[dom] / (stage_ms[dom] / 1e3) / 1e9
    return {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": pk["hbm"], "unit": "GB/s",
            "frac": ach / pk["hbm"], "traffic": None, "peak_src": pk["src"] + " copy GB/s"}


def timed_batches(sc, cams_list, ts_list, outs_list, masked, flush, stream, stages=None):
    import torch
    ms = []
    lat = []
    for cams, ts, outs in zip(cams_list, ts_list, outs_list):
        _flush(flush)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sc.render_batch(cams, ts, use_mask=masked, outs=outs)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        info = sc.batch_info(len(cams))
        lat += info["latency_ms"]
        if stages is not None:
            stages.append(info["stage_ms"])
    return ms, lat


def batch_counts(sc, cams_list, ts_list, outs):
    """Blend evaluations and culling tests of the given batches (counting profile: eager
    runs with the counting blend variant; untimed)."""
    sc.profile(2)
    ev = te = ep = 0
    for cams, ts in zip(cams_list, ts_list):
        sc.render_batch(cams, ts, outs=outs)
        e, t, p = sc.blend_counts()
        ev += e
        te += t
        ep += p
    sc.profile(0)
    return ev, te, ep


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2503_16422_gb300 import build, fdgs, scenes
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build.build()
    scene, kt, masks = pruned_masked()
    sc = fdgs.Scene.from_host(scene)
    sc.set_active_mask(torch.as_tensor(masks).cuda(), kt)
    times = scenes.frame_times()
    cams = {k: scenes.arc_camera(scenes.frame_theta(k)) for k in range(300)}
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    B = args.batch
    outs = [torch.empty((3, H_FULL, W_FULL), dtype=torch.float32, device="cuda")
            for _ in range(B)]

    def batch_args(step, base):
        fr = frame_list(B, base + step * B)
        return [cams[k] for k in fr], [float(times[k]) for k in fr]

    # autotune the batch launch shape once (untimed), then warm up (graph replays)
    c0, t0 = batch_args(0, 5000 + rank)
    if args.no_autotune:
        sc.render_batch(c0, t0, outs=outs)
    else:
        sc.batch_autotune(c0, t0, outs=outs)
    shape = sc.batch_info(B)
    for w in range(args.warmup):
        c_, t_ = batch_args(w, 6000 + rank)
        sc.render_batch(c_, t_, outs=outs)
    torch.cuda.synchronize()
    steps = [([cams[k] for k in fr], [float(times[k]) for k in fr])
             for fr in rank_requests(rank, args.steps, B)]
    clocks = Clocks(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    step_stages = []
    step_ms, lat = timed_batches(sc, [a for a, _ in steps], [b for _, b in steps],
                                 [outs] * len(steps), True, flush, stream, step_stages)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    def max_over_ranks(ms):
        tt = torch.tensor([ms], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        return float(tt.item())

    frames_done = B * len(steps)
    value, total_ms = job_fps(sum(step_ms), frames_done, world,
                              max_over_ranks if world > 1 else None)
    res = dict(clocks=clk, batch_shape=shape, lat=lat)

    # end to end through the public API: per step the cameras and times go host->device (the
    # request descriptors) and all B rendered images come back to pinned host memory. As a
    # serving loop would, the device->host copy of step i runs on a copy stream while step
    # i+1 renders (two device and two pinned host image sets); the timed region ends when
    # the last step's images are on the host.
    # two contiguous image sets on the device and in pinned host memory: one copy call per
    # copy stream moves a contiguous run of images
    dev2 = torch.empty((2, B, 3, H_FULL, W_FULL), dtype=torch.float32, device="cuda")
    host2 = torch.empty((2, B, 3, H_FULL, W_FULL), dtype=torch.float32, pin_memory=True)
    outs2 = [list(dev2[0]), list(dev2[1])]
    per = (B + E2E_COPY_STREAMS - 1) // E2E_COPY_STREAMS
    # the copies are spread over several streams so that several copy engines run at once
    copy_streams = [torch.cuda.Stream() for _ in range(E2E_COPY_STREAMS)]
    copied = [None, None]
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    te = time.perf_counter()
    for i, (c_, t_) in enumerate(steps):
        j = i % 2
        if copied[j] is not None:
            for ev in copied[j]:
                ev.synchronize()              # the copy out of this image set has finished
        sc.render_batch(c_, t_, outs=outs2[j])  # returns with the batch rendered
        copied[j] = []
        for k, cs in enumerate(copy_streams):
            with torch.cuda.stream(cs):
                lo, hi = k * per, min(B, (k + 1) * per)
                if lo < hi:
                    host2[j, lo:hi].copy_(dev2[j, lo:hi], non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(cs)
                copied[j].append(ev)
    for cs in copy_streams:
        cs.synchronize()
    e2e_fps, _ = job_fps((time.perf_counter() - te) * 1e3, frames_done, world,
                         max_over_ranks if world > 1 else None)
    res["e2e"] = dict(value=e2e_fps, unit="FPS",
                      h2d_bytes_per_step=B * (16 * 4 + 8 * 4 + 4),
                      d2h_bytes_per_step=B * 3 * H_FULL * W_FULL * 4,
                      overlap="device->host copy of step i (on %d streams) with the render "
                              "of step i+1" % E2E_COPY_STREAMS)

    if rank == 0:
        # the same batches without the L2 flush between steps, beside the flushed headline
        # (the pruned scene's attributes fit in L2); a side figure, measured after the timed
        # region, that must not cost the headline line
        try:
            no_flush = torch.empty(0, dtype=torch.float32, device="cuda")
            warm_ms, _ = timed_batches(sc, [a for a, _ in steps], [b for _, b in steps],
                                       [outs] * len(steps), True, no_flush, stream)
            res["warm_l2"] = dict(fps=frames_done / (sum(warm_ms) / 1e3),
                                  ms_per_step=sum(warm_ms) / len(warm_ms),
                                  l2="not flushed between steps")
        except Exception as e:  # noqa: BLE001
            res["warm_l2"] = {"error": repr(e)}
        # batch stages: CUDA events recorded inside the replayed graph, every timed step
        bst = {k: float(np.mean([s_[k] for s_ in step_stages])) for k in step_stages[0]}
        ev, te, ep = batch_counts(sc, [a for a, _ in steps], [b for _, b in steps], outs)
        blend_s = sum(s_["blend"] for s_ in step_stages) / 1e3
        pk = peaks()
        ach = ep * EVAL_FLOP / blend_s / 1e12
        peak = fp32_peak_tflops(pk["sm_mhz"])
        res["roofline"] = {
            "bound": "alu", "kernel": "k_blend_persist", "achieved": ach, "peak": peak,
            "unit": "TFLOP/s", "frac": ach / peak,
            "traffic": BLEND_PERSIST_DRAM_BYTES_PER_FRAME * B,
            "traffic_src": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one 8-frame "
                           "launch (profiles/k_blend_persist_batched_1352x1014.md), per frame "
                           f"x {B} frames per launch",
            "peak_src": f"derived: 152 SMs x 128 FP32 lanes x 2 FLOP x {pk['sm_mhz']:.0f} MHz",
            "work": "(Gaussian, pixel) evaluations reaching alpha >= 1/255 at a pixel still "
                    "compositing (the evaluations every blend order makes) x 20 FLOP, counted "
                    "on the same batches; time = in-graph %globaltimer stage stamps, timed steps",
            "executed_tflops": (ev * EVAL_FLOP + te * TEST_FLOP) / blend_s / 1e12,
            "blend_ms_per_batch": blend_s * 1e3 / len(steps),
            "evals_per_frame": ev / frames_done, "tests_per_frame": te / frames_done,
            "alpha_pass_evals_per_frame": ep / frames_done,
            "issue_active": BLEND_PERSIST_ISSUE_ACTIVE,
            "issue_src": "ncu smsp__issue_active of k_blend_persist<8, 4> on an 8-frame batch "
                         "(profiles/k_blend_persist_batched_1352x1014.md): the kernel is "
                         "bound by instruction issue, not by the FP32 pipes"}
        res["batch_stages_ms"] = bst
        # per-kernel profile on single renders of the same frames
        out1 = outs[0]
        fr_prof = frame_list(24, 11)
        stage_ms, counts, bytes_mean = profile_single(sc, cams, times, fr_prof, True, out1,
                                                      flush, scene)
        res.update(stage_ms=stage_ms, counts=counts,
                   single_roofline=roofline(stage_ms, counts, bytes_mean),
                   stage_gbs={s_: bytes_mean[s_] / (stage_ms[s_] / 1e3) / 1e9
                              for s_ in bytes_mean if stage_ms[s_] > 1e-4},
                   stage_rates={
                       "depth_sort_keys_per_s": counts["n_visible"] / (stage_ms["depth_sort"] / 1e3),
                       "tile_list_keys_per_s": counts["n_keys"] / (stage_ms["emit"] / 1e3),
                       "blend_evals_per_s": counts["blend_evals"] / (stage_ms["blend"] / 1e3)})
        # the batch's stages in the units of their rooflines: the preprocess in GB/s (the
        # per-request algorithmic bytes of the same frames, times the requests), the depth
        # sort (with its segment scan and compaction) and the list build in keys/s, the
        # blend in Gaussian-pixel evaluations/s
        bc = sc.batch_counts()
        res["batch_rates"] = {
            "preprocess_gbs": B * bytes_mean["preprocess"] / (bst["preprocess"] / 1e3) / 1e9,
            "depth_sort_keys_per_s": bc["n_visible"] / (bst["depth_sort"] / 1e3),
            "tile_list_keys_per_s": bc["n_keys"] / (bst["lists"] / 1e3),
            "blend_evals_per_s": ev / len(steps) / (bst["blend"] / 1e3),
            "n_visible_per_batch": bc["n_visible"], "n_keys_per_batch": bc["n_keys"]}
        if not args.no_extra:
            res["comparisons"] = comparisons(sc, cams, times, flush, stream)
    sc.close()
    return value, total_ms / len(steps), res, scene, kt, masks, world, rank


def comparisons(sc, cams, times, flush, stream):
    import torch

    from paper_2503_16422_gb300 import fdgs, scenes
    out = torch.empty((3, H_FULL, W_FULL), dtype=torch.float32, device="cuda")
    res = {}
    fr = frame_list(24, 3)

    def single(scene_obj, masked, frames, tight=False, flush_buf=flush):
        # warm-up over every timed frame, so no workspace grows inside the timed renders
        for k in frames:
            scene_obj.render(cams[k], float(times[k]), use_mask=masked, out=out, tight=tight)
        ms = []
        for k in frames:
            _flush(flush_buf)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            scene_obj.render(cams[k], float(times[k]), use_mask=masked, out=out, tight=tight)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return dict(fps=len(frames) / (sum(ms) / 1e3), ms_per_frame=sum(ms) / len(frames))

    res["single_masked"] = single(sc, True, fr)
    res["single_unmasked"] = single(sc, False, fr)
    # the same frames with the alpha-tight tile sets (same images, shorter lists)
    res["single_masked_tight"] = single(sc, True, fr, tight=True)
    res["single_unmasked_tight"] = single(sc, False, fr, tight=True)
    # the masked single renders without the L2 flush before each frame (side figure)
    try:
        res["single_masked_warm_l2"] = single(
            sc, True, fr, flush_buf=torch.empty(0, dtype=torch.float32, device="cuda"))
    except Exception as e:  # noqa: BLE001
        res["single_masked_warm_l2"] = {"error": repr(e)}
    # serving batch: 64 requests of mixed resolutions vs 64 sequential renders
    reqs, rts = scenes.random_requests(64, 4)
    outs = [torch.empty((3, c.height, c.width), dtype=torch.float32, device="cuda")
            for c in reqs]
    sc.batch_autotune(reqs, rts, outs=outs)
    for _ in range(2):
        sc.render_batch(reqs, rts, outs=outs)
    ms, lat = timed_batches(sc, [reqs] * 5, [rts] * 5, [outs] * 5, True, flush, stream)
    seq_lat, seq_ms = [], []
    for rep in range(3):
        _flush(flush)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for c, t, o in zip(reqs, rts, outs):
            sc.render(c, float(t), out=o)
            torch.cuda.synchronize()
            seq_lat.append((time.perf_counter() - t0) * 1e3)
        seq_ms.append((time.perf_counter() - t0) * 1e3)
    res["serving_batch_mixed"] = dict(
        requests=64, resolutions="uniform over 512x512, 800x800, 1014x1352, 1352x1014",
        fps=64 / (statistics.median(ms) / 1e3), ms_per_batch=statistics.median(ms),
        p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)),
        sequential_fps=64 / (statistics.median(seq_ms) / 1e3),
        sequential_p50_ms=float(np.percentile(seq_lat, 50)),
        sequential_p99_ms=float(np.percentile(seq_lat, 99)),
        shape=sc.batch_info(64))
    # backward (fine-tuning step): L1 loss against a render of the scene with means perturbed
    # by N(0, 0.01); render with a frame, then the reverse replay + per-Gaussian chain
    res["backward"] = backward_timing(sc, cams, times, flush, stream)
    res["backward_tight"] = backward_timing(sc, cams, times, flush, stream, tight=True)
    # spatial-temporal variation score pass: 1M Gaussians, 50 timestamps x 4 cameras
    res["variation_score"] = score_timing(stream)
    # key-frame masks built from 4 training views (Sec. 4.2.2) instead of the 3-sigma recipe
    res["keyframe_masks_from_views"] = keyframe_mask_timing(sc, cams, times, flush, stream)
    # the 4DGS-1K pipeline on a self-distillation target: score, prune 80%, masks, fine-tune
    res["prune_and_finetune"] = finetune_timing()
    # vector-quantised SH decoded in the per-Gaussian kernel (Ours-PP)
    res["sh_vector_quantised"] = vq_timing(sc, cams, times, flush, stream)
    # unpruned 3M scene, single requests
    big = scenes.unpruned_scene()
    kt = scenes.keyframe_times()
    sc2 = fdgs.Scene.from_host(big)
    sc2.set_active_mask(torch.as_tensor(scenes.keyframe_masks(big, kt)).cuda(), kt)
    res["unpruned_masked"] = dict(single(sc2, True, fr[:12]), n_gaussians=big.n)
    res["unpruned_unmasked"] = dict(single(sc2, False, fr[:12]), n_gaussians=big.n)
    # the same scene in batches of 64 frames (the headline's frame walk)
    B = 64
    outs = [torch.empty((3, H_FULL, W_FULL), dtype=torch.float32, device="cuda")
            for _ in range(B)]
    steps = [frame_list(B, 7 * B), frame_list(B, 9 * B), frame_list(B, 11 * B)]
    bargs = [([cams[k] for k in f], [float(times[k]) for k in f]) for f in steps]
    sc2.render_batch(*bargs[0], outs=outs)
    stages = []
    ms, _ = timed_batches(sc2, [a for a, _ in bargs], [b_ for _, b_ in bargs], [outs] * 3, True,
                          flush, stream, stages)
    res["unpruned_masked_batched"] = dict(
        fps=B / (statistics.median(ms) / 1e3), ms_per_batch=statistics.median(ms), batch=B,
        n_gaussians=big.n, stage_ms={k: statistics.median([x[k] for x in stages])
                                     for k in stages[0]})
    del outs
    sc2.close()
    del big
    torch.cuda.empty_cache()
    return res


def keyframe_mask_timing(sc, cams, times, flush, stream, B=64):
    """Masks of the 50 key-frames from 4 training views on the arc: build time, realised
    active ratio, activation IoU of key-frame 0 with later ones (Sec. 4.1), and the batched
    render through them (64 frames at 1352x1014); the scene's synthetic masks are restored."""
    import torch

    from paper_2503_16422_gb300 import scenes
    views = [scenes.arc_camera(th, W_FULL, H_FULL) for th in (-10.0, -10.0 / 3, 10.0 / 3, 10.0)]
    kt = scenes.keyframe_times()
    sc.build_keyframe_masks(views, kt[:4])           # warm-up: one batch of the timed geometry
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    masks = sc.build_keyframe_masks(views, kt)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    rows = np.unpackbits(masks.cpu().numpy(), axis=1, bitorder="little")[:, :sc.n] > 0
    ratio = rows.mean(axis=1)

    def iou(a, b):
        u = (a | b).sum()
        return float((a & b).sum() / u) if u else 1.0

    synthetic = sc.active_mask
    sc.set_active_mask(masks, kt)
    outs = [torch.empty((3, H_FULL, W_FULL), dtype=torch.float32, device="cuda")
            for _ in range(B)]
    steps = [rank_requests(0, 1, B)[0], frame_list(B, 3 * B), frame_list(B, 5 * B)]
    args = [([cams[k] for k in fr], [float(times[k]) for k in fr]) for fr in steps]
    sc.render_batch(*args[0], outs=outs)
    ms, _ = timed_batches(sc, [a for a, _ in args], [b for _, b in args], [outs] * 3, True,
                          flush, stream)
    sc.set_active_mask(synthetic, kt)
    return dict(views=4, key_frames=len(kt), build_s=build_s,
                build_ms_per_render=build_s * 1e3 / (4 * len(kt)),
                active_ratio={"min": float(ratio.min()), "median": float(np.median(ratio)),
                              "max": float(ratio.max())},
                activation_iou_vs_key0={f"+{6 * d} frames": iou(rows[0], rows[d])
                                        for d in (1, 3, 10, 49)},
                batch_fps_through_these_masks=B / (statistics.median(ms) / 1e3))


def vq_timing(sc, cams, times, flush, stream, n_code=4096, B=64):
    """SH of the 200k scene quantised to n_code codes: encode time, colour storage, batched
    FPS through the codebook (64 masked frames at 1352x1014) and PSNR against the renders
    with full coefficients; the codebook is cleared afterwards."""
    import torch

    from paper_2503_16422_gb300 import finetune, vq
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    cb, codes = vq.quantize_sh(sc.params.sh, n_code=n_code, iters=10)
    torch.cuda.synchronize()
    enc_s = time.perf_counter() - t0
    fr = frame_list(6, 17)
    full = [sc.render(cams[k], float(times[k])) for k in fr]
    sc.set_sh_codebook(cb, codes)
    psnrs = [finetune.psnr(sc.render(cams[k], float(times[k])), f) for k, f in zip(fr, full)]
    outs = [torch.empty((3, H_FULL, W_FULL), dtype=torch.float32, device="cuda")
            for _ in range(B)]
    steps = [frame_list(B, 7 * B), frame_list(B, 9 * B), frame_list(B, 11 * B)]
    args = [([cams[k] for k in f_], [float(times[k]) for k in f_]) for f_ in steps]
    sc.render_batch(*args[0], outs=outs)
    ms, _ = timed_batches(sc, [a for a, _ in args], [b for _, b in args], [outs] * 3, True,
                          flush, stream)
    sc.set_sh_codebook(None, None)
    st = vq.storage_bytes(sc.n, sc.params.sh_degree, int(cb.shape[0]))
    return dict(n_code=int(cb.shape[0]), encode_s=enc_s,
                colour_bytes_full=st["full"], colour_bytes_quantised=st["quantised"],
                psnr_vs_full_sh=float(np.mean(psnrs)),
                batch_fps=B / (statistics.median(ms) / 1e3))


def finetune_timing(iters=1000, prune_ratio=0.9, lr_scale=0.3):
    """Teacher: the 200k-Gaussian scene. 48 training targets (4 views x 12 times at
    1352x1014) from it; STVS over them; prune 90% (the lowest-scoring 80% of these synthetic
    scenes is nearly invisible, so the paper's 80% leaves nothing to recover); key-frame
    masks of the student from the 4 views at the 50 key-frames; Adam fine-tuning through the
    filter (L1) at lr_scale x the library's fine-tuning rates. Reports ms per iteration and
    the training and held-out PSNR against the teacher before and after."""
    import torch

    from paper_2503_16422_gb300 import fdgs, finetune, scenes
    teacher = scenes.pruned_scene()
    tsc = fdgs.Scene.from_host(teacher)
    views = [scenes.arc_camera(th, W_FULL, H_FULL) for th in (-10.0, -10.0 / 3, 10.0 / 3, 10.0)]
    ts = [float(x) for x in np.linspace(0.02, 0.98, 12)]
    train = [(c, t, tsc.render(c, t, use_mask=False)) for t in ts for c in views]
    held = [(scenes.arc_camera(0.0, W_FULL, H_FULL), t) for t in (0.25, 0.65)]
    held = [(c, t, tsc.render(c, t, use_mask=False)) for c, t in held]
    score = tsc.variation_score(views, ts)
    keep = tsc.select_keep(score, prune_ratio)
    student = fdgs.Scene(finetune.prune(tsc.params, keep))
    kt = scenes.keyframe_times()
    student.set_active_mask(student.build_keyframe_masks(views, kt), kt)

    def psnr_of(vs):
        with torch.no_grad():
            return float(np.mean([finetune.psnr(student.render(c, t, use_mask=True), ref)
                                  for c, t, ref in vs]))

    held0, train0 = psnr_of(held), psnr_of(train)
    ft = finetune.FineTuner(student, {k: v * lr_scale for k, v in finetune.DEFAULT_LR.items()})
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = ft.run(train, iters)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ls = losses.cpu().numpy()
    out = dict(teacher_gaussians=tsc.n, kept=student.n, prune_ratio=prune_ratio,
               lr_scale=lr_scale, train_views=len(train), iterations=iters,
               ms_per_iteration=wall * 1e3 / iters,
               l1_first50=float(ls[:50].mean()), l1_last50=float(ls[-50:].mean()),
               train_psnr_before=train0, train_psnr_after=psnr_of(train),
               held_out_psnr_before=held0, held_out_psnr_after=psnr_of(held))
    student.close()
    tsc.close()
    del train, held, teacher
    torch.cuda.empty_cache()
    return out


def backward_timing(sc, cams, times, flush, stream, n_frames=6, tight=False):
    import torch

    from paper_2503_16422_gb300 import fdgs
    p = sc.params
    rng = np.random.default_rng(55)
    pert = p.mean4.clone()
    pert[:, :3] += torch.as_tensor(rng.normal(0, 0.01, (sc.n, 3)).astype(np.float32)).cuda()
    target_scene = fdgs.Scene(fdgs.SceneTensors(pert, p.logscale4, p.q_left, p.q_right,
                                                p.opacity_logit, p.sh, p.sh_degree))
    grads = fdgs.SceneTensors(*[torch.zeros_like(x) for x in p.list()], p.sh_degree)
    fwd_ms, bwd_ms = [], []
    for k in frame_list(n_frames, 40):
        cam, t = cams[k], float(times[k])
        target = target_scene.render(cam, t, use_mask=False)
        _flush(flush)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        img, fr = sc.render(cam, t, use_mask=False, keep_frame=True, tight=tight)
        e1.record(stream)
        dL = torch.sign(img - target) / img.numel()
        e1b = torch.cuda.Event(enable_timing=True)
        e1b.record(stream)
        sc.render_backward(fr, dL, grads=grads)
        e2.record(stream)
        e2.synchronize()
        fwd_ms.append(e0.elapsed_time(e1))
        bwd_ms.append(e1b.elapsed_time(e2))
        fr.release()
    target_scene.close()
    return dict(frames=n_frames, scene="pruned 200k, unmasked, 1352x1014",
                tile_sets="alpha-tight" if tight else "3-sigma squares",
                forward_ms=float(np.mean(fwd_ms)), backward_ms=float(np.mean(bwd_ms)))


def score_timing(stream):
    import torch

    from paper_2503_16422_gb300 import fdgs, scenes
    s = scenes.stvs_scene()
    sc = fdgs.Scene.from_host(s)
    cams = [scenes.arc_camera(th) for th in (-10.0, -3.3, 3.3, 10.0)]
    ts = [float(x) for x in np.linspace(0.0, 1.0, 50)]
    walls = {}
    for batch in (1, 8):
        # warm-up with the timed batch geometry (8 renders: 2 times x 4 cameras)
        sc.variation_score(cams, ts[:2], batch=batch)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        score = sc.variation_score(cams, ts, batch=batch)
        keep = sc.select_keep(score, 0.8)
        torch.cuda.synchronize()
        walls[batch] = time.perf_counter() - t0
        kept = int(keep.sum())
    sc.close()
    n = len(cams) * len(ts)
    return dict(n_gaussians=s.n, renders=n, resolution="1352x1014", batch=8,
                wall_s=walls[8], ms_per_render=walls[8] * 1e3 / n, kept=kept,
                per_frame_path_wall_s=walls[1])


# DRAM bytes the persistent blend moves per frame of a batch at 1352x1014 on the 200k pruned
# scene, from one ncu capture of an 8-frame launch of k_blend_persist<8, 4> (42.9 MB read +
# 76.9 MB written); to be re-captured whenever the blend kernel changes.
BLEND_PERSIST_DRAM_BYTES_PER_FRAME = (42894848 + 76912896) / 8
# Fraction of cycles the persistent blend issues an instruction (ncu smsp__issue_active, same
# capture).
BLEND_PERSIST_ISSUE_ACTIVE = 0.879


def launches_per_batch():
    # start, preprocess, partition scan, bases, segment compaction, depth sort (histogram,
    # scan, 5 passes), gather, block counts, tile scan, block lists, queue sort (histogram,
    # scan, 3 passes), persistent blend, and the 8 one-thread %globaltimer stamps
    return 1 + 1 + 1 + 1 + 1 + 7 + 1 + 1 + 1 + 1 + 5 + 1 + 8


def run_only(args):
    """One side workload alone (the headline is not measured): small enough on the device to
    profile a single kernel of it."""
    import torch

    from paper_2503_16422_gb300 import build, fdgs, scenes
    build.build()
    scene, kt, masks = pruned_masked()
    sc = fdgs.Scene.from_host(scene)
    sc.set_active_mask(torch.as_tensor(masks).cuda(), kt)
    times = scenes.frame_times()
    cams = {k: scenes.arc_camera(scenes.frame_theta(k)) for k in range(300)}
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    res = {}
    if args.only == "backward":
        for tight in (False, True):
            res["backward_tight" if tight else "backward"] = backward_timing(
                sc, cams, times, flush, stream, n_frames=max(args.steps, 1), tight=tight)
    if args.only == "masks":
        res["keyframe_masks_from_views"] = keyframe_mask_timing(sc, cams, times, flush, stream)
    sc.close()
    if args.only == "unpruned":
        # the 3M scene in batches of --batch frames (a small batch keeps a capture small)
        big = scenes.unpruned_scene()
        sc2 = fdgs.Scene.from_host(big)
        sc2.set_active_mask(torch.as_tensor(scenes.keyframe_masks(big, kt)).cuda(), kt)
        B = args.batch
        outs = [torch.empty((3, H_FULL, W_FULL), dtype=torch.float32, device="cuda")
                for _ in range(B)]
        fr = [frame_list(B, (7 + 2 * i) * B) for i in range(max(args.steps, 1))]
        bargs = [([cams[k] for k in f], [float(times[k]) for k in f]) for f in fr]
        sc2.render_batch(*bargs[0], outs=outs)
        stages = []
        ms, _ = timed_batches(sc2, [a for a, _ in bargs], [b_ for _, b_ in bargs],
                              [outs] * len(bargs), True, flush, stream, stages)
        res["unpruned_masked_batched"] = dict(
            fps=B / (statistics.median(ms) / 1e3), batch=B, n_gaussians=big.n,
            stage_ms={k: statistics.median([x[k] for x in stages]) for k in stages[0]})
        sc2.close()
    if args.only == "score":
        res["variation_score"] = score_timing(stream)
    print(json.dumps({"only": args.only, "impl": "ours", "data": "synthetic", **res}))


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    if args.only:
        if rank == 0:
            run_only(args)
        return
    if args.impl == "reference":
        if rank != 0:
            return
        scene, kt, masks = pruned_masked()
        for w in range(args.warmup):
            cpu_oracle_frame(scene, kt, masks, frame=frame_list(1, 200 + w)[0], budget_s=1.0)
        secs = []
        for i in range(max(args.steps, 1)):
            s_, desc, cores = cpu_oracle_frame(scene, kt, masks, frame=frame_list(1, i)[0],
                                               budget_s=4.0)
            secs.append(s_)
        fps = len(secs) / sum(secs)
        line = {"metric": METRIC, "value": fps, "unit": "FPS", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / fps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic",
                "config": workload_config(scene, kt, args.batch), "impl": "reference",
                "cpu_baseline": {"value": fps, "unit": "FPS", "cores": cores, "kind": "oracle",
                                 "sample": "per step: one frame of the batched workload, "
                                           + desc},
                "e2e": {"value": fps, "unit": "FPS", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return
    value, ms, res, scene, kt, masks, world, rank = run_ours(args)
    if rank != 0:
        return
    lat = res["lat"]
    line = {"metric": METRIC, "value": value, "unit": "FPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": workload_config(scene, kt, args.batch),
            "roofline": res["roofline"], "clocks": res["clocks"], "e2e": res["e2e"],
            "gpu_launches": launches_per_batch() * args.steps,
            "latency_ms": {"p50": float(np.percentile(lat, 50)),
                           "p99": float(np.percentile(lat, 99))},
            "batch_shape": {k: v for k, v in res["batch_shape"].items() if k != "latency_ms"},
            "batch_stages_ms": res["batch_stages_ms"],
            "batch_rates": res["batch_rates"],
            "single_frame_stages_ms": res["stage_ms"], "stage_gbs": res["stage_gbs"],
            "stage_rates": res["stage_rates"],
            "single_frame_roofline": res["single_roofline"],
            "counts_per_frame": res["counts"]}
    if "warm_l2" in res:
        line["warm_l2"] = res["warm_l2"]
    if "comparisons" in res:
        line["comparisons"] = res["comparisons"]
    if not args.no_cpu_baseline:
        s_, desc, cores = cpu_oracle_frame(scene, kt, masks)
        line["cpu_baseline"] = {"value": 1.0 / s_, "unit": "FPS", "cores": cores,
                                "kind": "oracle", "sample": desc}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
