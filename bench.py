#!/usr/bin/env python
"""Benchmark: masked 4D Gaussian render FPS at 1352x1014 on one GB300, with per-stage times,
the roofline fraction of the dominant stage, an end-to-end number and the CPU oracle.

Workload (default): the pruned 4DGS-1K-like scene (200,000 Gaussians, degree-3 SH, temporal
log-scales N(-1, 0.5)) rendered with the key-frame temporal filter (masks every 6 frames,
|t_k - mu_t| < 3 s_t) at 1352x1014, frames k = 0..299 with t_k = k/299 and the camera on a
20-degree arc; one step = one full render (all stages) of the next frame. Inputs are
synthetic (seeded), resident in HBM; L2 is flushed (256 MiB write) before every timed step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload pruned_masked|unpruned_masked|pruned_unmasked|unpruned_unmasked]

With --gpus N > 1 (launched under torchrun) every rank renders its own frames of a replica of
the scene (no collective: the frames are independent), timing is the max over ranks and the
value is the total frames of all ranks per second.
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
BLEND_FLOP_PER_EVAL = 20      # algorithmic FP32 FLOP per (Gaussian, pixel) evaluation


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="pruned_masked",
                    choices=["pruned_masked", "unpruned_masked", "pruned_unmasked",
                             "unpruned_unmasked"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the comparison workloads")
    return ap.parse_args()


def make_workload(name):
    from paper_2503_16422_gb300 import scenes
    scene = scenes.pruned_scene() if name.startswith("pruned") else scenes.unpruned_scene()
    masked = name.endswith("_masked")
    kt = scenes.keyframe_times()
    masks = scenes.keyframe_masks(scene, kt) if masked else None
    return scene, masked, kt, masks


def frame_list(steps, offset=0):
    """Frame indices visited by the steps: a stride-7 walk over the 300 frames."""
    return [((offset + i) * 7) % 300 for i in range(steps)]


def workload_config(name, scene, masked, kt):
    return {"workload": f"{name}: {scene.n} Gaussians, degree-{scene.sh_degree} SH, 1352x1014, "
                        f"300 frames on a 20-degree arc" +
                        (f", key-frame masks every 6 frames ({len(kt)})" if masked else ", no mask"),
            "n_gaussians": scene.n, "width": 1352, "height": 1014, "tile": 16,
            "masked": masked, "l2": "flushed before every timed step (256 MiB write)"}


# ---- peaks ---------------------------------------------------------------------------------

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


# ---- clocks sampler ------------------------------------------------------------------------

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
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
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


# ---- CPU oracle baseline -------------------------------------------------------------------

def cpu_oracle_fps(scene, masked, kt, masks, n_tiles=24, frame=150):
    """FP64 oracle on a bounded sample of one frame: the whole per-Gaussian stage plus the
    blend of n_tiles randomly chosen tiles (of 5,440); the tile time is scaled to the frame."""
    import torch

    import oracle
    from paper_2503_16422_gb300 import scenes
    cam = scenes.arc_camera(scenes.frame_theta(frame))
    t = float(scenes.frame_times()[frame])
    active = oracle.active_from_masks(masks, kt, t, scene.n) if masked else None
    P = oracle.Params.from_scene(scene)
    t0 = time.perf_counter()
    pre = oracle.preprocess(P, cam, t, active)
    t1 = time.perf_counter()
    gx, gy = pre["grid"]
    tiles = np.random.default_rng(0).choice(gx * gy, n_tiles, replace=False).tolist()
    oracle.render(P, cam, t, active, tiles=tiles, pre=pre)
    t2 = time.perf_counter()
    frame_s = (t1 - t0) + (t2 - t1) * (gx * gy) / n_tiles
    return dict(value=1.0 / frame_s, unit="FPS", cores=torch.get_num_threads(), kind="oracle",
                sample=f"1 frame (k={frame}): per-Gaussian stage of all {scene.n} Gaussians "
                       f"+ blend of {n_tiles}/{gx * gy} random tiles, scaled to the frame "
                       f"({t2 - t0:.1f} s of CPU work)")


# ---- our implementation ----------------------------------------------------------------------

def stage_bytes(stats, n, deg, masked):
    """Algorithmic DRAM bytes of each HBM-bound stage for one frame."""
    na, nv, K, kb = stats["n_active"], stats["n_visible"], stats["n_keys"], stats["key_bytes"]
    sh = (deg + 1) ** 2 * 3 * 4
    tiles = stats["tiles_x"] * stats["tiles_y"]
    passes = math.ceil(math.ceil(math.log2(max(tiles, 2))) / 8)
    return {
        "preprocess": (2 * math.ceil(n / 32) * 4 if masked else 0) + na * 68 + nv * (sh + 48 + 8),
        "depth_sort": nv * 8 + 4 * nv * 16,
        "gather_scan": nv * (8 + 48 + 64 + 4 + 16),
        "emit": nv * (20 + 4) + K * kb,
        "tile_sort": passes * K * kb * 2,
        "tile_scan": (stats["tiles_x"] + 1) * (stats["tiles_y"] + 1) * 4 * 3 + tiles * 8,
    }


def _timed_steps(sc, cams, times, frames, masked, out, flush, stream):
    import torch
    step_ms = []
    for k in frames:
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sc.render(cams[k], float(times[k]), use_mask=masked, out=out)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    return step_ms


def _profile_frames(sc, cams, times, frames, masked, out, flush, scene):
    """Untimed pass over the same frames: per-stage CUDA-event times, frame counts and the
    blend evaluation count (the counting kernel variant is not the timed one)."""
    from paper_2503_16422_gb300 import fdgs
    sc.profile(1)
    acc = {s: 0.0 for s in fdgs.PROFILE_STAGES}
    stats_acc = []
    for k in frames:
        flush.fill_(1.0)
        _, fr = sc.render(cams[k], float(times[k]), use_mask=masked, out=out, keep_frame=True)
        ms, _ = sc.profile_read()
        for s_ in acc:
            acc[s_] += ms[s_]
        stats_acc.append(fr.stats())
        fr.release()
    sc.profile(2)
    evals = 0
    for k in frames:
        sc.render(cams[k], float(times[k]), use_mask=masked, out=out)
        evals += sc.profile_read()[1]
    sc.profile(0)
    nfr = len(frames)
    stage_ms = {s_: acc[s_] / nfr for s_ in acc}
    mean_stats = {f: float(np.mean([st[f] for st in stats_acc]))
                  for f in ("n_active", "n_visible", "n_keys")}
    sb = [stage_bytes(st, scene.n, scene.sh_degree, masked) for st in stats_acc]
    bytes_mean = {s_: float(np.mean([b[s_] for b in sb])) for s_ in sb[0]}
    return stage_ms, mean_stats, bytes_mean, evals / nfr


def _roofline(stage_ms, bytes_mean, evals_per_frame):
    pk = peaks()
    dom = max((s_ for s_ in stage_ms if s_ != "host_sync"), key=stage_ms.get)
    if dom == "blend":
        ach = evals_per_frame * BLEND_FLOP_PER_EVAL / (stage_ms["blend"] / 1e3) / 1e12
        peak = fp32_peak_tflops(pk["sm_mhz"])
        return {"bound": "alu", "kernel": "k_blend", "achieved": ach, "peak": peak,
                "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
                "peak_src": f"derived: 152 SMs x 128 FP32 lanes x 2 FLOP x {pk['sm_mhz']:.0f} MHz"}
    ach = bytes_mean[dom] / (stage_ms[dom] / 1e3) / 1e9
    return {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": pk["hbm"], "unit": "GB/s",
            "frac": ach / pk["hbm"], "traffic": None, "peak_src": pk["src"]}


def _scene_on_gpu(name):
    import torch

    from paper_2503_16422_gb300 import fdgs
    scene, masked, kt, masks = make_workload(name)
    sc = fdgs.Scene.from_host(scene)
    if masked:
        sc.set_active_mask(torch.as_tensor(masks).cuda(), kt)
    return scene, masked, kt, masks, sc


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2503_16422_gb300 import build, scenes
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build.build()
    scene, masked, kt, masks, sc = _scene_on_gpu(args.workload)
    times = scenes.frame_times()
    cams = {k: scenes.arc_camera(scenes.frame_theta(k)) for k in range(300)}
    out = torch.empty((3, 1014, 1352), dtype=torch.float32, device="cuda")
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    for k in frame_list(args.warmup, 1000 + rank):
        sc.render(cams[k], float(times[k]), use_mask=masked, out=out)
    torch.cuda.synchronize()
    frames = frame_list(args.steps, rank * 37)
    clocks = Clocks(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms = _timed_steps(sc, cams, times, frames, masked, out, flush, stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    total_ms = sum(step_ms)
    if world > 1:
        tt = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms = float(tt.item())
    value = world * len(frames) / (total_ms / 1e3)

    # end to end through the public API: per step the camera and t go host->device as
    # launch arguments and the rendered image comes back to pinned host memory
    host = torch.empty((3, 1014, 1352), dtype=torch.float32, pin_memory=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in frames:
        sc.render(cams[k], float(times[k]), use_mask=masked, out=out)
        host.copy_(out, non_blocking=True)
        stream.synchronize()
    e2e_s = time.perf_counter() - t0
    cam_bytes = 16 * 4 + 4 * 4 + 3 * 4 + 4 + 4 + 4   # fdgs_camera + t + opts
    res = {}
    if rank == 0:
        stage_ms, mean_stats, bytes_mean, evals = _profile_frames(
            sc, cams, times, frames, masked, out, flush, scene)
        res = dict(stage_ms=stage_ms, mean_counts=mean_stats, evals_per_frame=evals,
                   roofline=_roofline(stage_ms, bytes_mean, evals), clocks=clk,
                   e2e=dict(value=len(frames) / e2e_s, unit="FPS",
                            h2d_bytes_per_step=cam_bytes,
                            d2h_bytes_per_step=3 * 1014 * 1352 * 4),
                   stage_gbs={s_: bytes_mean[s_] / (stage_ms[s_] / 1e3) / 1e9
                              for s_ in bytes_mean if stage_ms[s_] > 0},
                   blend_tflops=evals * BLEND_FLOP_PER_EVAL / max(stage_ms["blend"], 1e-9) / 1e9)
    sc.close()
    if rank == 0 and not args.no_extra:
        res["comparisons"] = {}
        for name in ("pruned_unmasked", "unpruned_masked", "unpruned_unmasked"):
            if name == args.workload:
                continue
            sc2 = None
            try:
                scn, msk, _, _, sc2 = _scene_on_gpu(name)
                fr = frame_list(12, 5)
                for k in frame_list(2, 900):
                    sc2.render(cams[k], float(times[k]), use_mask=msk, out=out)
                ms = _timed_steps(sc2, cams, times, fr, msk, out, flush, stream)
                st_ms, counts, _, ev = _profile_frames(sc2, cams, times, fr[:4], msk, out,
                                                       flush, scn)
                res["comparisons"][name] = dict(
                    fps=len(fr) / (sum(ms) / 1e3), ms_per_frame=sum(ms) / len(fr),
                    raster_ms=sum(st_ms[s_] for s_ in ("tile_scan", "emit", "tile_sort", "blend")),
                    stages_ms=st_ms, counts_per_frame=dict(counts, blend_evals=ev))
            except Exception as e:   # a comparison must not hide the headline number
                res["comparisons"][name] = {"error": str(e)[:200]}
            finally:
                if sc2 is not None:
                    sc2.close()
                torch.cuda.empty_cache()
    return value, total_ms / len(frames), res, scene, masked, kt, masks, world, rank


def launches_per_frame(masked):
    # memsets are not kernels; per frame: preprocess, depth sort (hist, scan, 4 passes),
    # gather_scan, emit, tile sort (hist, scan, 2 passes), ranges, blend
    return 1 + 6 + 1 + 1 + 4 + 1 + 1


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return
        scene, masked, kt, masks = make_workload(args.workload)
        for _ in range(args.warmup):
            pass
        vals = []
        for i in range(max(args.steps, 1)):
            r = cpu_oracle_fps(scene, masked, kt, masks, n_tiles=4, frame=frame_list(1, i)[0])
            vals.append(1.0 / r["value"])
        fps = len(vals) / sum(vals)
        cb = dict(r, value=fps)
        line = {"metric": METRIC, "value": fps, "unit": "FPS", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / fps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic",
                "config": workload_config(args.workload, scene, masked, kt),
                "impl": "reference", "cpu_baseline": cb,
                "e2e": {"value": fps, "unit": "FPS", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return
    value, ms, res, scene, masked, kt, masks, world, rank = run_ours(args)
    if rank != 0:
        return
    line = {"metric": METRIC, "value": value, "unit": "FPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": workload_config(args.workload, scene, masked, kt)}
    line.update({k: res[k] for k in ("roofline", "clocks", "e2e")})
    line["gpu_launches"] = launches_per_frame(masked) * args.steps
    line["stages_ms"] = res["stage_ms"]
    line["stage_gbs"] = res["stage_gbs"]
    line["blend_tflops"] = res["blend_tflops"]
    line["counts_per_frame"] = dict(res["mean_counts"], blend_evals=res["evals_per_frame"])
    line["raster_ms"] = sum(res["stage_ms"][s_] for s_ in ("tile_scan", "emit", "tile_sort", "blend"))
    if "comparisons" in res:
        line["comparisons"] = res["comparisons"]
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_oracle_fps(scene, masked, kt, masks)
    print(json.dumps(line))


if __name__ == "__main__":
    main()
