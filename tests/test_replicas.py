"""Multi-GPU replica logic of bench.py on CPU: two gloo ranks run the per-rank request walk
and the whole-job throughput with the maximum over ranks, as `bench.py --gpus 2` does under
torchrun (there over NCCL, one GPU per rank). No GPU and no CUDA call is involved."""
import os
import socket

import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        reqs = bench.rank_requests(rank, steps=3, batch=4)
        gathered = [None] * world
        dist.all_gather_object(gathered, reqs)

        def max_over_ranks(ms):
            t = torch.tensor([ms], dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            return float(t.item())

        local_ms = 100.0 + 20.0 * rank           # rank 1 is the slower replica
        fps, t_ms = bench.job_fps(local_ms, 3 * 4, world, max_over_ranks)
        dist.barrier()
        q.put((rank, gathered, fps, t_ms))
    finally:
        dist.destroy_process_group()


def test_two_replicas_over_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    results.sort()
    for rank, gathered, fps, t_ms in results:
        # every rank sees the same slowest time and the whole-job frames over it
        assert t_ms == 120.0
        assert abs(fps - 2 * 12 / 0.120) < 1e-9
        # each replica renders its own request stream: 3 steps of 4 frames in [0, 300)
        assert len(gathered) == 2 and gathered[0] != gathered[1]
        for stream in gathered:
            assert len(stream) == 3 and all(len(step) == 4 for step in stream)
            assert all(0 <= k < 300 for step in stream for k in step)


def test_job_fps_single_gpu():
    import bench
    fps, t_ms = bench.job_fps(250.0, 64 * 20, 1)
    assert t_ms == 250.0 and abs(fps - 64 * 20 / 0.25) < 1e-9
    assert bench.rank_requests(0, 2, 3) == [bench.frame_list(3, 0), bench.frame_list(3, 3)]
