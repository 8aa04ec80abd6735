"""The multi-replica bookkeeping of bench.py on CPU: world_size 2 over gloo
(one process per rank, as torchrun launches them).  Each rank fits its own
image, so the job time is the slowest rank's and the throughput counts the
spectra of all ranks."""
import multiprocessing as mp
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    ms = 10.0 + 5.0 * rank  # rank 1 is slower
    slowest = bench.max_over_ranks(ms, dist, device="cpu")
    q.put((rank, slowest, bench.job_throughput(world, 1000, slowest)))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_throughput_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    env_keep = os.environ.get("PYTHONPATH", "")
    os.environ["PYTHONPATH"] = os.pathsep.join([os.path.dirname(os.path.dirname(__file__)), env_keep])
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, thr in got:
        assert slowest == 15.0
        assert thr == pytest.approx(2 * 1000 / 0.015)


def test_single_process_passthrough():
    import bench

    assert bench.max_over_ranks(12.5, None) == 12.5
    assert bench.job_throughput(1, 500, 10.0) == pytest.approx(50_000.0)
