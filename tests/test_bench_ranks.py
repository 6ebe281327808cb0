"""The replica (N > 1) timing logic of bench.py on CPU with two gloo ranks: the job's time
is the slowest rank's, and the whole-job throughput counts every rank's units against
it (weak scaling; one MPDO circuit does not shard, so ranks are independent replicas)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = 100.0 + 50.0 * rank                     # rank 1 is the slower replica
        job_ms = bench.max_over_ranks(ms, dist, device="cpu")
        out[rank] = (job_ms, bench.job_throughput(world, 3, 32 * 297, job_ms))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_replica_timing_takes_the_slowest_rank():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        job_ms, value = out[r]
        assert job_ms == 150.0
        assert value == pytest.approx(world * 3 * 32 * 297 / 0.150)


def test_single_process_passes_through():
    import bench
    assert bench.max_over_ranks(12.5, None) == 12.5
    assert bench.job_throughput(1, 2, 100, 1000.0) == pytest.approx(200.0)
