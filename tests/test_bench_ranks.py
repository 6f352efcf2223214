"""The host side of the multi-GPU bench path (replicas: every rank solves its
own inputs, the slowest rank sets the time), on CPU with two gloo ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        m = bench.max_over_ranks([float(rank + 1), 5.0 - rank, 7.0], world, device="cpu")
        bench.dist_barrier(world)
        # replicas solve different inputs: a checksum of each rank's video
        y = bench.rpca_inputs(rank, T=4, H=16, W=16)
        sums = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(sums, torch.tensor([float(y.sum())], dtype=torch.float64))
        ref = bench.run_reference(type("A", (), {"workload": "prox", "warmup": 0, "steps": 1, "n_inner": 1})(),
                                  rank, world) if rank == 1 else "skipped"
        out[rank] = (m, [float(v) for v in sums], ref)
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_max_and_solve_different_inputs():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        m, sums, _ = out[r]
        assert m == [2.0, 5.0, 7.0]
        assert sums[0] != sums[1]
    assert out[1][2] is None          # the reference arm runs on rank 0 only


def test_single_rank_is_the_identity():
    import bench
    assert bench.max_over_ranks([3.0, 1.0], 1) == [3.0, 1.0]
    bench.dist_barrier(1)
