"""Multi-rank logic of bench.py on CPU: world size 2 over gloo.  Every rank
solves its own problem (no data-path collective); the timing reported is the
maximum over ranks and the throughput counts the units of all ranks."""
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


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r pretends its K steps took (r + 1) seconds
    total = bench.max_over_ranks(float(rank + 1), world)
    bench.barrier(world)
    out[rank] = total
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == 2.0 and out[1] == 2.0


def test_replica_seeds_differ_by_rank():
    import pn_inputs
    a, b = pn_inputs.p5_64_fbm(0), pn_inputs.p5_64_fbm(1)
    assert a.source_voxel != b.source_voxel or (a.sigma_t != b.sigma_t).any()
