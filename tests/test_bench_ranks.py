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


def test_threaded_csr_products_equal_scipy_and_drive_the_oracle_cgls():
    """The CPU baseline's threaded sparse products (row blocks of A and of
    A^T on separate threads) equal SciPy's own A @ v and A.T @ v, for thread
    counts that do and do not divide the row count, and the oracle's CGLS
    takes the same iterates through them as through the plain matrix."""
    np = pytest.importorskip("numpy")
    sp = pytest.importorskip("scipy.sparse")
    import bench
    from oracle import pn as opn
    rng = np.random.Generator(np.random.PCG64(5))
    A = sp.random(101, 101, density=0.05, random_state=7, format="csr") + sp.identity(101, format="csr") * 3.0
    v = rng.standard_normal(101)
    for threads in (1, 3, 8):
        op = bench.ThreadedCSR(A.tocsr(), threads)
        assert np.array_equal(op @ v, A @ v)
        assert np.array_equal(op.T @ v, A.T @ v)
        op.close()
    b = rng.standard_normal(101)
    op = bench.ThreadedCSR(A.tocsr(), 4)
    x1 = opn.cgls(op, b, tol=1e-300, max_iter=12)
    x2 = opn.cgls(A.tocsr(), b, tol=1e-300, max_iter=12)
    op.close()
    r1 = x1[0] if isinstance(x1, tuple) else x1
    r2 = x2[0] if isinstance(x2, tuple) else x2
    assert np.array_equal(r1, r2)


def test_reference_arm_prints_one_contract_line():
    """bench.py --impl reference (the FP64 oracle's CGLS on the host cores,
    the reference arm of this paper-only build) prints one JSON line with the
    contract's keys: the metric and unit of the GPU arm, impl "reference", a
    cpu_baseline naming the method, cores and sample, and an e2e object whose
    value is the line's own with no host-device copies."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1"],
                         cwd=root, env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "solve/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["steps"] == 1 and d["warmup"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and "CGLS" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
