"""Host logic of the sharded path on CPU (gloo, world size 2): the partition
of a tensor along its last mode, the fixed-order reduction of the partial
Grams (Algorithm 2's sum over slabs split across ranks), and bench.py's
max-over-ranks timing.  The partial Grams come from the oracle here; the GPU
kernels' partials are checked in test_gpu_parity.py."""
import datetime
import os
import socket

import numpy as np
import pytest

import oracle
from paper_1901_06043_gb300 import shard

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=60))
    return dist


def _gram_worker(rank, world, port, dims, outdir):
    dist = _init(rank, world, port)
    try:
        x = np.random.default_rng(7).standard_normal(oracle.linear_size(dims))
        a, b = shard.shard_slice(dims, world, rank)
        sd = shard.shard_dims(dims, world, rank)
        for n in range(len(dims) - 1):
            part = torch.from_numpy(oracle.gram(x[a:b], sd, n))
            S = shard.allreduce_fixed_order(part)
            np.save(os.path.join(outdir, f"S{n}_r{rank}.npy"), S.numpy())
    finally:
        dist.destroy_process_group()


def _bench_worker(rank, world, port, outdir):
    dist = _init(rank, world, port)
    try:
        import bench
        bench.barrier(world)
        m = bench.reduce_max(10.0 + rank, world)
        np.save(os.path.join(outdir, f"max_r{rank}.npy"), np.array([m]))
    finally:
        dist.destroy_process_group()


def test_shard_bounds_partition():
    for dims in [(5, 4, 7), (3, 2, 1), (6, 9), (4, 4, 4, 11, 8)]:
        for world in (1, 2, 3, 4):
            spans = [shard.shard_bounds(dims, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == dims[-1]
            for (lo, hi), (lo2, _) in zip(spans, spans[1:]):
                assert hi == lo2
            sizes = [hi - lo for lo, hi in spans]
            assert max(sizes) - min(sizes) <= 1
            # the flat slices tile the whole array in order
            sl = [shard.shard_slice(dims, world, r) for r in range(world)]
            assert sl[0][0] == 0 and sl[-1][1] == oracle.linear_size(dims)
            assert all(b == c for (_, b), (c, _) in zip(sl, sl[1:]))


def test_sharded_gram_fixed_order_gloo(tmp_path):
    """Sum over two shards of the last mode equals the full Gram of every
    mode n < N-1, and both ranks hold bitwise-identical results."""
    dims = (6, 5, 4, 7)
    world = 2
    torch.multiprocessing.spawn(_gram_worker, args=(world, _free_port(), dims, str(tmp_path)),
                                nprocs=world, join=True)
    x = np.random.default_rng(7).standard_normal(oracle.linear_size(dims))
    for n in range(len(dims) - 1):
        S0 = np.load(tmp_path / f"S{n}_r0.npy")
        S1 = np.load(tmp_path / f"S{n}_r1.npy")
        assert np.array_equal(S0, S1)
        want = oracle.gram(x, dims, n)
        assert np.abs(S0 - want).max() <= 1e-13 * np.abs(want).max()


def test_bench_max_over_ranks_gloo(tmp_path):
    world = 2
    torch.multiprocessing.spawn(_bench_worker, args=(world, _free_port(), str(tmp_path)),
                                nprocs=world, join=True)
    for r in range(world):
        assert float(np.load(tmp_path / f"max_r{r}.npy")[0]) == 11.0
