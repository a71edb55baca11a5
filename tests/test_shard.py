"""Host logic of the sharded path on CPU (gloo, world size 2 and 3): the
partition of a tensor along its last mode, the fixed-order reduction of the
partial Grams (Algorithm 2's sum over slabs split across ranks), the
all-gather of uneven last-mode shards, the whole sharded ST-HOSVD against
the unsharded oracle (the per-rank steps done by the oracle here), and
bench.py's max-over-ranks timing.  One GPU test runs the sharded driver
with the library's own steps (LibraryOps) as a single gloo rank."""
import datetime
import os
import socket

import numpy as np
import pytest

import oracle
from paper_1901_06043_gb300 import shard, synth

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


class _OracleOps:
    """The per-rank steps of the sharded ST-HOSVD done by the oracle on the
    host (torch FP64 tensors in and out), so the exchange pattern runs on
    gloo ranks without a GPU."""

    def norm_sq(self, y):
        return oracle.norm_sq(y.numpy())

    def gram(self, y, dims, n):
        return torch.from_numpy(oracle.gram(y.numpy(), dims, n))

    def eig_trunc(self, S, thr, R):
        lam, V = oracle.eig_desc(S.numpy())
        if R > 0:
            _, tail = oracle.rank_cut(lam, 0.0)
        else:
            R, tail = oracle.rank_cut(lam, thr)
        return torch.from_numpy(lam), torch.from_numpy(V[:, :R].copy()), R, float(tail[R])

    def ttm(self, y, dims, n, U):
        return torch.from_numpy(oracle.ttm(y.numpy(), dims, n, U.numpy().T))

    def to_comm(self, t):
        return t

    def from_comm(self, t):
        return t


def _sthosvd_worker(rank, world, port, dims, spec, outdir):
    dist = _init(rank, world, port)
    try:
        x, _ = synth.tucker_numpy(dims, tuple(max(1, d // 2) for d in dims), decay=0.1, eta=1e-4,
                                  seed=13)
        a, b = shard.shard_slice(dims, world, rank)
        kw = {"eps": 1e-2} if spec == "eps" else {"ranks": tuple(max(1, d // 3) for d in dims)}
        res = shard.sharded_sthosvd(torch.from_numpy(x[a:b].copy()), dims, world, rank,
                                    _OracleOps(), **kw)
        np.save(os.path.join(outdir, f"core_r{rank}.npy"), res["core"].numpy())
        np.save(os.path.join(outdir, f"ranks_r{rank}.npy"), np.array(res["ranks"]))
        np.save(os.path.join(outdir, f"disc_r{rank}.npy"), np.array(res["discarded"]))
        for n, U in enumerate(res["factors"]):
            np.save(os.path.join(outdir, f"U{n}_r{rank}.npy"), U.numpy())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("dims,world,spec", [((6, 5, 4, 7), 2, "eps"), ((6, 5, 4, 7), 2, "ranks"),
                                             ((9, 8, 5), 3, "eps")])
def test_sharded_sthosvd_matches_the_unsharded_oracle(tmp_path, dims, world, spec):
    """The whole sharded ST-HOSVD on gloo ranks (per mode n < N-1: local Gram,
    fixed-order sum, redundant eigensolve and cut, local TTM; then the
    all-gather of the partial core and the last mode): every rank holds the
    same ranks, factors and core, and they match the oracle's ST-HOSVD of
    the whole tensor."""
    torch.multiprocessing.spawn(_sthosvd_worker,
                                args=(world, _free_port(), dims, spec, str(tmp_path)),
                                nprocs=world, join=True)
    x, _ = synth.tucker_numpy(dims, tuple(max(1, d // 2) for d in dims), decay=0.1, eta=1e-4,
                              seed=13)
    kw = {"eps": 1e-2} if spec == "eps" else {"ranks": tuple(max(1, d // 3) for d in dims)}
    ref = oracle.sthosvd(x, dims, **kw)
    cores = [np.load(tmp_path / f"core_r{r}.npy") for r in range(world)]
    for r in range(world):
        assert tuple(np.load(tmp_path / f"ranks_r{r}.npy")) == ref["ranks"]
        assert np.array_equal(cores[r], cores[0])          # bitwise identical on every rank
        assert np.allclose(np.load(tmp_path / f"disc_r{r}.npy"), ref["discarded"],
                           rtol=1e-10, atol=1e-13 * ref["norm_sq"])
    for n in range(len(dims)):
        U = np.load(tmp_path / f"U{n}_r0.npy")
        W = ref["factors"][n]
        assert np.linalg.norm(W - U @ (U.T @ W), 2) <= 1e-10
    ours = {"core": cores[0], "core_dims": ref["ranks"],
            "factors": [np.load(tmp_path / f"U{n}_r0.npy") for n in range(len(dims))],
            "discarded": list(np.load(tmp_path / "disc_r0.npy")), "norm_sq": ref["norm_sq"]}
    e1 = oracle.relative_errors(x, dims, ours)["err_explicit"]
    e0 = oracle.relative_errors(x, dims, ref)["err_explicit"]
    assert abs(e1 - e0) <= 1e-12


def _gather_worker(rank, world, port, dims, outdir):
    dist = _init(rank, world, port)
    try:
        x = np.arange(oracle.linear_size(dims), dtype=np.float64)
        a, b = shard.shard_slice(dims, world, rank)
        full = shard.allgather_last_mode(torch.from_numpy(x[a:b].copy()), dims, world, rank)
        np.save(os.path.join(outdir, f"g_r{rank}.npy"), full.numpy())
    finally:
        dist.destroy_process_group()


def test_allgather_of_uneven_last_mode_shards(tmp_path):
    dims, world = (3, 4, 5), 3                     # shards of 1, 2, 2 last indices
    torch.multiprocessing.spawn(_gather_worker, args=(world, _free_port(), dims, str(tmp_path)),
                                nprocs=world, join=True)
    for r in range(world):
        assert np.array_equal(np.load(tmp_path / f"g_r{r}.npy"), np.arange(60, dtype=np.float64))


@pytest.mark.gpu
def test_sharded_driver_with_library_ops_one_rank():
    """LibraryOps on this GPU as a world of one gloo rank: the sharded
    driver's result equals tucker_sthosvd's (same kernels, same order)."""
    import torch.distributed as dist
    from paper_1901_06043_gb300 import tucker
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(_free_port())
    dist.init_process_group("gloo", rank=0, world_size=1)
    try:
        dims = (40, 30, 20, 6)
        x, _ = synth.tucker_numpy(dims, (8, 8, 6, 3), decay=0.1, eta=1e-4, seed=2)
        xd = torch.from_numpy(x).cuda()
        ctx = tucker.Context()
        got = shard.sharded_sthosvd(xd, dims, 1, 0, shard.LibraryOps(ctx, "fp64"), eps=1e-3)
        ref = oracle.sthosvd(x, dims, eps=1e-3)
        assert got["ranks"] == ref["ranks"]
        ours = {"core": got["core"].cpu().numpy(), "core_dims": got["ranks"],
                "factors": [U.cpu().numpy() for U in got["factors"]],
                "discarded": got["discarded"], "norm_sq": got["norm_sq"]}
        e1 = oracle.relative_errors(x, dims, ours)["err_explicit"]
        e0 = oracle.relative_errors(x, dims, ref)["err_explicit"]
        assert abs(e1 - e0) <= 1e-12
        ctx.close()
    finally:
        dist.destroy_process_group()
