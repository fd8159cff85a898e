"""The multi-rank path on the host: world_size 2 over gloo (127.0.0.1).
Each rank evaluates its contiguous share of the parameter points (here with
the FP64 oracle standing in for the GPU), the gathered log-likelihoods equal
a single-process evaluation in point order, and the step-time reduction
returns the max over ranks."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1505_07674_gb300.shard import loglike_sharded, reduce_max, shard_range  # noqa: E402


def test_shard_range_partitions():
    for n in (0, 1, 7, 4096, 4097):
        for world in (1, 2, 3, 8):
            got = [shard_range(n, r, world) for r in range(world)]
            assert got[0][0] == 0 and got[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(got, got[1:]))
            sizes = [e - s for s, e in got]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_range(10, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import oracle as O
        import workloads as W
        spec = W.shrink(W.c1_small(), 24, 20)
        obs = O.mock_observation(spec)
        osys = O.OracleSystem(spec, obs)
        pts = W.draw_points(spec, 9, 3)  # 9 points: uneven shares 5 / 4
        ll = loglike_sharded(lambda p: osys.loglike(p, nthreads=1), pts)
        mx = reduce_max(10.0 + rank)
        own = loglike_sharded(lambda p: osys.loglike(p, nthreads=1), pts, gather=False)
        q.put((rank, ll, mx, len(own)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gather_and_max():
    from oracle import oracle as O
    import workloads as W
    O.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    spec = W.shrink(W.c1_small(), 24, 20)
    obs = O.mock_observation(spec)
    ref = O.OracleSystem(spec, obs).loglike(W.draw_points(spec, 9, 3), nthreads=1)
    for rank, ll, mx, n_own in sorted(res, key=lambda r: r[0]):
        assert np.array_equal(ll, ref)
        assert mx == 11.0
        assert n_own == (5 if rank == 0 else 4)
