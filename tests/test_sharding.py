"""Multi-rank path on the CPU (gloo, world size 2): ranks simulate disjoint
slices of the sample-index range and gather the accepted samples on the host;
the union equals the unsplit run (Sec. 3.1). The per-rank compute here is the
oracle, so no GPU is needed; the CUDA library is sharded the same way."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2012_14332_gb300.sharding import shard, step_range


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_shard_partitions_the_range():
    for n in (0, 1, 7, 100, 2**24 + 3):
        for world in (1, 2, 3, 8):
            parts = [shard(11, n, r, world) for r in range(world)]
            assert parts[0][0] == 11
            for (a, ca), (b, _) in zip(parts, parts[1:]):
                assert a + ca == b
            assert sum(c for _, c in parts) == n
            assert max(c for _, c in parts) - min(c for _, c in parts) <= 1
    assert step_range(3, 1, 4, 100) == ((3 * 4 + 1) * 100, 100)
    with pytest.raises(ValueError):
        shard(0, 10, 2, 2)


def _rank_main(rank, world, port, n, queue):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    import oracle
    from paper_2012_14332_gb300.sharding import gather_accepted, shard
    from tests import inputs
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = inputs.workload("region_1e6_T49")
        first, count = shard(500, n, rank, world)
        r = oracle.abc(w["observed"], w["P"], w["eps"], count, w["seed"], first_index=first, capacity=count,
                       n_threads=2)
        res = gather_accepted(r["idx"], r["theta"], r["dist"], r["n_accepted"])
        if rank == 0:
            queue.put(res)
    finally:
        dist.destroy_process_group()


def test_two_rank_union_equals_unsplit_run():
    import oracle
    from tests import inputs
    n, world = 20001, 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, n, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = None
    for _ in range(600):
        try:
            res = q.get(timeout=0.5)
            break
        except Exception:
            if any(p.exitcode not in (None, 0) for p in procs):
                break
    for p in procs:
        p.join(timeout=120)
        if p.is_alive():
            p.kill()
        assert p.exitcode == 0
    assert res is not None
    ix, th, di, total = res
    w = inputs.workload("region_1e6_T49")
    ref = oracle.abc(w["observed"], w["P"], w["eps"], n, w["seed"], first_index=500, capacity=n)
    assert total == ref["n_accepted"] > 0
    assert np.array_equal(ix, ref["idx"]) and np.array_equal(th, ref["theta"]) and np.array_equal(di, ref["dist"])


def _quantile_rank_main(rank, world, port, n, k, queue):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    import oracle
    from paper_2012_14332_gb300.sharding import kth_smallest_global, shard
    from tests import inputs
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = inputs.workload("region_1e6_T49")
        first, count = shard(0, n, rank, world)
        r = oracle.abc(w["observed"], w["P"], 0.0, count, w["seed"], first_index=first, capacity=1, n_threads=2,
                       want_all=True)
        eps = kth_smallest_global(np.sort(r["dist_all"])[:k], k)
        queue.put((rank, eps))
    finally:
        dist.destroy_process_group()


def test_two_rank_quantile_eps_equals_the_unsplit_one():
    """eps as the 0.1 % quantile of the small workload's 65,536 distances
    (k = 66), with the distances split over two ranks: each rank passes its
    own 66 smallest, and both get the k-th smallest of the whole run, the
    workload's eps (written by the oracle over all 65,536)."""
    from tests import inputs
    w = inputs.workload("region_1e6_T49")
    n, k, world = w["n_samples"], 66, 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_quantile_rank_main, args=(r, world, port, n, k, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = {}
    for _ in range(1200):
        try:
            r, e = q.get(timeout=0.5)
            got[r] = e
            if len(got) == world:
                break
        except Exception:
            if any(p.exitcode not in (None, 0) for p in procs):
                break
    for p in procs:
        p.join(timeout=120)
        if p.is_alive():
            p.kill()
        assert p.exitcode == 0
    assert got == {0: w["eps"], 1: w["eps"]}
