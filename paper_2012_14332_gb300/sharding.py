"""Sharding of the sample-index range across ranks (Sec. 3.1: the samples are
independent, so any partition of the index range computes the same accept set;
the multi-device runs of Sec. 4.5 are independent replicas gathered on the host).

The counter-based random numbers depend only on (seed, stream, sample index),
so rank r simulating indices [first_r, first_r + count_r) reproduces exactly
the samples an unsplit run would draw there. The one exchange is the gather of
the accepted (idx, theta, dist) sets, done on the host after the compute. With
eps chosen as a distance quantile of the whole run (the k-th smallest), the
ranks first exchange their own k smallest distances (kth_smallest_global).
"""
import numpy as np


def shard(first_index, n_total, rank, world):
    """Contiguous slice of [first_index, first_index + n_total) for `rank` of
    `world`: the first n_total % world ranks get one extra index."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    per, rem = divmod(int(n_total), int(world))
    start = first_index + rank * per + min(rank, rem)
    count = per + (1 if rank < rem else 0)
    return start, count


def step_range(step, rank, world, n_per_rank, first_index=0):
    """Weak scaling: step s of rank r covers its own n_per_rank indices."""
    return first_index + (step * world + rank) * n_per_rank, n_per_rank


def _host(a):
    if hasattr(a, "detach"):
        a = a.detach().cpu().numpy()
    return np.asarray(a)


def local_k_smallest(dist, k):
    """This rank's k smallest distances (a CUDA f64 tensor, e.g. from
    abc_distances), found on the device: its k-th smallest by the radix select,
    then the accept step at that value (ties included). Returns them ascending
    in host memory, min(k, n) values."""
    from . import binding
    n = dist.numel()
    kk = min(int(k), n)
    if kk == 0:
        return np.empty(0, dtype=np.float64)
    eps = binding.abc_kth_smallest(dist, kk)
    cap = kk
    while True:
        try:
            _, di, _, _ = binding.abc_select_below(dist, eps, capacity=cap)
            break
        except binding.AbcError as e:   # more values equal to eps than room
            if e.status != binding.ABC_ERR_CAPACITY:
                raise
            cap *= 2
    return np.sort(di.cpu().numpy())[:kk]


def kth_smallest_global(local_smallest, k, group=None):
    """The k-th smallest distance over all ranks, from each rank's own k
    smallest (any order; fewer if the rank has fewer distances): the global
    k-th smallest is among them. The one exchange is an all-gather of at most
    k values per rank; every rank gets the same eps. Raises ValueError when
    the ranks hold fewer than k distances in all."""
    import torch.distributed as tdist

    mine = np.sort(_host(local_smallest).astype(np.float64).ravel())[:int(k)]
    out = [None] * tdist.get_world_size(group)
    tdist.all_gather_object(out, mine, group=group)
    allv = np.sort(np.concatenate(out))
    if k < 1 or len(allv) < k:
        raise ValueError("%d distances in all, k = %d" % (len(allv), k))
    return float(allv[int(k) - 1])


def gather_accepted(idx, theta, dist, n_accepted, group=None, dst=0):
    """Gather each rank's accepted samples on rank `dst` (host memory).

    idx, theta, dist: this rank's accepted samples (numpy or CPU/CUDA torch
    tensors). Returns (idx, theta, dist, total_accepted) sorted by index on
    `dst`, None elsewhere. Uses torch.distributed (any backend)."""
    import torch.distributed as tdist

    mine = (_host(idx).astype(np.uint64), _host(theta).astype(np.float32).reshape(-1, 8),
            _host(dist).astype(np.float64), int(n_accepted))
    world = tdist.get_world_size(group)
    out = [None] * world if tdist.get_rank(group) == dst else None
    tdist.gather_object(mine, out, dst=dst, group=group)
    if out is None:
        return None
    ix = np.concatenate([o[0] for o in out])
    th = np.concatenate([o[1] for o in out])
    di = np.concatenate([o[2] for o in out])
    order = np.argsort(ix, kind="stable")
    return ix[order], th[order], di[order], sum(o[3] for o in out)
