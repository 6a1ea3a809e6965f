"""Stripe-range sharding across ranks (host logic, no data-path collective
until the final gather).

Stripes are independent subproblems (the paper's Abstract and Sec. 3, where
stripe ranges ran as separate jobs on many chips).  With G ranks, rank r
computes the contiguous stripe range ``stripe_ranges(S, G)[r]`` through
``uf_compute(..., stripe_start, stripe_stop)`` and the stripe-major parts are
gathered once and stitched into the condensed matrix.  Equal stripe counts
give equal work: every stripe has n cells per branch.
"""
from __future__ import annotations

import numpy as np

__all__ = ["stripe_ranges", "job_ranges", "stitch_condensed", "gather_parts", "gather_and_stitch"]


def stripe_ranges(n_stripes: int, world: int):
    """Contiguous [start, stop) stripe ranges, sizes differing by at most one."""
    if world < 1:
        raise ValueError("world must be >= 1")
    base, extra = divmod(n_stripes, world)
    out, start = [], 0
    for r in range(world):
        stop = start + base + (1 if r < extra else 0)
        out.append((start, stop))
        start = stop
    return out


def job_ranges(n_stripes: int, per_rank: int, world: int):
    """The stripe ranges of a job that gives every rank ``per_rank`` stripes
    of one matrix: rank r takes [r * per_rank, (r + 1) * per_rank) while
    world * per_rank stripes exist (per-rank work fixed as ranks are added);
    once they would run past the matrix, the whole matrix [0, n_stripes) is
    split evenly instead."""
    if per_rank <= 0 or world * per_rank >= n_stripes:
        return stripe_ranges(n_stripes, world)
    return [(r * per_rank, (r + 1) * per_rank) for r in range(world)]


def stitch_condensed(n: int, ranges, parts) -> np.ndarray:
    """Condensed distances (pair (i, j), i < j, at n*i - i*(i+1)/2 + j-i-1)
    from stripe-major parts: parts[r][s - start][k] is the pair
    (k, (k + s + 1) mod n)."""
    out = np.empty(n * (n - 1) // 2, dtype=np.float64)
    k = np.arange(n, dtype=np.int64)
    for (start, stop), part in zip(ranges, parts):
        part = np.asarray(part).reshape(stop - start, n)
        for s in range(start, stop):
            j = (k + s + 1) % n
            keep = slice(None) if 2 * (s + 1) != n else slice(0, n // 2)  # duplicate half stripe
            i_, j_ = np.minimum(k, j)[keep], np.maximum(k, j)[keep]
            out[n * i_ - i_ * (i_ + 1) // 2 + (j_ - i_ - 1)] = part[s - start][keep]
    return out


def gather_parts(dist, n: int, ranges, local_part):
    """All ranks send their stripe-major part to rank 0 (point-to-point: the
    one collective of a sharded run); rank 0 returns the list of parts as
    tensors (on its GPU under NCCL, on the host under gloo), the others None.

    local_part is a numpy array or a torch tensor (a device output of
    uf_compute may be passed as it is; its dtype is kept, float32 or
    float64).  With the NCCL backend the parts travel as CUDA tensors on the
    current device; with gloo, as host tensors."""
    import torch
    rank, world = dist.get_rank(), dist.get_world_size()
    nccl = str(dist.get_backend()).lower() == "nccl"
    dev = torch.device("cuda", torch.cuda.current_device()) if nccl else torch.device("cpu")
    if isinstance(local_part, torch.Tensor):
        dtype = local_part.dtype if local_part.dtype in (torch.float32, torch.float64) else torch.float64
        t = local_part.reshape(-1).to(device=dev, dtype=dtype)
    else:
        t = torch.as_tensor(np.ascontiguousarray(local_part, dtype=np.float64).ravel()).to(dev)
    sizes = [(stop - start) * n for start, stop in ranges]
    if t.numel() != sizes[rank]:
        raise ValueError(f"rank {rank}: part has {t.numel()} values, its stripe range {sizes[rank]}")
    if rank == 0:
        bufs = [torch.empty(sz, dtype=t.dtype, device=dev) for sz in sizes]
        bufs[0].copy_(t)
        for r in range(1, world):
            if sizes[r]:
                dist.recv(bufs[r], src=r)
        return bufs
    if sizes[rank]:
        dist.send(t, dst=0)
    return None


def gather_and_stitch(dist, n: int, ranges, local_part) -> np.ndarray | None:
    """All ranks send their stripe-major part; rank 0 returns the stitched
    condensed matrix of the whole stripe set (ranges covering [0, S)), the
    others None."""
    bufs = gather_parts(dist, n, ranges, local_part)
    if bufs is None:
        return None
    return stitch_condensed(n, ranges, [b.double().cpu().numpy() for b in bufs])
