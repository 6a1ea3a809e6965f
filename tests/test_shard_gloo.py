"""Stripe-range sharding over 2 processes (gloo, CPU): each rank computes its
stripe range with the plain striped loop, rank 0 gathers and stitches, and
the result equals the full condensed matrix of the per-pair oracle."""
import os
import socket

import numpy as np
import pytest

from paper_2005_05826_gb300.shard import stitch_condensed, stripe_ranges


def test_stripe_ranges_cover_and_balance():
    for S in (0, 1, 5, 32, 33):
        for world in (1, 2, 3, 8):
            r = stripe_ranges(S, world)
            assert len(r) == world and r[0][0] == 0 and r[-1][1] == S
            assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
            sizes = [b - a for a, b in r]
            assert max(sizes) - min(sizes) <= 1


@pytest.mark.parametrize("world", [1, 2, 3, 5])
@pytest.mark.parametrize("n", [2, 3, 4, 5, 9, 10, 13])
def test_stitch_equals_full_oracle(n, world):
    # every rank count, including ranks whose stripe range is empty (world > S)
    import oracle
    from synth import table_iid, yule_tree
    tree = yule_tree(30, seed=80)
    table = table_iid(n, tree.n_tips, 0.3, seed=81)
    S = n // 2
    ranges = stripe_ranges(S, world)
    parts = [oracle.striped(tree, table, "weighted_normalized", 1.0, a, b)[2] if b > a else np.zeros(0)
             for a, b in ranges]
    got = stitch_condensed(n, ranges, parts)
    exp = oracle.condensed(tree, table, "weighted_normalized", 1.0)
    np.testing.assert_allclose(got, exp, rtol=1e-13, atol=1e-15)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, n, q, as_tensor=False):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    import oracle
    from paper_2005_05826_gb300.shard import gather_and_stitch
    from synth import table_iid, yule_tree
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        tree = yule_tree(40, seed=82)
        table = table_iid(n, tree.n_tips, 0.25, seed=83)
        ranges = stripe_ranges(n // 2, world)
        a, b = ranges[rank]
        part = oracle.striped(tree, table, "unweighted", 1.0, a, b)[2] if b > a else np.zeros(0)
        if as_tensor:  # a torch tensor part (as a device output would be), here on the host
            import torch
            part = torch.as_tensor(np.ascontiguousarray(part))
        out = gather_and_stitch(dist, n, ranges, part)
        if rank == 0:
            exp = oracle.condensed(tree, table, "unweighted", 1.0)
            q.put(float(np.max(np.abs(out - exp))))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("n,as_tensor", [(11, False), (12, False), (12, True)])
def test_two_rank_gloo_gather(n, as_tensor):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, n, q, as_tensor)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    assert q.get(timeout=5) <= 1e-14


def test_three_rank_gloo_gather_with_an_empty_range():
    # n = 4 has two stripes: the third rank's range is empty and it sends nothing
    import multiprocessing as mp
    assert stripe_ranges(2, 3)[2] == (2, 2)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 3, port, 4, q)) for r in range(3)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    assert q.get(timeout=5) <= 1e-14


def test_job_ranges_fixed_per_rank_then_split():
    from paper_2005_05826_gb300.shard import job_ranges
    assert job_ranges(56500, 8192, 1) == [(0, 8192)]
    assert job_ranges(56500, 8192, 4) == [(0, 8192), (8192, 16384), (16384, 24576), (24576, 32768)]
    # eight ranks would run past the matrix: the whole matrix split evenly
    r = job_ranges(56500, 8192, 8)
    assert r[0][0] == 0 and r[-1][1] == 56500 and len(r) == 8
    assert job_ranges(1024, 0, 2) == [(0, 512), (512, 1024)]
