"""The sharded job on the GPU: two processes (gloo, both on cuda:0; their
kernels never wait on each other) each compute their stripe range of one
matrix through uf_compute with a device output, rank 0 gathers the parts
(paper_2005_05826_gb300.shard) and the stitched matrix equals a full-range
uf_compute bit for bit.  Stripes are independent subproblems (Abstract;
Table 2's multi-chip runs).  Chunk autotuning is off so that every process
uses the same work units (their floating-point partial sums then agree to
the bit)."""
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [("weighted_normalized", 1.0, "mixed"), ("unweighted", 1.0, "mixed"), ("generalized", 0.5, "fp64")]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist

    import paper_2005_05826_gb300 as uf
    from paper_2005_05826_gb300.shard import gather_and_stitch, stripe_ranges
    from synth import workload
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        uf.uf_set_option("autotune", 0)
        tree_s, table_s = workload("yule50k_n2048")
        tree = uf.Tree(tree_s.parent, tree_s.length)
        table = uf.Table(table_s.indptr, table_s.indices, table_s.data, tree)
        n = table_s.n_samples
        ranges = stripe_ranges(n // 2, world)
        start, stop = ranges[rank]
        res = []
        for method, alpha, precision in CASES:
            part = torch.empty((stop - start) * n, dtype=torch.float64, device="cuda")
            uf.uf_compute(tree, table, method, alpha, precision, start, stop, out=part)
            torch.cuda.synchronize()
            out = gather_and_stitch(dist, n, ranges, part)
            if rank == 0:
                full, _ = uf.uf_compute(tree, table, method, alpha, precision)
                res.append((method, precision, int(np.count_nonzero(out != full)), out.size))
        if rank == 0:
            q.put(res)
    finally:
        dist.destroy_process_group()


def test_two_processes_stitch_the_full_matrix_bitwise():
    from paper_2005_05826_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=600)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    res = q.get(timeout=5)
    assert len(res) == len(CASES)
    for method, precision, mismatched, size in res:
        assert mismatched == 0, f"{method}/{precision}: {mismatched} of {size} values differ"
