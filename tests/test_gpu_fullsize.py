"""Parity at the full sizes of the large synthetic workloads, in the launch
configuration bench.py times (sparse rows, stripe regions, overlap, CUDA
graphs), on outputs the FP64 oracle computes one by one:

- EMP-shaped: 300,000-tip Yule tree x 25,000 samples (37.8 M nonzeros), all
  four methods, the seeded 10,000-pair subset (seed 12345): the mixed path on
  the full matrix, the FP64 path on the stripe range [0, 1,024) of 12,500
  (10,000 seeded cells of the range; the whole FP64 matrix takes minutes per
  method);
- 113k-shaped: 500,000-tip Yule tree x 113,000 samples (169 M nonzeros), the
  workload's methods (weighted_normalized and unweighted): 10,000 seeded cells
  of the mixed stripe range [0, 8,192), and 10,000 of the FP64 range [0, 64);
- batched: 64 tables of 200-5,000 samples over one 100,000-tip tree, one
  batched call per method, 60 seeded pairs of every table.

Generating the 113k-shaped workload takes about two minutes of host time."""
import numpy as np
import pytest

import oracle
import paper_2005_05826_gb300 as uf
from synth import pair_subset, workload
from tests.gpu_util import METHODS, assert_close, condensed_index

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2005_05826_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def range_cells(n, start, stop, count, seed):
    """`count` seeded cells of the stripe range [start, stop): their index in the
    stripe-major output and their pair (a, b), a < b."""
    rng = np.random.default_rng(seed)
    cells = np.sort(rng.choice((stop - start) * n, size=count, replace=False))
    s = start + cells // n
    k = cells % n
    j = (k + s + 1) % n
    return cells, np.minimum(k, j), np.maximum(k, j)


def test_emp_shaped_full_size_pair_subset():
    tree_s, table_s = workload("yule300k_n25000")
    tree = uf.Tree(tree_s.parent, tree_s.length)
    table = uf.Table(table_s.indptr, table_s.indices, table_s.data, tree)
    n = table_s.n_samples
    i, j = pair_subset(n, 10_000, seed=12345)
    idx = torch.as_tensor(condensed_index(n, i, j), device="cuda")
    out = torch.empty(n * (n - 1) // 2, dtype=torch.float64, device="cuda")
    start, stop = 0, 1024
    cells, a, b = range_cells(n, start, stop, 10_000, seed=12345)
    cells_d = torch.as_tensor(cells, device="cuda")
    out_r = torch.empty((stop - start) * n, dtype=torch.float64, device="cuda")
    for method in METHODS:
        alpha = 0.5 if method == "generalized" else 1.0
        uf.uf_compute(tree, table, method, alpha, "mixed", out=out)
        torch.cuda.synchronize()
        exp = oracle.pairs(tree_s, table_s, method, alpha, i, j)[0]
        assert_close(out[idx].cpu().numpy(), exp, method, "mixed", "EMP-shaped, full size")
        uf.uf_compute(tree, table, method, alpha, "fp64", start, stop, out=out_r)
        torch.cuda.synchronize()
        exp_r = oracle.pairs(tree_s, table_s, method, alpha, a, b)[0]
        assert_close(out_r[cells_d].cpu().numpy(), exp_r, method, "fp64", "EMP-shaped, stripes [0, 1024)")


def test_113k_shaped_stripe_range_sample():
    tree_s, table_s = workload("yule500k_n113000")
    tree = uf.Tree(tree_s.parent, tree_s.length)
    table = uf.Table(table_s.indptr, table_s.indices, table_s.data, tree)
    n = table_s.n_samples
    for precision, (start, stop) in (("mixed", (0, 8192)), ("fp64", (0, 64))):
        cells, a, b = range_cells(n, start, stop, 10_000, seed=12345)
        cells_d = torch.as_tensor(cells, device="cuda")
        out = torch.empty((stop - start) * n, dtype=torch.float64, device="cuda")
        for method in ("weighted_normalized", "unweighted"):
            _, rep = uf.uf_compute(tree, table, method, 1.0, precision, start, stop, out=out)
            torch.cuda.synchronize()
            if method == "unweighted" and precision == "mixed":
                assert rep.path == 1  # the tensor-core gram, on the tiles of the range
            got = out[cells_d].cpu().numpy()
            exp = oracle.pairs(tree_s, table_s, method, 1.0, a, b)[0]
            assert_close(got, exp, method, precision, f"113k-shaped, stripes [{start}, {stop})")
        del out


def test_batched_64_tables_full_size_pair_subsets():
    # the batched workload in full (64 tables, 200-5,000 samples, one
    # 100,000-tip tree), both of its methods in one batched call each; 60
    # seeded pairs of every table against the oracle
    from synth import batched_workload
    tree_s, tables_s = batched_workload()
    tree = uf.Tree(tree_s.parent, tree_s.length)
    tables = [uf.Table(t.indptr, t.indices, t.data, tree) for t in tables_s]
    for method in ("unweighted", "weighted_normalized"):
        outs, _ = uf.uf_compute_batch(tree, tables, method, 1.0, "mixed")
        for t, (ts, got) in enumerate(zip(tables_s, outs)):
            n = ts.n_samples
            i, j = pair_subset(n, 60, seed=12345 + t)
            exp = oracle.pairs(tree_s, ts, method, 1.0, i, j)[0]
            assert_close(got[condensed_index(n, i, j)], exp, method, "mixed", f"batched table {t}")
