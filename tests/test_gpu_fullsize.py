"""Parity at the full sizes of the two large synthetic workloads, in the
launch configuration bench.py times (sparse rows, stripe regions, overlap,
CUDA graphs), on outputs the FP64 oracle computes one by one:

- EMP-shaped: 300,000-tip Yule tree x 25,000 samples (37.8 M nonzeros), all
  four methods in mixed precision, 1,000 seeded random pairs;
- 113k-shaped: 500,000-tip Yule tree x 113,000 samples (169 M nonzeros), the
  stripe range [0, 64) for weighted_normalized and unweighted (the
  workload's methods), 500 seeded random cells of the range;
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


def test_emp_shaped_full_size_pair_subset():
    tree_s, table_s = workload("yule300k_n25000")
    tree = uf.Tree(tree_s.parent, tree_s.length)
    table = uf.Table(table_s.indptr, table_s.indices, table_s.data, tree)
    n = table_s.n_samples
    i, j = pair_subset(n, 1000, seed=12345)
    idx = condensed_index(n, i, j)
    out = torch.empty(n * (n - 1) // 2, dtype=torch.float64, device="cuda")
    for method in METHODS:
        alpha = 0.5 if method == "generalized" else 1.0
        uf.uf_compute(tree, table, method, alpha, "mixed", out=out)
        torch.cuda.synchronize()
        got = out[torch.as_tensor(idx, device="cuda")].cpu().numpy()
        exp = oracle.pairs(tree_s, table_s, method, alpha, i, j)[0]
        assert_close(got, exp, method, "mixed", "EMP-shaped, full size")


def test_113k_shaped_stripe_range_sample():
    tree_s, table_s = workload("yule500k_n113000")
    tree = uf.Tree(tree_s.parent, tree_s.length)
    table = uf.Table(table_s.indptr, table_s.indices, table_s.data, tree)
    n = table_s.n_samples
    start, stop = 0, 64
    rng = np.random.default_rng(12345)
    cells = rng.choice((stop - start) * n, size=500, replace=False)
    s = start + cells // n
    k = cells % n
    j = (k + s + 1) % n
    a, b = np.minimum(k, j), np.maximum(k, j)
    out = torch.empty((stop - start) * n, dtype=torch.float64, device="cuda")
    for method in ("weighted_normalized", "unweighted"):
        uf.uf_compute(tree, table, method, 1.0, "mixed", start, stop, out=out)
        torch.cuda.synchronize()
        got = out[torch.as_tensor(cells, device="cuda")].cpu().numpy()
        exp = oracle.pairs(tree_s, table_s, method, 1.0, a, b)[0]
        assert_close(got, exp, method, "mixed", "113k-shaped, stripes [0, 64)")


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
