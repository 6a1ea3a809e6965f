"""GPU parity of the further Striped UniFrac family members against the FP64
oracle: unweighted unnormalized (the unweighted numerator; on the tensor
cores in mixed precision) and variance-adjusted weighted UniFrac (Chang,
Luan & Sun 2011), unnormalized and normalized, on the CUDA-core stripe
kernels.  All pairs of the 1,024-tip / 64-sample workload, tile-edge sample
counts on random trees with unary nodes and zero-length branches, stripe
ranges, identical samples, and the seeded 10,000-pair subset of the
50,000-tip / 2,048-sample workload, in both precisions."""
import numpy as np
import pytest

import oracle
import paper_2005_05826_gb300 as uf
from synth import Table as STable, pair_subset, table_iid, workload, yule_tree
from tests.gpu_util import VARIANTS, assert_close, condensed_index
from tests.test_oracle_pins import random_small_tree, random_table_for

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRECISIONS = ["fp64", "mixed"]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2005_05826_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def handles(tree_s, table_s):
    tree = uf.Tree(tree_s.parent, tree_s.length)
    return tree, uf.Table(table_s.indptr, table_s.indices, table_s.data, tree)


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("method", VARIANTS)
def test_variants_yule1k_n64_all_pairs(method, precision):
    tree_s, table_s = workload("yule1k_n64")
    tree, table = handles(tree_s, table_s)
    got, rep = uf.uf_compute(tree, table, method, 1.0, precision)
    exp = oracle.condensed(tree_s, table_s, method)
    assert_close(got, exp, method, precision, "variants yule1k_n64")
    assert rep.updates == 2016 * (tree_s.n_nodes - 1)
    if method == "unweighted_unnormalized":
        assert rep.path == 0  # CUDA-core kernels, abs form on every stripe


@pytest.mark.parametrize("n", [2, 3, 4, 5, 7, 8, 31, 32, 33, 63, 64, 65, 127, 128, 129, 257])
def test_variants_tile_edges(n):
    rng = np.random.default_rng(300 + n)
    tree_s = random_small_tree(rng, int(rng.integers(3, 60)), unary=3, zero_len=3)
    table_s = random_table_for(rng, tree_s, n, density=0.3)
    tree, table = handles(tree_s, table_s)
    for method in VARIANTS:
        exp = oracle.condensed(tree_s, table_s, method)
        for precision in PRECISIONS:
            got, _ = uf.uf_compute(tree, table, method, 1.0, precision)
            assert_close(got, exp, method, precision, f"variants n={n}")


@pytest.mark.parametrize("precision", PRECISIONS)
def test_variants_stripe_ranges_and_identical_samples(precision):
    tree_s = yule_tree(300, seed=61)
    counts = table_iid(70, tree_s.n_tips, 0.05, seed=62).dense()
    counts[5] = counts[17]
    counts[33] = counts[17] * 3.0  # proportional counts
    table_s = STable.from_dense(counts)
    tree, table = handles(tree_s, table_s)
    n = table_s.n_samples
    S = n // 2
    for method in VARIANTS:
        full, _ = uf.uf_compute(tree, table, method, 1.0, precision)
        exp = oracle.condensed(tree_s, table_s, method)
        assert_close(full, exp, method, precision, "variants full")
        # exact copies give exactly 0 on every method
        assert full[condensed_index(n, 5, 17)] == 0.0
        if method == "unweighted_unnormalized":  # presence is scale-free
            assert full[condensed_index(n, 17, 33)] == 0.0
        for start, stop in ((0, 7), (7, 20), (20, S)):
            part, _ = uf.uf_compute(tree, table, method, 1.0, precision, start, stop)
            s = np.arange(start, stop)[:, None]
            k = np.arange(n)[None, :]
            j = (k + s + 1) % n
            want = full[condensed_index(n, np.minimum(k, j), np.maximum(k, j))]
            assert_close(part.ravel(), want.ravel(), method, precision, f"variants range [{start}, {stop})")


@pytest.mark.parametrize("method", VARIANTS)
def test_variants_yule50k_n2048_pair_subset(method):
    tree_s, table_s = workload("yule50k_n2048")
    tree, table = handles(tree_s, table_s)
    n = table_s.n_samples
    i, j = pair_subset(n, 10_000, seed=12345)
    idx = condensed_index(n, i, j)
    exp = oracle.pairs(tree_s, table_s, method, 1.0, i, j)[0]
    for precision in PRECISIONS:
        got, rep = uf.uf_compute(tree, table, method, 1.0, precision)
        assert_close(got[idx], exp, method, precision, "variants yule50k_n2048")
        if precision == "fp64":
            assert rep.clamped == 0
