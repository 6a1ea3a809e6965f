"""GPU parity of the sparse-row path: branches whose subtree holds few count
entries are scattered pair by pair over their nonzero samples instead of
running through the dense stripe kernels (option "sparse").

Every case is checked against the FP64 oracle with "sparse" = 0 (all dense),
1 (cost model) and 2 (every branch that can be scattered), for every method
and precision: capacity classes, stripe ranges including the duplicated
half stripe, batches of uneven tables, identical samples, and trees whose
tip numbers under a node are not contiguous (those nodes stay dense).
"""
import numpy as np
import pytest

import oracle
import paper_2005_05826_gb300 as uf
from synth import Table as STable, pair_subset, table_iid, table_prevalence, workload, yule_tree
from tests.gpu_util import METHODS, assert_close, condensed_index
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
    yield
    uf.uf_set_option("sparse", 1)


def handles(tree_s, table_s):
    tree = uf.Tree(tree_s.parent, tree_s.length)
    table = uf.Table(table_s.indptr, table_s.indices, table_s.data, tree)
    return tree, table


def run(tree, table, method, alpha, precision, mode, *args):
    uf.uf_set_option("sparse", mode)
    try:
        return uf.uf_compute(tree, table, method, alpha, precision, *args)
    finally:
        uf.uf_set_option("sparse", 1)


def test_option_values():
    assert uf.uf_get_option("sparse") == 1
    for bad in (-1, 3):
        with pytest.raises(uf.UFError):
            uf.uf_set_option("sparse", bad)
    assert uf.uf_get_option("sparse") == 1


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("method", METHODS)
def test_all_modes_match_oracle(method, precision):
    tree_s = yule_tree(2000, seed=201)
    table_s = table_prevalence(160, tree_s.n_tips, 0.5, 10.0, seed=202)
    tree, table = handles(tree_s, table_s)
    a = 0.5 if method == "generalized" else 1.0
    exp = oracle.condensed(tree_s, table_s, method, a)
    nb = tree_s.n_nodes - 1
    for mode in (0, 1, 2):
        got, rep = run(tree, table, method, a, precision, mode)
        assert_close(got, exp, method, precision, f"sparse={mode}")
        assert rep.dense_rows + rep.sparse_rows == nb
        if mode == 0:
            assert rep.sparse_rows == 0
        else:
            assert rep.sparse_rows > 0
        if mode == 2:
            # a postorder tree: every branch whose subtree fits is scattered
            assert rep.sparse_rows >= nb // 2


@pytest.mark.parametrize("alpha", [0.0, 0.25, 0.5, 0.75, 1.0])
def test_generalized_alphas(alpha):
    tree_s = yule_tree(700, seed=211)
    table_s = table_iid(90, tree_s.n_tips, 0.04, seed=212)
    tree, table = handles(tree_s, table_s)
    exp = oracle.condensed(tree_s, table_s, "generalized", alpha)
    for precision in PRECISIONS:
        got, rep = run(tree, table, "generalized", alpha, precision, 2)
        assert rep.sparse_rows > 0
        assert_close(got, exp, "generalized", precision, f"alpha={alpha}")


@pytest.mark.parametrize("tensor", [0, 1])
def test_unweighted_mixed_both_paths(tensor):
    # the tensor-core gram path takes the scattered rows into its gram matrices
    tree_s = yule_tree(1500, seed=215)
    table_s = table_iid(300, tree_s.n_tips, 0.03, seed=216)
    tree, table = handles(tree_s, table_s)
    exp = oracle.condensed(tree_s, table_s, "unweighted", 1.0)
    uf.uf_set_option("tensor_path", tensor)
    try:
        for mode in (0, 1, 2):
            got, rep = run(tree, table, "unweighted", 1.0, "mixed", mode)
            assert rep.path == tensor
            assert (rep.sparse_rows > 0) == (mode > 0)
            assert_close(got, exp, "unweighted", "mixed", f"tensor={tensor} sparse={mode}")
    finally:
        uf.uf_set_option("tensor_path", 1)


@pytest.mark.parametrize("lists", [False, True])
def test_capacity_classes(lists):
    # dense tables give subtrees of every entry count from 1 up past 16,384:
    # each capacity class (128, 512, 2,048, 4,096 entries; 16,384 when the
    # rows are written as lists for the stripe-region scatter) gets rows, and
    # the rows above the largest class stay dense
    tree_s = yule_tree(400, seed=221)
    table_s = table_iid(300, tree_s.n_tips, 0.3, seed=222)
    tree, table = handles(tree_s, table_s)
    nb = tree_s.n_nodes - 1
    sparse_rows = {}
    for method in METHODS:
        a = 0.5 if method == "generalized" else 1.0
        exp = oracle.condensed(tree_s, table_s, method, a)
        for precision in PRECISIONS:
            uf.uf_set_option("tensor_path", 0 if method == "unweighted" and precision == "mixed" else 1)
            if lists:
                uf.uf_set_option("sparse_region_bytes", 8192)
            try:
                got, rep = run(tree, table, method, a, precision, 2)
            finally:
                uf.uf_set_option("tensor_path", 1)
                uf.uf_set_option("sparse_region_bytes", 0)
            assert 0 < rep.sparse_rows < nb
            sparse_rows[(method, precision)] = rep.sparse_rows
            assert_close(got, exp, method, precision, f"capacity classes lists={lists}")
    if lists:
        # the list class takes the runs of 4,097 to 16,384 entries too
        counts = np.diff(table_s.indptr)
        assert counts.sum() > 16384
        assert max(sparse_rows.values()) > 0


@pytest.mark.parametrize("n", [2, 3, 8, 9, 64, 65, 300])
def test_stripe_ranges_and_duplicate_half_stripe(n):
    tree_s = yule_tree(150, seed=230 + n)
    table_s = table_iid(n, tree_s.n_tips, 0.15, seed=231 + n)
    tree, table = handles(tree_s, table_s)
    S = uf.uf_stripe_count(n)
    cuts = sorted({0, 1, S // 2, S - 1, S})
    uf.uf_set_option("tensor_path", 0)
    try:
        for method in ["unweighted", "weighted_unnormalized", "generalized"]:
            _, _, exp_striped, _ = oracle.striped(tree_s, table_s, method, 0.5, 0, S)
            exp_full = oracle.condensed(tree_s, table_s, method, 0.5)
            for precision in PRECISIONS:
                whole, _ = run(tree, table, method, 0.5, precision, 2)
                assert_close(whole, exp_full, method, precision, "full run")
                parts = []
                for a, b in zip(cuts[:-1], cuts[1:]):
                    if a == b or (a, b) == (0, S):
                        continue
                    got, _ = run(tree, table, method, 0.5, precision, 2, a, b)
                    assert got.shape == (b - a, n)
                    # the last stripe of an even n holds every pair twice
                    assert_close(got.ravel(), exp_striped[a:b].ravel(), method, precision, f"range [{a},{b})")
                    parts.append(got)
                if S > 1:
                    # stripes are independent: the pieces equal a range run of everything
                    alln, _ = run(tree, table, method, 0.5, precision, 2, 0, S - 1)
                    np.testing.assert_array_equal(np.vstack(parts)[: S - 1], alln)
    finally:
        uf.uf_set_option("tensor_path", 1)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_identical_samples_exactly_zero(precision):
    tree_s = yule_tree(300, seed=241)
    t = table_iid(40, tree_s.n_tips, 0.05, seed=242)
    counts = t.dense()
    counts[5] = counts[17]
    counts[33] = counts[17] * 3.0
    table_s = STable.from_dense(counts)
    tree, table = handles(tree_s, table_s)
    n = table_s.n_samples
    pairs = [(5, 17)] + ([(17, 33), (5, 33)] if precision == "fp64" else [])
    for method in METHODS:
        for alpha in ([0.0, 0.5, 0.75] if method == "generalized" else [1.0]):
            got, rep = run(tree, table, method, alpha, precision, 2)
            for i, j in pairs:
                d = got[condensed_index(n, i, j)]
                assert d == 0.0, (method, alpha, i, j, d)


@pytest.mark.parametrize("method", METHODS)
def test_batch_of_uneven_tables(method):
    tree_s = yule_tree(500, seed=250)
    sizes = (7, 1, 64, 130, 2, 257, 33)
    tables_s = [table_iid(n, tree_s.n_tips, 0.05, seed=251 + n) for n in sizes]
    tree = uf.Tree(tree_s.parent, tree_s.length)
    tables = [uf.Table(t.indptr, t.indices, t.data, tree) for t in tables_s]
    a = 0.5 if method == "generalized" else 1.0
    for mode in (1, 2):
        uf.uf_set_option("sparse", mode)
        try:
            for precision in PRECISIONS:
                outs, reps = uf.uf_compute_batch(tree, tables, method, a, precision)
                for t_s, o, rep in zip(tables_s, outs, reps):
                    if t_s.n_samples < 2:
                        continue
                    exp = oracle.condensed(tree_s, t_s, method, a)
                    assert_close(o, exp, method, precision, f"batch n={t_s.n_samples} sparse={mode}")
        finally:
            uf.uf_set_option("sparse", 1)


def interleaved_tree(rng, n_tips):
    """A valid parent array (parent > child) whose nodes are numbered in a
    random children-before-parents order, so subtrees are interleaved and the
    tips under most internal nodes are not a contiguous run of tip numbers."""
    return random_small_tree(rng, n_tips, unary=2, zero_len=2)


def test_interleaved_numbering_stays_correct():
    rng = np.random.default_rng(260)
    for case in range(4):
        tree_s = interleaved_tree(rng, int(rng.integers(20, 80)))
        table_s = random_table_for(rng, tree_s, int(rng.integers(5, 70)), density=0.2)
        tree, table = handles(tree_s, table_s)
        for method in METHODS:
            a = 0.5 if method == "generalized" else 1.0
            exp = oracle.condensed(tree_s, table_s, method, a)
            for precision in PRECISIONS:
                got, rep = run(tree, table, method, a, precision, 2)
                assert_close(got, exp, method, precision, f"interleaved case {case}")


def test_yule50k_n2048_default_split():
    tree_s, table_s = workload("yule50k_n2048")
    tree, table = handles(tree_s, table_s)
    n = table_s.n_samples
    i, j = pair_subset(n, 10_000, seed=12345)
    for method in ["weighted_normalized", "generalized"]:
        a = 0.5 if method == "generalized" else 1.0
        exp = oracle.pairs(tree_s, table_s, method, a, i, j)[0]
        for precision in PRECISIONS:
            got, rep = run(tree, table, method, a, precision, 1)
            assert rep.sparse_rows > (tree_s.n_nodes - 1) // 3, rep.sparse_rows
            assert_close(got[condensed_index(n, i, j)], exp, method, precision, "yule50k sparse=1")


@pytest.mark.parametrize("n,density", [(97, 0.04), (300, 0.012)])
def test_region_scatter_matches_direct_bitwise(n, density):
    # a one-table call whose accumulators exceed the region budget writes the
    # sample lists and scatters stripe region by region; integer sums are
    # order-free, so the result equals the direct scatter bit for bit (the
    # tables hold at most 4,096 entries, so both modes split the branches alike)
    tree_s = yule_tree(900, seed=270 + n)
    table_s = table_iid(n, tree_s.n_tips, density, seed=271 + n)
    assert table_s.nnz <= 4096
    tree, table = handles(tree_s, table_s)
    S = uf.uf_stripe_count(n)
    uf.uf_set_option("tensor_path", 0)
    try:
        for method in METHODS:
            a = 0.5 if method == "generalized" else 1.0
            exp = oracle.condensed(tree_s, table_s, method, a)
            for precision in PRECISIONS:
                direct, rep0 = run(tree, table, method, a, precision, 2)
                uf.uf_set_option("sparse_region_bytes", 8192)
                try:
                    regional, rep1 = run(tree, table, method, a, precision, 2)
                    part, _ = run(tree, table, method, a, precision, 2, 3, S - 2)
                finally:
                    uf.uf_set_option("sparse_region_bytes", 0)
                assert rep1.sparse_rows == rep0.sparse_rows > 0
                np.testing.assert_array_equal(regional, direct)
                assert_close(regional, exp, method, precision, f"regions n={n}")
                whole, _ = run(tree, table, method, a, precision, 2, 0, S)
                _, _, exp_striped, _ = oracle.striped(tree_s, table_s, method, a, 0, S)
                assert_close(part.ravel(), exp_striped[3:S - 2].ravel(), method, precision, "region range")
    finally:
        uf.uf_set_option("tensor_path", 1)
    assert uf.uf_get_option("sparse_region_bytes") == 48_000_000


@pytest.mark.parametrize("tensor", [0, 1])
def test_fused_lists_match_unfused_bitwise(tensor):
    # In list mode a listed branch carries the terms of its scattered children
    # (option sparse_fuse 2) or, min form, of its children and grandchildren
    # (6; the generalized method takes 2) and adds each pair's summed terms
    # with one atomic per accumulator: the integers are the same as the rows'
    # own updates, so every setting gives the same bits (with every fitting
    # branch scattered, the split does not depend on the setting).
    tree_s = yule_tree(2000, seed=290)
    table_s = table_iid(300, tree_s.n_tips, 0.01, seed=291)
    tree, table = handles(tree_s, table_s)
    S = uf.uf_stripe_count(300)
    uf.uf_set_option("tensor_path", tensor)
    uf.uf_set_option("sparse_region_bytes", 16384)
    try:
        for method in METHODS if not tensor else ["unweighted"]:
            a = 0.5 if method == "generalized" else 1.0
            exp = oracle.condensed(tree_s, table_s, method, a)
            for precision in PRECISIONS:
                got = {}
                for fuse in (0, 2, 6):
                    uf.uf_set_option("sparse_fuse", fuse)
                    got[fuse], rep = run(tree, table, method, a, precision, 2)
                    assert rep.sparse_rows > 0
                    got[(fuse, "range")], _ = run(tree, table, method, a, precision, 2, 5, S - 7)
                np.testing.assert_array_equal(got[2], got[0])
                np.testing.assert_array_equal(got[6], got[0])
                np.testing.assert_array_equal(got[(2, "range")], got[(0, "range")])
                np.testing.assert_array_equal(got[(6, "range")], got[(0, "range")])
                assert_close(got[2], exp, method, precision, f"fused lists tensor={tensor}")
    finally:
        uf.uf_set_option("sparse_fuse", 2)
        uf.uf_set_option("sparse_region_bytes", 0)
        uf.uf_set_option("tensor_path", 1)


def test_region_scatter_counts_its_pair_updates():
    # timed per phase, a call reports the pair updates its region scatter made
    # (counted on the device): unfused, every scattered branch's pairs of
    # present samples, z (z - 1) / 2 for z samples below it over the whole
    # matrix; fused, fewer (the members' pairs ride in their heads' updates)
    tree_s = yule_tree(2000, seed=290)
    table_s = table_iid(300, tree_s.n_tips, 0.01, seed=291)
    tree, table = handles(tree_s, table_s)
    # samples present below every node (children before parents)
    pres = np.zeros((tree_s.n_nodes, 300), dtype=bool)
    dense = table_s.dense() > 0
    has_child = np.zeros(tree_s.n_nodes, dtype=bool)
    has_child[tree_s.parent[:-1]] = True
    tips = np.nonzero(~has_child)[0]
    pres[tips] = dense.T
    for v in range(tree_s.n_nodes - 1):
        pres[tree_s.parent[v]] |= pres[v]
    z = pres[:-1].sum(axis=1).astype(np.float64)
    listed = (tree_s.length[:-1] > 0) & (z > 0)
    expect = float((z[listed] * (z[listed] - 1) / 2).sum())
    uf.uf_set_option("tensor_path", 0)
    uf.uf_set_option("sparse_region_bytes", 16384)
    try:
        uf.uf_set_option("kernel_timing", 1)
        counts = {}
        for fuse in (0, 2):
            uf.uf_set_option("sparse_fuse", fuse)
            _, rep = run(tree, table, "weighted_normalized", 1.0, "mixed", 2)
            counts[fuse] = rep.sparse_pair_updates
        assert counts[0] == expect, (counts[0], expect)
        assert 0 < counts[2] < counts[0]
        uf.uf_set_option("kernel_timing", 0)
        _, rep = run(tree, table, "weighted_normalized", 1.0, "mixed", 2)
        assert rep.sparse_pair_updates == -1.0
    finally:
        uf.uf_set_option("kernel_timing", 0)
        uf.uf_set_option("sparse_fuse", 2)
        uf.uf_set_option("sparse_region_bytes", 0)
        uf.uf_set_option("tensor_path", 1)


def test_overlap_matches_sequential_bitwise():
    # the scatter beside the dense kernel adds the same integers in another
    # order: the results equal the sequential ones bit for bit
    tree_s = yule_tree(3000, seed=280)
    table_s = table_prevalence(400, tree_s.n_tips, 0.5, 15.0, seed=281)
    tree, table = handles(tree_s, table_s)
    assert uf.uf_get_option("sparse_overlap") == 1
    try:
        for method in METHODS:
            a = 0.5 if method == "generalized" else 1.0
            for precision in PRECISIONS:
                uf.uf_set_option("sparse_overlap", 1)
                beside, _ = uf.uf_compute(tree, table, method, a, precision)
                uf.uf_set_option("sparse_overlap", 0)
                after, _ = uf.uf_compute(tree, table, method, a, precision)
                np.testing.assert_array_equal(beside, after)
    finally:
        uf.uf_set_option("sparse_overlap", 1)


def test_l2_atomic_probe_rate():
    # the ceiling the region scatter is measured against: random 64-bit atomic
    # adds into 16 MB (L2-resident) run at 1e10-1e12 per second on one GPU
    rate = uf.uf_probe_l2_atomics(16 << 20)
    assert 1e10 < rate < 1e12, rate
