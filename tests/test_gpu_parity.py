"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

FP64 path within 1e-10 relative, mixed path within 1e-5 absolute (scaled by
max(1, d) for weighted_unnormalized), element by element on seeded inputs:
all pairs of the 1,024-tip / 64-sample workload, tile-edge sample counts,
unary nodes and zero-length branches, stripe ranges, identical samples,
multi-block plans, device / FP32 outputs, and a seeded 10,000-pair subset
of the 50,000-tip / 2,048-sample workload.
"""
import numpy as np
import pytest

import oracle
import paper_2005_05826_gb300 as uf
from synth import Table as STable, pair_subset, table_iid, workload, yule_tree
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


def handles(tree_s, table_s):
    tree = uf.Tree(tree_s.parent, tree_s.length)
    table = uf.Table(table_s.indptr, table_s.indices, table_s.data, tree)
    return tree, table


def alpha_for(method):
    return 0.5 if method == "generalized" else 1.0


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("method", METHODS)
def test_yule1k_n64_all_pairs(method, precision):
    tree_s, table_s = workload("yule1k_n64")
    tree, table = handles(tree_s, table_s)
    a = alpha_for(method)
    got, rep = uf.uf_compute(tree, table, method, a, precision)
    exp = oracle.condensed(tree_s, table_s, method, a)
    assert got.shape == exp.shape
    assert_close(got, exp, method, precision, "yule1k_n64")
    assert rep.updates == 2016 * (tree_s.n_nodes - 1)


@pytest.mark.parametrize("n", [2, 3, 4, 5, 7, 8, 31, 32, 33, 63, 64, 65, 127, 128, 129, 257])
def test_tile_edges_all_methods(n):
    rng = np.random.default_rng(100 + n)
    tree_s = random_small_tree(rng, int(rng.integers(3, 60)), unary=3, zero_len=3)
    table_s = random_table_for(rng, tree_s, n, density=0.3)
    tree, table = handles(tree_s, table_s)
    for method in METHODS:
        for alpha in ([0.0, 0.5, 0.75, 1.0] if method == "generalized" else [1.0]):
            exp = oracle.condensed(tree_s, table_s, method, alpha)
            for precision in PRECISIONS:
                got, _ = uf.uf_compute(tree, table, method, alpha, precision)
                assert_close(got, exp, method, precision, f"n={n} alpha={alpha}")


@pytest.mark.parametrize("precision", PRECISIONS)
def test_identical_samples_are_exactly_zero(precision):
    tree_s = yule_tree(300, seed=31)
    t = table_iid(40, tree_s.n_tips, 0.05, seed=32)
    counts = t.dense()
    counts[5] = counts[17]
    counts[33] = counts[17] * 3.0  # proportional counts: same proportions
    table_s = STable.from_dense(counts)
    tree, table = handles(tree_s, table_s)
    n = table_s.n_samples
    # exact copies give 0 on both paths; proportional counts give the same
    # FP64 proportions (correctly rounded quotients), hence 0 on the FP64 path
    pairs = [(5, 17)] + ([(17, 33), (5, 33)] if precision == "fp64" else [])
    for method in METHODS:
        got, _ = uf.uf_compute(tree, table, method, alpha_for(method), precision)
        for i, j in pairs:
            d = got[condensed_index(n, i, j)]
            assert d == 0.0, (method, i, j, d)


@pytest.mark.parametrize("n", [9, 64, 300])
def test_stripe_ranges(n):
    tree_s = yule_tree(200, seed=40 + n)
    table_s = table_iid(n, tree_s.n_tips, 0.1, seed=41 + n)
    tree, table = handles(tree_s, table_s)
    S = uf.uf_stripe_count(n)
    cuts = sorted({0, 1, S // 3, S // 2 + 1, S - 1, S})
    for method in ["unweighted", "weighted_normalized", "generalized"]:
        _, _, exp_striped, _ = oracle.striped(tree_s, table_s, method, 0.5, 0, S)
        for precision in PRECISIONS:
            parts = []
            for a, b in zip(cuts[:-1], cuts[1:]):
                if a == b:
                    continue
                got, _ = uf.uf_compute(tree, table, method, 0.5, precision, a, b)
                assert got.shape == (b - a, n)
                assert_close(got.ravel(), exp_striped[a:b].ravel(), method, precision, f"range [{a},{b})")
                parts.append(got)
            whole = np.vstack(parts)
            # stripes are independent: the pieces equal a run of everything
            alln, _ = uf.uf_compute(tree, table, method, 0.5, precision, 0, S - 1)
            np.testing.assert_array_equal(whole[: S - 1], alln)


def test_device_and_fp32_outputs():
    tree_s, table_s = workload("yule1k_n64")
    tree, table = handles(tree_s, table_s)
    n = table_s.n_samples
    host, _ = uf.uf_compute(tree, table, "weighted_normalized", 1.0, "mixed")
    dev = torch.empty(n * (n - 1) // 2, dtype=torch.float64, device="cuda")
    uf.uf_compute(tree, table, "weighted_normalized", 1.0, "mixed", out=dev)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(dev.cpu().numpy(), host)
    f32, _ = uf.uf_compute(tree, table, "weighted_normalized", 1.0, "mixed", out_fp32=True)
    assert f32.dtype == np.float32
    np.testing.assert_array_equal(f32, host.astype(np.float32))


@pytest.mark.parametrize("method", METHODS)
def test_batch_of_uneven_tables(method):
    # one embedding pass and one accumulate launch serve every table
    tree_s = yule_tree(500, seed=50)
    sizes = (7, 1, 64, 130, 2, 257, 33)
    tables_s = [table_iid(n, tree_s.n_tips, 0.05, seed=51 + n) for n in sizes]
    tree = uf.Tree(tree_s.parent, tree_s.length)
    tables = [uf.Table(t.indptr, t.indices, t.data, tree) for t in tables_s]
    a = alpha_for(method)
    for precision in PRECISIONS:
        outs, reps = uf.uf_compute_batch(tree, tables, method, a, precision)
        for t_s, o, rep in zip(tables_s, outs, reps):
            if t_s.n_samples < 2:
                assert o.size == 0
                continue
            exp = oracle.condensed(tree_s, t_s, method, a)
            assert_close(o, exp, method, precision, f"batch n={t_s.n_samples}")
            assert rep.updates == t_s.n_samples * (t_s.n_samples - 1) // 2 * (tree_s.n_nodes - 1)


@pytest.mark.parametrize("method", METHODS)
def test_yule50k_n2048_pair_subset(method):
    tree_s, table_s = workload("yule50k_n2048")
    tree, table = handles(tree_s, table_s)
    n = table_s.n_samples
    i, j = pair_subset(n, 10_000, seed=12345)
    a = alpha_for(method)
    exp = oracle.pairs(tree_s, table_s, method, a, i, j)[0]
    for precision in PRECISIONS:
        got, _ = uf.uf_compute(tree, table, method, a, precision)
        assert_close(got[condensed_index(n, i, j)], exp, method, precision, "yule50k_n2048")


@pytest.mark.parametrize("tensor", [0, 1])
def test_multi_block_plans_and_both_unweighted_paths(tensor):
    # small branch blocks exercise count-slot reuse across blocks
    tree_s = yule_tree(400, seed=60)
    table_s = table_iid(150, tree_s.n_tips, 0.05, seed=61)
    tree, table = handles(tree_s, table_s)
    uf.uf_set_option("tensor_path", tensor)
    try:
        for block in (0, 97, 300):
            uf.uf_set_option("branch_block", block)
            for method in METHODS:
                a = alpha_for(method)
                exp = oracle.condensed(tree_s, table_s, method, a)
                for precision in PRECISIONS:
                    got, rep = uf.uf_compute(tree, table, method, a, precision)
                    assert_close(got, exp, method, precision, f"block={block} tensor={tensor}")
                    if block:
                        assert rep.n_blocks == -(-(tree_s.n_nodes - 1) // block)
                    if method == "unweighted" and precision == "mixed":
                        assert rep.path == tensor
    finally:
        uf.uf_set_option("branch_block", 0)
        uf.uf_set_option("tensor_path", 1)


def test_tensor_path_large_n_pair_subset():
    # several 128 x 256 tiles, several K chunks, ragged n
    tree_s = yule_tree(9000, seed=62)
    table_s = table_iid(1000, tree_s.n_tips, 0.02, seed=63)
    tree, table = handles(tree_s, table_s)
    n = table_s.n_samples
    i, j = pair_subset(n, 4000, seed=12345)
    exp = oracle.pairs(tree_s, table_s, "unweighted", 1.0, i, j)[0]
    got, rep = uf.uf_compute(tree, table, "unweighted", 1.0, "mixed")
    assert rep.path == 1
    assert_close(got[condensed_index(n, i, j)], exp, "unweighted", "mixed", "tensor path")


def test_graph_and_plain_launches_agree():
    tree_s = yule_tree(600, seed=90)
    tables_s = [table_iid(n, tree_s.n_tips, 0.05, seed=91 + n) for n in (40, 150)]
    tree = uf.Tree(tree_s.parent, tree_s.length)
    tables = [uf.Table(t.indptr, t.indices, t.data, tree) for t in tables_s]
    try:
        for method in ["unweighted", "weighted_normalized", "generalized"]:
            for precision in PRECISIONS:
                res = {}
                for graph in (0, 1):
                    uf.uf_set_option("graph", graph)
                    outs, reps = uf.uf_compute_batch(tree, tables, method, 0.5, precision)
                    assert all(r.graph == graph for r in reps)
                    res[graph] = outs
                for a, b in zip(res[0], res[1]):
                    np.testing.assert_array_equal(a, b)
    finally:
        uf.uf_set_option("graph", 1)


def test_queued_device_output_calls_match_synchronous_ones():
    # device outputs on a non-default stream: each call returns once its work
    # is queued (its graph is retired by a later call); 40 calls back to back
    # pass the 32 graphs kept in flight, and every result equals the same
    # call made synchronously with a host output, bit for bit
    tree_s = yule_tree(800, seed=95)
    table_s = table_iid(160, tree_s.n_tips, 0.05, seed=96)
    tree = uf.Tree(tree_s.parent, tree_s.length)
    table = uf.Table(table_s.indptr, table_s.indices, table_s.data, tree)
    n = table_s.n_samples
    cases = [(m, 0.5 if m == "generalized" else 1.0, p) for m in METHODS for p in PRECISIONS]
    expect = {c: uf.uf_compute(tree, table, c[0], c[1], c[2])[0] for c in cases}
    outs = [torch.empty(n * (n - 1) // 2, dtype=torch.float64, device="cuda") for _ in range(40)]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for i, o in enumerate(outs):
            m, a, p = cases[i % len(cases)]
            uf.uf_compute(tree, table, m, a, p, out=o)
    s.synchronize()
    for i, o in enumerate(outs):
        np.testing.assert_array_equal(o.cpu().numpy(), expect[cases[i % len(cases)]])


def test_autotuned_chunk_sizes():
    tree_s = yule_tree(3000, seed=92)
    table_s = table_iid(200, tree_s.n_tips, 0.03, seed=93)
    tree, table = handles(tree_s, table_s)
    exp = oracle.condensed(tree_s, table_s, "weighted_normalized", 1.0)
    try:
        uf.uf_set_option("autotune", 2)  # forget earlier choices: this call tunes
        got, rep = uf.uf_compute(tree, table, "weighted_normalized", 1.0, "mixed")
        assert rep.chunk_rows in (1024, 2048, 4096, 8192)
        assert_close(got, exp, "weighted_normalized", "mixed", "tuning call")
        got2, rep2 = uf.uf_compute(tree, table, "weighted_normalized", 1.0, "mixed")
        assert rep2.chunk_rows == rep.chunk_rows
        np.testing.assert_array_equal(got, got2)
        uf.uf_set_option("autotune", 0)
        got3, rep3 = uf.uf_compute(tree, table, "weighted_normalized", 1.0, "mixed")
        assert rep3.chunk_rows == 2048
        assert_close(got3, exp, "weighted_normalized", "mixed", "fixed chunk")
    finally:
        uf.uf_set_option("autotune", 1)


@pytest.mark.parametrize("factor", [1e-8, 1.0, 1e16])
def test_generalized_length_scales(factor):
    # uniformly scaled lengths leave normalized distances unchanged; tiny and
    # huge lengths exercise the FP32 embedding floor and the fixed-point scale
    tree_s = yule_tree(800, seed=95)
    tree_s = type(tree_s)(tree_s.parent, tree_s.length * factor)
    table_s = table_iid(150, tree_s.n_tips, 0.05, seed=96)
    tree, table = handles(tree_s, table_s)
    for alpha in (0.5, 0.25):
        exp = oracle.condensed(tree_s, table_s, "generalized", alpha)
        for sparse in (0, 1):
            uf.uf_set_option("sparse", sparse)
            try:
                for precision in PRECISIONS:
                    got, _ = uf.uf_compute(tree, table, "generalized", alpha, precision)
                    assert_close(got, exp, "generalized", precision, f"x{factor} alpha={alpha} sparse={sparse}")
            finally:
                uf.uf_set_option("sparse", 1)


def test_concurrent_calls_from_threads():
    # each host thread captures its call on its own private stream; results
    # equal those of one thread bit for bit
    import threading
    tree_s = yule_tree(2000, seed=97)
    table_s = table_iid(300, tree_s.n_tips, 0.03, seed=98)
    tree, table = handles(tree_s, table_s)
    jobs = [(m, 0.5 if m == "generalized" else 1.0, p) for m in METHODS for p in PRECISIONS]
    ref = {j: uf.uf_compute(tree, table, j[0], j[1], j[2])[0] for j in jobs}
    got, errors = {}, []

    def work(sub):
        try:
            for _ in range(2):
                for j in sub:
                    got[j] = uf.uf_compute(tree, table, j[0], j[1], j[2])[0]
        except Exception as e:  # reported below
            errors.append(e)

    threads = [threading.Thread(target=work, args=(jobs[k::4],)) for k in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for j in jobs:
        np.testing.assert_array_equal(got[j], ref[j])


def test_degenerate_inputs():
    # one sample: no pairs, an empty result and UF_OK
    tree_s = yule_tree(30, seed=120)
    one = STable.from_dense(np.ones((1, tree_s.n_tips)))
    tree = uf.Tree(tree_s.parent, tree_s.length)
    t1 = uf.Table(one.indptr, one.indices, one.data, tree)
    for method in METHODS:
        for precision in PRECISIONS:
            got, _ = uf.uf_compute(tree, t1, method, 0.5, precision)
            assert got.size == 0
    # a single tip under the root: every sample is the same, every distance 0
    parent, length = np.array([1, -1]), np.array([0.7, 0.0])
    single = uf.Tree(parent, length)
    rng = np.random.default_rng(121)
    tab_s = STable.from_dense(rng.integers(1, 9, size=(7, 1)).astype(np.float64))
    t7 = uf.Table(tab_s.indptr, tab_s.indices, tab_s.data, single)
    for method in METHODS:
        for precision in PRECISIONS:
            got, _ = uf.uf_compute(single, t7, method, 0.5, precision)
            np.testing.assert_array_equal(got, np.zeros(21))
    # every branch length zero: den = 0 everywhere, so every distance is 0
    zero_s = yule_tree(40, seed=122)
    zero_s.length[:] = 0.0
    ztab = table_iid(12, zero_s.n_tips, 0.3, seed=123)
    zt = uf.Tree(zero_s.parent, zero_s.length)
    ztable = uf.Table(ztab.indptr, ztab.indices, ztab.data, zt)
    for method in METHODS:
        exp = oracle.condensed(zero_s, ztab, method, 0.5)
        assert not exp.any()
        for precision in PRECISIONS:
            got, _ = uf.uf_compute(zt, ztable, method, 0.5, precision)
            np.testing.assert_array_equal(got, exp)
