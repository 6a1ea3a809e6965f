"""Seeded generators: deterministic, valid inputs of the stated shapes."""
import numpy as np

import oracle
from synth import pair_subset, table_iid, table_prevalence, yule_tree


def test_yule_tree_shape_and_order():
    t = yule_tree(257, seed=3)
    assert t.n_nodes == 2 * 257 - 1 and t.n_tips == 257
    assert t.parent[-1] == -1
    assert np.all(t.parent[:-1] > np.arange(t.n_nodes - 1))
    # binary: every internal node has exactly two children
    kids = np.bincount(t.parent[:-1], minlength=t.n_nodes)
    assert set(np.unique(kids)) == {0, 2}
    # postorder: each subtree is a contiguous index range ending at its root
    size = np.ones(t.n_nodes, np.int64)
    first = np.arange(t.n_nodes)
    for v in range(t.n_nodes - 1):
        size[t.parent[v]] += size[v]
        first[t.parent[v]] = min(first[t.parent[v]], first[v])
    assert np.all(first == np.arange(t.n_nodes) - size + 1)
    assert oracle.check_tree(t) == "OK"
    t2 = yule_tree(257, seed=3)
    assert np.array_equal(t.parent, t2.parent) and np.array_equal(t.length, t2.length)
    assert abs(t.length.mean() - 0.1) < 0.02


def test_tables_valid_and_deterministic():
    t = yule_tree(500, seed=1)
    a = table_iid(40, t.n_tips, 0.05, seed=2)
    b = table_iid(40, t.n_tips, 0.05, seed=2)
    assert a.digest() == b.digest()
    assert oracle.check_table(t, a) == "OK"
    c = table_prevalence(300, t.n_tips, 0.5, 20.0, seed=4, heavy=True)
    assert oracle.check_table(t, c) == "OK"
    assert np.all(np.diff(c.indptr) >= 1)
    assert np.all(c.data >= 1) and np.all(c.data == np.round(c.data))


def test_pair_subset_valid():
    n = 97
    i, j = pair_subset(n, 1000, seed=12345)
    assert i.size == 1000 and np.all(i < j) and np.all(j < n)
    assert np.unique(i * n + j).size == 1000
    i2, j2 = pair_subset(n, 1000, seed=12345)
    assert np.array_equal(i, i2) and np.array_equal(j, j2)
    ia, ja = pair_subset(10, 1000)
    ti, tj = np.triu_indices(10, 1)
    assert np.array_equal(ia, ti) and np.array_equal(ja, tj)
