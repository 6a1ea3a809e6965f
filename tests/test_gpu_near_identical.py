"""GPU parity on nearly identical samples: pairs whose distance is tiny.

Each near-identical group is a sample whose counts are scaled to a total of
about 1e4, 1e5 or 1e6, plus three variants of it: one count added to a
feature it already has, one count of a feature it lacks, and one count moved
from one of its features to another.  Their distances are of order
1 / total, so they test what the random tables cannot: that the FP64 path
forms no numerator by cancelling two nearly equal sums (its error must stay
within 1e-10 relative plus the 1e-15 absolute floor), and that no cell's
numerator has to be clamped at zero (report field ``clamped``).

Cases: the 1,024-tip tree with 64 samples (all pairs against the oracle), and
the 50,000-tip tree with its first 1,024 samples of the 2,048-sample table plus
36 near-identical samples (every within-group pair and 2,000 seeded random
pairs against the oracle).
"""
import numpy as np
import pytest

import oracle
import paper_2005_05826_gb300 as uf
from synth import Table as STable, pair_subset, workload
from tests.gpu_util import METHODS, VARIANTS, assert_close, condensed_index

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRECISIONS = ["fp64", "mixed"]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2005_05826_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def rows_of(table_s):
    ip = table_s.indptr
    return [(table_s.indices[ip[k]:ip[k + 1]].astype(np.int64), table_s.data[ip[k]:ip[k + 1]].copy())
            for k in range(table_s.n_samples)]


def csr(rows, n_features):
    indptr = np.zeros(len(rows) + 1, dtype=np.int64)
    np.cumsum([r[0].size for r in rows], out=indptr[1:])
    idx = np.concatenate([r[0] for r in rows]).astype(np.int32)
    dat = np.concatenate([r[1] for r in rows]).astype(np.float64)
    return STable(len(rows), n_features, indptr, idx, dat)


def near_identical_group(row, total, n_features, rng):
    """The sample scaled to about `total` and its three one-count variants."""
    idx, dat = row
    f = max(1.0, round(total / dat.sum()))
    base = (idx.copy(), dat * f)
    added = (idx.copy(), base[1].copy())
    added[1][int(rng.integers(idx.size))] += 1.0
    absent = np.setdiff1d(np.arange(n_features), idx)
    g = int(rng.choice(absent))
    at = int(np.searchsorted(idx, g))
    new_feat = (np.insert(idx, at, g), np.insert(base[1], at, 1.0))
    moved = (idx.copy(), base[1].copy())
    if idx.size >= 2:
        a, b = rng.choice(idx.size, size=2, replace=False)
        moved[1][a] -= 1.0  # scaled counts are >= f >= 1; a count of 1 moves away entirely
        moved[1][b] += 1.0
        if moved[1][a] == 0.0:
            moved = (np.delete(moved[0], a), np.delete(moved[1], a))
    return [base, added, new_feat, moved]


def build_table(tree_s, base_rows, sources, totals, seed):
    rng = np.random.default_rng(seed)
    rows = list(base_rows)
    groups = []
    for s in sources:
        for tot in totals:
            g = near_identical_group(base_rows[s], tot, tree_s.n_tips, rng)
            groups.append(list(range(len(rows), len(rows) + len(g))))
            rows.extend(g)
    return csr(rows, tree_s.n_tips), groups


def check(tree_s, table_s, i, j, what):
    tree = uf.Tree(tree_s.parent, tree_s.length)
    table = uf.Table(table_s.indptr, table_s.indices, table_s.data, tree)
    n = table_s.n_samples
    idx = condensed_index(n, i, j)
    for method in METHODS + VARIANTS:
        alpha = 0.5 if method == "generalized" else 1.0
        exp = oracle.pairs(tree_s, table_s, method, alpha, i, j)[0]
        for precision in PRECISIONS:
            got, rep = uf.uf_compute(tree, table, method, alpha, precision)
            assert_close(got[idx], exp, method, precision, what)
            if precision == "fp64":
                # every FP64 numerator is a sum of nonnegative terms
                assert rep.clamped == 0, f"{what} {method}: {rep.clamped} numerators clamped"


def within_group_pairs(groups):
    i, j = [], []
    for g in groups:
        for a in range(len(g)):
            for b in range(a + 1, len(g)):
                i.append(g[a])
                j.append(g[b])
    return np.asarray(i, dtype=np.int64), np.asarray(j, dtype=np.int64)


def test_near_identical_yule1k():
    tree_s, t = workload("yule1k_n64")
    base = rows_of(t)[:40]
    table_s, groups = build_table(tree_s, base, sources=[0, 1], totals=[1e4, 1e5, 1e6], seed=501)
    assert table_s.n_samples == 64
    n = table_s.n_samples
    i, j = np.triu_indices(n, k=1)
    check(tree_s, table_s, i.astype(np.int64), j.astype(np.int64), "near-identical, 1,024-tip tree")
    # the groups' own distances are indeed tiny
    gi, gj = within_group_pairs(groups)
    d = oracle.pairs(tree_s, table_s, "weighted_normalized", 1.0, gi, gj)[0]
    assert 0 < d.min() and d.max() < 1e-2


def test_near_identical_yule50k():
    tree_s, t = workload("yule50k_n2048")
    base = rows_of(t)[:1024]
    table_s, groups = build_table(tree_s, base, sources=[0, 1, 2], totals=[1e4, 1e5, 1e6], seed=502)
    gi, gj = within_group_pairs(groups)
    ri, rj = pair_subset(table_s.n_samples, 2000, seed=12345)
    i = np.concatenate([gi, ri])
    j = np.concatenate([gj, rj])
    check(tree_s, table_s, i, j, "near-identical, 50,000-tip tree")
