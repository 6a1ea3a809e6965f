"""Many stripe ranges in one call (uf_compute_ranges): jobs over two tables
of one tree, a table in several jobs with adjacent and overlapping ranges and
a full-range job, every method's kernels (CUDA-core stripes, tensor-core
gram, sparse rows), against the FP64 oracle cell by cell and against
single-range uf_compute calls."""
import numpy as np
import pytest

import oracle
import paper_2005_05826_gb300 as uf
from synth import table_iid, yule_tree
from tests.gpu_util import METHODS, VARIANTS, assert_close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2005_05826_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def stripe_pairs(n, start, stop):
    s = np.arange(start, stop)[:, None]
    k = np.arange(n)[None, :]
    j = (k + s + 1) % n
    return np.minimum(k, j).ravel(), np.maximum(k, j).ravel()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_many_ranges_in_one_call(precision):
    tree_s = yule_tree(2000, seed=91)
    ta = table_iid(300, tree_s.n_tips, 0.02, seed=92)
    tb = table_iid(129, tree_s.n_tips, 0.05, seed=93)
    tree = uf.Tree(tree_s.parent, tree_s.length)
    a = uf.Table(ta.indptr, ta.indices, ta.data, tree)
    b = uf.Table(tb.indptr, tb.indices, tb.data, tree)
    jobs = [(a, 0, 20), (a, 20, 57), (a, 50, 150), (b, 0, 64), (b, 10, 11), (a, 149, 150)]
    for method in METHODS + VARIANTS:
        alpha = 0.5 if method == "generalized" else 1.0
        outs, reps = uf.uf_compute_ranges(tree, jobs, method, alpha, precision)
        for (t, start, stop), got, rep, ts in zip(jobs, outs, reps, [ta, ta, ta, tb, tb, ta]):
            n = ts.n_samples
            full = start == 0 and stop == n // 2
            if full:
                exp = oracle.condensed(tree_s, ts, method, alpha)
            else:
                i, j = stripe_pairs(n, start, stop)
                exp = oracle.pairs(tree_s, ts, method, alpha, i, j)[0]
            assert_close(np.asarray(got).ravel(), exp, method, precision, f"ranges job [{start}, {stop})")
            single, _ = uf.uf_compute(tree, t, method, alpha, precision, start, stop)
            assert_close(np.asarray(got).ravel(), np.asarray(single).ravel(), method, precision,
                         f"ranges job [{start}, {stop}) vs uf_compute")
            if method == "unweighted" and precision == "mixed":
                assert rep.path == 1
