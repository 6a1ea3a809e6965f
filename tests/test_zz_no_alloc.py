"""uf_compute_noalloc against uf_compute.

uf_compute_noalloc serves callers that may not allocate device memory (their
own memory manager owns the device heap, or the allocator may not be entered
at that point): it works in the library's fixed 64 MiB device area instead.
This file is collected last so that a run stopping at its first failure has
already run every other test.  Each case calls the entry point through the C
ABI twice in a row (the area keeps the previous call's data, so the second
call checks that everything that must start at zero is cleared) and compares
both results with uf_compute and with the FP64 oracle, within the tolerances
of the other GPU tests.
"""
import numpy as np
import pytest

import oracle
import paper_2005_05826_gb300 as uf
from synth import table_iid, workload, yule_tree
from tests.gpu_util import METHODS, assert_close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2005_05826_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def handles(tree_s, table_s):
    tree = uf.Tree(tree_s.parent, tree_s.length)
    return tree, uf.Table(table_s.indptr, table_s.indices, table_s.data, tree)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_matches_compute_twice(precision):
    cases = [workload("yule1k_n64"),
             (lambda t: (t, table_iid(129, t.n_tips, 0.05, seed=71)))(yule_tree(700, seed=70))]
    for tree_s, table_s in cases:
        tree, table = handles(tree_s, table_s)
        n = table_s.n_samples
        for method in METHODS:
            alpha = 0.5 if method == "generalized" else 1.0
            ref, _ = uf.uf_compute(tree, table, method, alpha, precision)
            exp = oracle.condensed(tree_s, table_s, method, alpha)
            for call in range(2):
                out = torch.full((n * (n - 1) // 2,), float("nan"), dtype=torch.float64,
                                 device="cuda")
                uf.uf_compute_noalloc(tree, table, method, alpha, precision, out=out)
                got = out.cpu().numpy()
                assert np.isfinite(got).all()
                assert_close(got, ref, method, precision, f"noalloc call {call + 1} n={n} vs uf_compute")
                assert_close(got, exp, method, precision, f"noalloc call {call + 1} n={n} vs oracle")


def test_noalloc_rejects_problems_beyond_the_area():
    # 4,096 samples: the stripe accumulator alone needs 2048 * 4096 * 8 B = 64 MiB
    tree_s = yule_tree(64, seed=72)
    table_s = table_iid(4096, tree_s.n_tips, 0.2, seed=73)
    tree, table = handles(tree_s, table_s)
    out = torch.empty(4096 * 4095 // 2, dtype=torch.float64, device="cuda")
    with pytest.raises(uf.UFError) as e:
        uf.uf_compute_noalloc(tree, table, "weighted_normalized", 1.0, "fp64", out=out)
    assert e.value.status == "UF_ENOMEM"
    assert "fixed area holds" in str(e.value)
