"""Downstream agreement of the mixed-precision and FP64 matrices (the
validation of the paper's Sec. 4: a Mantel test between FP32 and FP64
results), plus principal-coordinate agreement, on the GPU."""
import numpy as np
import pytest

import paper_2005_05826_gb300 as uf
from paper_2005_05826_gb300 import downstream as ds
from synth import table_prevalence, yule_tree
from tests.gpu_util import METHODS

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2005_05826_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def test_mixed_and_fp64_matrices_agree_downstream():
    tree_s = yule_tree(5000, seed=301)
    table_s = table_prevalence(400, tree_s.n_tips, 0.5, 20.0, seed=302)
    tree = uf.Tree(tree_s.parent, tree_s.length)
    table = uf.Table(table_s.indptr, table_s.indices, table_s.data, tree)
    for method in METHODS:
        a = 0.5 if method == "generalized" else 1.0
        d64, _ = uf.uf_compute(tree, table, method, a, "fp64")
        d32, _ = uf.uf_compute(tree, table, method, a, "mixed")
        r, p = ds.mantel(d32, d64, permutations=99, seed=7)
        assert r * r >= 0.99999, (method, r)
        assert p <= 0.01, (method, p)
        c64, _ = ds.pcoa(d64, k=5)
        c32, _ = ds.pcoa(d32, k=5)
        assert ds.procrustes(c64, c32) < 1e-6, method
