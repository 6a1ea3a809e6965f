"""Failure detection on the GPU without a fault: the tensor-core kernel's
bounded waits are made to run out (option "tensor_wait_test": its MMA
issuer first waits on an mbarrier nothing signals).  A synchronous call
then returns UF_ETIMEOUT, an asynchronous one (device output on a stream)
writes NaN to every value, and the context stays usable: the next call
matches the oracle."""
import numpy as np
import pytest

import oracle
import paper_2005_05826_gb300 as uf
from synth import table_iid, yule_tree
from tests.gpu_util import assert_close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2005_05826_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def test_tensor_kernel_wait_runs_out_and_the_context_survives():
    tree_s = yule_tree(300, seed=71)
    table_s = table_iid(96, tree_s.n_tips, 0.1, seed=72)
    tree = uf.Tree(tree_s.parent, tree_s.length)
    table = uf.Table(table_s.indptr, table_s.indices, table_s.data, tree)
    n = table_s.n_samples
    assert uf.uf_get_option("tensor_wait_test") == 0
    uf.uf_set_option("sparse", 0)  # every branch through the tensor-core kernel
    try:
        uf.uf_set_option("tensor_wait_test", 1)
        with pytest.raises(uf.UFError) as e:
            uf.uf_compute(tree, table, "unweighted", 1.0, "mixed")
        assert e.value.status == "UF_ETIMEOUT"
        out = torch.zeros(n * (n - 1) // 2, dtype=torch.float64, device="cuda")
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            uf.uf_compute(tree, table, "unweighted", 1.0, "mixed", out=out)  # returns once enqueued
        s.synchronize()
        assert torch.isnan(out).all()
    finally:
        uf.uf_set_option("tensor_wait_test", 0)
    try:
        got, _ = uf.uf_compute(tree, table, "unweighted", 1.0, "mixed")
        exp = oracle.condensed(tree_s, table_s, "unweighted", 1.0)
        assert_close(got, exp, "unweighted", "mixed")
    finally:
        uf.uf_set_option("sparse", 1)
