"""Both accumulate tile shapes of the FP32 min kernel (128 x 128 with 8 x 8
register micro-tiles, 64 x 128 with 4 x 8 at three CTAs per SM; the
autotuner picks between them per size class) against the FP64 oracle, on
tile-edge sample counts and on stripe ranges that start and end inside a
tile, forced with option "tile_shape"."""
import numpy as np
import pytest

import oracle
import paper_2005_05826_gb300 as uf
from synth import table_iid, yule_tree
from tests.gpu_util import assert_close, condensed_index

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2005_05826_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


@pytest.fixture()
def shape_option():
    yield
    uf.uf_set_option("tile_shape", -1)
    uf.uf_set_option("tensor_path", 1)


@pytest.mark.parametrize("shape", [0, 1])
@pytest.mark.parametrize("n", [65, 129, 200, 257])
def test_tile_shape(shape, n, shape_option):
    uf.uf_set_option("tile_shape", shape)
    uf.uf_set_option("tensor_path", 0)  # unweighted on the CUDA-core min kernel as well
    tree_s = yule_tree(400, seed=500 + n)
    table_s = table_iid(n, tree_s.n_tips, 0.05, seed=600 + n)
    tree = uf.Tree(tree_s.parent, tree_s.length)
    table = uf.Table(table_s.indptr, table_s.indices, table_s.data, tree)
    S = n // 2
    for method in ("weighted_normalized", "unweighted", "weighted_unnormalized"):
        exp = oracle.condensed(tree_s, table_s, method)
        got, rep = uf.uf_compute(tree, table, method, 1.0, "mixed")
        assert_close(got, exp, method, "mixed", f"tile shape {shape} n={n}")
        assert rep.stripe_tile == (128 if shape == 0 else 64)
        start = min(37, S // 4 + 1)  # inside a tile, past the first micro-tile rows
        stop = min(S, start + 63)
        part, _ = uf.uf_compute(tree, table, method, 1.0, "mixed", start, stop)
        s = np.arange(start, stop)[:, None]
        k = np.arange(n)[None, :]
        j = (k + s + 1) % n
        want = exp[condensed_index(n, np.minimum(k, j), np.maximum(k, j))]
        assert_close(part.ravel(), want.ravel(), method, "mixed", f"tile shape {shape} n={n} range")
