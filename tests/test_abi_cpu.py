"""The C-ABI library on the CPU: it loads, exports every declared symbol,
and its host-side validation returns the documented codes.  No kernel runs
here; a compute call without a GPU must fail loudly (no CPU fallback)."""
import os
import re

import numpy as np
import pytest

import paper_2005_05826_gb300 as uf
from paper_2005_05826_gb300 import build as ufbuild
from synth import Table as STable, table_iid, yule_tree

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    ufbuild.build()


def declared_functions():
    names = []
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            text = open(os.path.join(inc, f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(uf_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


def test_exports_every_declared_symbol():
    lib = uf.load()
    names = declared_functions()
    assert "uf_compute" in names and "uf_tree_create" in names
    for name in names:
        assert hasattr(lib, name), f"{name} declared but not exported"


def test_report_layout_matches_header(tmp_path):
    # the binding's ctypes Report has the size and field offsets of the C
    # uf_report: a small C program built against the header prints them
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    fields = [name for name, _ in uf.Report._fields_]
    src = ["#include <stddef.h>", "#include <stdio.h>", '#include "unifrac_gb300.h"', "int main(void) {",
           '  printf("size %zu\\n", sizeof(uf_report));']
    src += [f'  printf("{f} %zu\\n", offsetof(uf_report, {f}));' for f in fields]
    src += ["  return 0;", "}"]
    c = tmp_path / "layout.c"
    c.write_text("\n".join(src) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                        check=True).stdout.splitlines())
    import ctypes
    assert int(got["size"]) == ctypes.sizeof(uf.Report)
    for f in fields:
        assert int(got[f]) == getattr(uf.Report, f).offset, f


def test_header_compiles_as_c_and_cpp(tmp_path):
    # the public header stands alone in strict C99 and in C++ without warnings
    import shutil
    import subprocess
    src = '#include "unifrac_gb300.h"\nint main(void) { uf_report r; (void)r; return (int)UF_OK; }\n'
    for compiler, ext, std in (("gcc", "c", "-std=c99"), ("g++", "cpp", "-std=c++11")):
        cc = shutil.which(compiler)
        if cc is None:
            continue
        f = tmp_path / f"h.{ext}"
        f.write_text(src)
        p = subprocess.run([cc, std, "-Wall", "-Wextra", "-pedantic", "-Werror", "-I",
                            os.path.join(ROOT, "include"), "-c", str(f), "-o", str(tmp_path / f"h_{ext}.o")],
                           capture_output=True, text=True)
        assert p.returncode == 0, p.stderr


def test_enum_values_match_header():
    # the binding's method, precision and status numbers are the header's
    text = open(os.path.join(ROOT, "include", "unifrac_gb300.h")).read()
    vals = {k: int(v) for k, v in re.findall(r"\b(UF_[A-Z0-9_]+)\s*=\s*(\d+)", text)}
    for name, code in uf.METHODS.items():
        assert vals["UF_" + name.upper()] == code, name
    for name, code in uf.PRECISIONS.items():
        assert vals["UF_" + name.upper()] == code, name
    lib = uf.load()
    for code, name in uf.STATUS.items():
        assert vals[name] == code, name
        assert lib.uf_status_name(code).decode() == name


OPTIONS = {  # name: (default, accepted values, rejected values)
    "branch_block": (0, [1, 4096, 0], [-1]),
    "kernel_timing": (0, [1, 0], [-1, 2]),
    "tensor_path": (1, [0, 1], [-1, 2]),
    "graph": (1, [0, 1], [-1, 2]),
    "autotune": (1, [0, 1], [-1, 3]),
    "sparse": (1, [0, 2, 1], [-1, 3]),
    "sparse_overlap": (1, [0, 1], [-1, 2]),
    "tensor_wait_test": (0, [1, 0], [-1, 2]),
    "sparse_region_bytes": (48_000_000, [4096, 10**9, 48_000_000], [1, 4095, -5]),
    "sparse_fuse": (2, [0, 6, 2], [-1, 1, 3, 7]),
    "tile_shape": (-1, [0, 1, -1], [-2, 2]),
}


def test_options():
    header = open(os.path.join(ROOT, "include", "unifrac_gb300.h")).read()
    for name, (default, good, bad) in OPTIONS.items():
        assert f'"{name}"' in header, f"option {name} not documented"
        assert uf.uf_get_option(name) == default, name
        for v in good:
            uf.uf_set_option(name, v)
            assert uf.uf_get_option(name) == v, (name, v)
        for v in bad:
            assert _code(lambda: uf.uf_set_option(name, v)) == "UF_EINVAL", (name, v)
            assert uf.uf_get_option(name) == good[-1], (name, v)
        uf.uf_set_option(name, default)
    # autotune 2 forgets the tuned chunk sizes and reads back as 1; region bytes 0 is the default
    uf.uf_set_option("autotune", 2)
    assert uf.uf_get_option("autotune") == 1
    uf.uf_set_option("sparse_region_bytes", 0)
    assert uf.uf_get_option("sparse_region_bytes") == 48_000_000
    assert _code(lambda: uf.uf_set_option("no_such_option", 1)) == "UF_EINVAL"
    assert uf.uf_get_option("no_such_option") == -1


def test_stripe_count():
    assert [uf.uf_stripe_count(n) for n in (0, 1, 2, 3, 4, 5, 64, 65)] == [0, 0, 1, 1, 2, 2, 32, 32]


def _code(fn):
    with pytest.raises(uf.UFError) as e:
        fn()
    return e.value.status


def test_table_validation_many_threads():
    # a table large enough for one validating pass per host thread: the
    # reported error is still the first failing sample in sample order
    tree_s = yule_tree(4000, seed=41)
    n, per = 40_000, 60
    rng = np.random.default_rng(42)
    ix = np.sort(np.stack([rng.choice(tree_s.n_tips, per, replace=False) for _ in range(n)]), axis=1)
    ip = np.arange(n + 1, dtype=np.int64) * per
    d = np.ones(n * per)
    tree = uf.Tree(tree_s.parent, tree_s.length)
    uf.Table(ip, ix.ravel().astype(np.int32), d, tree)  # valid
    bad_ix = ix.copy()
    bad_ix[35_000, [3, 4]] = bad_ix[35_000, [4, 3]]       # unsorted, late sample
    bad_d = d.copy()
    bad_d[12_345 * per + 7] = 0.0                          # zero count, earlier sample
    with pytest.raises(uf.UFError) as e:
        uf.Table(ip, bad_ix.ravel().astype(np.int32), bad_d, tree)
    assert e.value.status == "UF_ETABLE" and "sample 12345:" in str(e.value)
    with pytest.raises(uf.UFError) as e:
        uf.Table(ip, bad_ix.ravel().astype(np.int32), d, tree)
    assert "sample 35000: feature indices not strictly increasing" in str(e.value)


def test_tree_validation():
    ok = uf.Tree(np.array([2, 2, -1]), np.array([1.0, 2.0, 0.0]))
    assert ok.n_tips == 2
    assert _code(lambda: uf.Tree(np.array([2, 2, 0]), np.ones(3))) == "UF_ETREE"
    assert _code(lambda: uf.Tree(np.array([2, 0, -1]), np.ones(3))) == "UF_ETREE"
    assert _code(lambda: uf.Tree(np.array([2, 2, -1]), np.array([1.0, -1.0, 0]))) == "UF_ETREE"
    assert _code(lambda: uf.Tree(np.array([2, 2, -1]), np.array([np.inf, 1.0, 0]))) == "UF_ETREE"
    assert _code(lambda: uf.Tree(np.array([], dtype=np.int64), np.array([]))) == "UF_EINVAL"
    # the root's length is ignored, even when not finite
    uf.Tree(np.array([2, 2, -1]), np.array([1.0, 2.0, np.nan]))
    # unary nodes are fine
    assert uf.Tree(np.array([1, 3, 3, -1]), np.ones(4)).n_tips == 2


def test_table_validation():
    tree = uf.Tree(np.array([2, 2, -1]), np.array([1.0, 2.0, 0.0]))
    uf.Table(np.array([0, 2, 3]), np.array([0, 1, 0]), np.array([1.0, 2.0, 3.0]), tree)
    bad = [
        (np.array([0, 2, 2]), np.array([0, 1]), np.array([1.0, 1.0])),          # empty sample
        (np.array([0, 2]), np.array([1, 0]), np.array([1.0, 1.0])),             # unsorted
        (np.array([0, 2]), np.array([0, 0]), np.array([1.0, 1.0])),             # duplicate
        (np.array([0, 1]), np.array([2]), np.array([1.0])),                     # out of range
        (np.array([0, 1]), np.array([0]), np.array([0.0])),                     # zero count
        (np.array([0, 1]), np.array([0]), np.array([np.nan])),                  # NaN count
        (np.array([1, 2]), np.array([0, 1]), np.array([1.0, 1.0])),             # indptr[0] != 0
    ]
    for ip, ix, d in bad:
        assert _code(lambda: uf.Table(ip, ix, d, tree)) == "UF_ETABLE"
    assert _code(lambda: uf.Table(np.array([0, 1]), np.array([0]), np.array([1.0]), tree,
                                  n_features=3)) == "UF_ETABLE"


def test_compute_argument_errors():
    tree_s = yule_tree(20, seed=1)
    tab_s = table_iid(9, tree_s.n_tips, 0.3, seed=2)
    tree = uf.Tree(tree_s.parent, tree_s.length)
    table = uf.Table(tab_s.indptr, tab_s.indices, tab_s.data, tree)
    S = uf.uf_stripe_count(9)
    assert _code(lambda: uf.uf_compute(tree, table, "generalized", 1.5)) == "UF_EINVAL"
    assert _code(lambda: uf.uf_compute(tree, table, "generalized", float("nan"))) == "UF_EINVAL"
    assert _code(lambda: uf.uf_compute(tree, table, "unweighted", 1.0, "fp64", 0, S + 1)) == "UF_ERANGE"
    assert _code(lambda: uf.uf_compute(tree, table, "unweighted", 1.0, "fp64", 3, 2)) == "UF_ERANGE"
    assert _code(lambda: uf.uf_compute(tree, table, "unweighted", 1.0, "fp64", -1, 2)) == "UF_ERANGE"
    # an empty range is a no-op
    out, rep = uf.uf_compute(tree, table, "unweighted", 1.0, "fp64", 2, 2)
    assert out.size == 0
    # a table built for another tree is rejected
    other = uf.Tree(*(lambda t: (t.parent, t.length))(yule_tree(21, seed=3)))
    t_other = uf.Table(*(lambda t: (t.indptr, t.indices, t.data))(table_iid(4, 21, 0.5, seed=4)), other)
    assert _code(lambda: uf.uf_compute(tree, t_other, "unweighted")) == "UF_ETABLE"


def test_call_sample_cap():
    # one compute call takes at most 2^30 samples on its combined axis: 1,025
    # copies of a 2^20-sample table are rejected before any device work (the
    # output pointers are never written)
    import ctypes
    n = 1 << 20
    tree = uf.Tree(np.array([2, 2, -1], np.int64), np.array([1.0, 2.0, 0.0]))
    table = uf.Table(np.arange(n + 1, dtype=np.int64), np.zeros(n, np.int32), np.ones(n), tree)
    lib = uf.load()
    nt = 1025
    dummy = np.zeros(1)
    handles = (ctypes.c_void_p * nt)(*([table.handle.value] * nt))
    outs = (ctypes.c_void_p * nt)(*([dummy.ctypes.data] * nt))
    st = lib.uf_compute_batch(tree.handle, handles, nt, 2, 1.0, 1, outs, 0, None, None)
    assert lib.uf_status_name(st).decode() == "UF_EINVAL"
    assert "2^30" in uf.uf_last_error()


def test_binding_argument_checks():
    # the Python binding rejects unknown names and unusable output buffers
    # before any library call
    tree_s = yule_tree(20, seed=1)
    tab_s = table_iid(9, tree_s.n_tips, 0.3, seed=2)
    tree = uf.Tree(tree_s.parent, tree_s.length)
    table = uf.Table(tab_s.indptr, tab_s.indices, tab_s.data, tree)
    need = uf.condensed_size(9)
    with pytest.raises(ValueError, match="unknown method"):
        uf.uf_compute(tree, table, "weighted")
    with pytest.raises(ValueError, match="unknown precision"):
        uf.uf_compute(tree, table, "unweighted", 1.0, "fp16")
    with pytest.raises(ValueError, match="unknown method"):
        uf.uf_compute_batch(tree, [table], "bray_curtis")
    for bad in (np.zeros(need, np.float32), np.zeros(need - 1), np.zeros((need, 2))[:, 0]):
        with pytest.raises(ValueError, match="output array"):
            uf.uf_compute(tree, table, "unweighted", out=bad)
    with pytest.raises(ValueError, match="output array"):
        uf.uf_compute(tree, table, "unweighted", out=np.zeros(need), out_fp32=True)
    torch = pytest.importorskip("torch")
    with pytest.raises(ValueError, match="output tensor"):
        uf.uf_compute(tree, table, "unweighted", out=torch.zeros(need, dtype=torch.float32))


def test_no_cpu_fallback():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present; the GPU tests cover the compute path")
    tree_s = yule_tree(20, seed=1)
    tab_s = table_iid(9, tree_s.n_tips, 0.3, seed=2)
    tree = uf.Tree(tree_s.parent, tree_s.length)
    table = uf.Table(tab_s.indptr, tab_s.indices, tab_s.data, tree)
    assert _code(lambda: uf.uf_compute(tree, table, "unweighted")) == "UF_ECUDA"
    assert _code(lambda: uf.uf_compute_batch(tree, [table, table], "generalized", 0.5, "mixed")) == "UF_ECUDA"


def test_compute_ranges_validates_before_the_device():
    # job ranges are checked on the host: a range past the table's stripes is
    # UF_ERANGE, and valid jobs without a GPU are UF_ECUDA (no CPU fallback)
    from synth import table_iid, yule_tree
    tree_s = yule_tree(50, seed=3)
    table_s = table_iid(12, tree_s.n_tips, 0.3, seed=4)
    tree = uf.Tree(tree_s.parent, tree_s.length)
    table = uf.Table(table_s.indptr, table_s.indices, table_s.data, tree)
    with pytest.raises(uf.UFError) as e:
        uf.uf_compute_ranges(tree, [(table, 0, 3), (table, 4, 7)], "weighted_normalized")
    assert e.value.status == "UF_ERANGE"
    # empty ranges only: nothing to compute, UF_OK on any machine
    outs, reps = uf.uf_compute_ranges(tree, [(table, 2, 2)], "unweighted")
    assert outs[0].size == 0
    import torch
    if not torch.cuda.is_available():
        with pytest.raises(uf.UFError) as e:
            uf.uf_compute_ranges(tree, [(table, 0, 3), (table, 3, 6)], "unweighted", precision="mixed")
        assert e.value.status == "UF_ECUDA"


def test_probe_validates_before_the_device():
    # the diagnostic atomic-rate probe rejects bad sizes before any CUDA call
    for nbytes in (0, 8 * 1000, 8 * 1023, 8 * 3000, 8 * (1 << 31) * 2):
        assert _code(lambda: uf.uf_probe_l2_atomics(nbytes)) == "UF_EINVAL", nbytes
    lib = uf.load()
    assert lib.uf_probe_l2_atomics(16 << 20, None) == 1  # UF_EINVAL
