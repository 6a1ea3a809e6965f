"""FP64 CPU oracle for UniFrac (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product path (the CUDA library and its
Python binding) never calls it and shares no code with it.

``uf_oracle.c`` holds the arithmetic: a per-pair tree walk straight from the
UniFrac definitions (refs [1] and [3] of the paper, Sec. 1; the
variance-adjusted weighted form of Chang, Luan & Sun 2011) and the plain
striped loop of the paper's Sec. 2-3.  This wrapper only builds that file
with gcc and marshals numpy arrays into it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "uf_oracle.c")
LIB = os.path.join(HERE, "_build", "liboracle.so")

METHODS = {"unweighted": 0, "weighted_unnormalized": 1, "weighted_normalized": 2, "generalized": 3,
           "unweighted_unnormalized": 4, "vaw_weighted_unnormalized": 5, "vaw_weighted_normalized": 6}
STATUS = {0: "OK", 1: "EINVAL", 2: "ETREE", 3: "ETABLE", 4: "ERANGE", 5: "ENOMEM"}

_lock = threading.Lock()
_lib = None


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what} failed: {STATUS.get(code, code)}")
        self.code = code
        self.status = STATUS.get(code, str(code))


def build(src: str = SRC, out: str = LIB, force: bool = False) -> str:
    """Compile the oracle with gcc (strict IEEE: no contraction, no fast-math)."""
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = f"{out}.{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-ffp-contract=off",
           "-fno-fast-math", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def load(path: str | None = None):
    global _lib
    with _lock:
        if path is not None:
            return _declare(ctypes.CDLL(path))
        if _lib is None:
            _lib = _declare(ctypes.CDLL(build()))
        return _lib


def _declare(lib):
    i64, i32, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_double
    p = ctypes.c_void_p
    lib.uo_host_cores.restype = i32
    lib.uo_check_tree.argtypes = [i64, p, p]
    lib.uo_check_tree.restype = i32
    lib.uo_tip_count.argtypes = [i64, p]
    lib.uo_tip_count.restype = i64
    lib.uo_check_table.argtypes = [i64, i64, p, p, p, i64]
    lib.uo_check_table.restype = i32
    lib.uo_pairs.argtypes = [i64, p, p, i64, i64, p, p, p, i32, dbl, i64, p, p, p, p, p, i32,
                             ctypes.POINTER(ctypes.c_int)]
    lib.uo_pairs.restype = i32
    lib.uo_striped.argtypes = [i64, p, p, i64, i64, p, p, p, i32, dbl, i64, i64, p, p, p, i32,
                               ctypes.POINTER(ctypes.c_int)]
    lib.uo_striped.restype = i32
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _tree_arrays(tree):
    return (np.ascontiguousarray(tree.parent, dtype=np.int64),
            np.ascontiguousarray(tree.length, dtype=np.float64))


def _table_arrays(table):
    return (np.ascontiguousarray(table.indptr, dtype=np.int64),
            np.ascontiguousarray(table.indices, dtype=np.int32),
            np.ascontiguousarray(table.data, dtype=np.float64))


def host_cores() -> int:
    return int(load().uo_host_cores())


def check_tree(tree) -> str:
    parent, length = _tree_arrays(tree)
    return STATUS[load().uo_check_tree(parent.size, _ptr(parent), _ptr(length))]


def check_table(tree, table) -> str:
    parent, _ = _tree_arrays(tree)
    indptr, indices, data = _table_arrays(table)
    lib = load()
    n_tips = lib.uo_tip_count(parent.size, _ptr(parent))
    return STATUS[lib.uo_check_table(table.n_samples, table.n_features, _ptr(indptr),
                                     _ptr(indices), _ptr(data), n_tips)]


def pairs(tree, table, method: str, alpha: float, pi, pj, n_threads: int = 0, lib=None):
    """FP64 distances (and num, den) of the pairs (pi[q], pj[q]).

    Returns ``(d, num, den, threads_used)``."""
    lib = lib or load()
    parent, length = _tree_arrays(tree)
    indptr, indices, data = _table_arrays(table)
    pi = np.ascontiguousarray(pi, dtype=np.int64)
    pj = np.ascontiguousarray(pj, dtype=np.int64)
    d = np.zeros(pi.size)
    num = np.zeros(pi.size)
    den = np.zeros(pi.size)
    used = ctypes.c_int(0)
    st = lib.uo_pairs(parent.size, _ptr(parent), _ptr(length), table.n_samples, table.n_features,
                      _ptr(indptr), _ptr(indices), _ptr(data), METHODS[method], float(alpha),
                      pi.size, _ptr(pi), _ptr(pj), _ptr(d), _ptr(num), _ptr(den), int(n_threads),
                      ctypes.byref(used))
    if st:
        raise OracleError(st, "uo_pairs")
    return d, num, den, used.value


def condensed(tree, table, method: str, alpha: float = 1.0, n_threads: int = 0, lib=None):
    """All pairs i < j in row-major condensed order."""
    n = table.n_samples
    i, j = np.triu_indices(n, k=1)
    return pairs(tree, table, method, alpha, i, j, n_threads, lib)[0]


def striped(tree, table, method: str, alpha: float, start: int, stop: int, n_threads: int = 0,
            lib=None):
    """The plain striped loop: ``(num, den, dist, threads_used)``, each
    ``[(stop - start), n]`` with stripe s, column k = pair (k, (k+s+1) mod n)."""
    lib = lib or load()
    parent, length = _tree_arrays(tree)
    indptr, indices, data = _table_arrays(table)
    n = table.n_samples
    rows = max(stop - start, 0)
    num = np.zeros((rows, n))
    den = np.zeros((rows, n))
    dist = np.zeros((rows, n))
    used = ctypes.c_int(0)
    st = lib.uo_striped(parent.size, _ptr(parent), _ptr(length), n, table.n_features,
                        _ptr(indptr), _ptr(indices), _ptr(data), METHODS[method], float(alpha),
                        int(start), int(stop), _ptr(num), _ptr(den), _ptr(dist), int(n_threads),
                        ctypes.byref(used))
    if st:
        raise OracleError(st, "uo_striped")
    return num, den, dist, used.value
