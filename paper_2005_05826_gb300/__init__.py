"""GB300 Striped UniFrac engine: Python binding of libunifrac_gb300.so.

Argument marshalling only: every step of the computation runs in the CUDA
kernels behind the C ABI (include/unifrac_gb300.h).  The functions keep the
C names (``uf_tree_create``, ``uf_table_create``, ``uf_compute``,
``uf_compute_batch``, ``uf_stripe_count``, ``uf_last_error``).  Arrays may be
numpy arrays (host memory) or torch tensors; a CUDA torch tensor as output
is written in place on torch's current stream.

There is no CPU fallback: if the shared library is missing or no GPU is
present the calls raise.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import threading

import numpy as np

__all__ = ["UFError", "Tree", "Table", "Report", "METHODS", "PRECISIONS", "library_path", "load",
           "uf_last_error", "uf_stripe_count", "uf_tree_create", "uf_table_create", "uf_compute",
           "uf_compute_batch", "uf_compute_ranges", "uf_compute_noalloc", "uf_set_option", "uf_get_option",
           "condensed_size"]

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libunifrac_gb300.so")

METHODS = {"unweighted": 0, "weighted_unnormalized": 1, "weighted_normalized": 2, "generalized": 3,
           "unweighted_unnormalized": 4, "vaw_weighted_unnormalized": 5, "vaw_weighted_normalized": 6}
PRECISIONS = {"fp64": 0, "mixed": 1}
STATUS = {0: "UF_OK", 1: "UF_EINVAL", 2: "UF_ETREE", 3: "UF_ETABLE", 4: "UF_ERANGE",
          5: "UF_ENOMEM", 6: "UF_ECUDA", 7: "UF_ETIMEOUT", 8: "UF_ECANCELLED"}


class Report(ctypes.Structure):
    _fields_ = [("seconds", ctypes.c_double), ("updates", ctypes.c_double),
                ("alg_flops", ctypes.c_double), ("exec_flops", ctypes.c_double),
                ("hbm_bytes_est", ctypes.c_double), ("stripe_tile", ctypes.c_int64),
                ("sample_tile", ctypes.c_int64), ("branch_block", ctypes.c_int64),
                ("n_blocks", ctypes.c_int64), ("kernels", ctypes.c_int64),
                ("path", ctypes.c_int32), ("clamped", ctypes.c_int32),
                ("h2d_bytes", ctypes.c_double), ("d2h_bytes", ctypes.c_double),
                ("t_embed_ms", ctypes.c_double), ("t_accumulate_ms", ctypes.c_double),
                ("t_diag_ms", ctypes.c_double), ("t_finalize_ms", ctypes.c_double),
                ("acc_launches", ctypes.c_int64), ("chunk_rows", ctypes.c_int64),
                ("graph", ctypes.c_int32), ("reserved2", ctypes.c_int32),
                ("dense_rows", ctypes.c_int64), ("sparse_rows", ctypes.c_int64),
                ("sparse_pairs", ctypes.c_double), ("t_sparse_ms", ctypes.c_double),
                ("sparse_pair_updates", ctypes.c_double)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_ if not name.startswith("reserved")}


class UFError(RuntimeError):
    def __init__(self, code: int, msg: str):
        self.code = code
        self.status = STATUS.get(code, str(code))
        super().__init__(f"{self.status}: {msg}")


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return LIB_PATH


def load():
    """Load the in-tree shared library (build it first with
    ``paper_2005_05826_gb300.build.build()``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is not built; run paper_2005_05826_gb300/build.py")
        lib = ctypes.CDLL(LIB_PATH)
        i64, i32, dbl, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
        lib.uf_last_error.restype = ctypes.c_char_p
        lib.uf_status_name.argtypes = [i32]
        lib.uf_status_name.restype = ctypes.c_char_p
        lib.uf_probe_l2_atomics.argtypes = [i64, ctypes.POINTER(dbl)]
        lib.uf_probe_l2_atomics.restype = i32
        lib.uf_stripe_count.argtypes = [i64]
        lib.uf_stripe_count.restype = i64
        lib.uf_tree_create.argtypes = [i64, vp, vp, ctypes.POINTER(vp)]
        lib.uf_tree_create.restype = i32
        lib.uf_tree_destroy.argtypes = [vp]
        lib.uf_tree_destroy.restype = None
        lib.uf_tree_tips.argtypes = [vp]
        lib.uf_tree_tips.restype = i64
        lib.uf_table_create.argtypes = [i64, i64, vp, vp, vp, vp, ctypes.POINTER(vp)]
        lib.uf_table_create.restype = i32
        lib.uf_table_destroy.argtypes = [vp]
        lib.uf_table_destroy.restype = None
        lib.uf_table_samples.argtypes = [vp]
        lib.uf_table_samples.restype = i64
        lib.uf_compute.argtypes = [vp, vp, i32, dbl, i32, i64, i64, vp, i32, i32,
                                   ctypes.POINTER(Report), vp]
        lib.uf_compute.restype = i32
        lib.uf_compute_batch.argtypes = [vp, vp, i64, i32, dbl, i32, vp, i32,
                                         ctypes.POINTER(Report), vp]
        lib.uf_compute_batch.restype = i32
        lib.uf_compute_ranges.argtypes = [vp, vp, vp, vp, i64, i32, dbl, i32, vp, i32, i32,
                                          ctypes.POINTER(Report), vp]
        lib.uf_compute_ranges.restype = i32
        lib.uf_compute_noalloc.argtypes = [vp, vp, i32, dbl, i32, vp, vp]
        lib.uf_compute_noalloc.restype = i32
        lib.uf_set_option.argtypes = [ctypes.c_char_p, i64]
        lib.uf_set_option.restype = i32
        lib.uf_get_option.argtypes = [ctypes.c_char_p]
        lib.uf_get_option.restype = i64
        _lib = lib
        return lib


def _check(code: int):
    if code != 0:
        raise UFError(code, load().uf_last_error().decode(errors="replace"))


def uf_last_error() -> str:
    return load().uf_last_error().decode(errors="replace")


def uf_set_option(name: str, value: int) -> None:
    _check(load().uf_set_option(name.encode(), int(value)))


def uf_get_option(name: str) -> int:
    return int(load().uf_get_option(name.encode()))


def uf_stripe_count(n_samples: int) -> int:
    return int(load().uf_stripe_count(int(n_samples)))


def condensed_size(n_samples: int) -> int:
    return n_samples * (n_samples - 1) // 2


def _host(a, dtype):
    """numpy view of a host array (torch CPU tensors included)."""
    if hasattr(a, "detach") and hasattr(a, "numpy"):
        a = a.detach().cpu().numpy()
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a) -> int:
    return a.ctypes.data


class Tree:
    """Owns a ``uf_tree`` handle (see uf_tree_create in the C header)."""

    def __init__(self, parent, length):
        lib = load()
        self._parent = _host(parent, np.int64)
        self._length = _host(length, np.float64)
        if self._length.shape != self._parent.shape:
            raise ValueError("parent and length must have the same length")
        h = ctypes.c_void_p()
        _check(lib.uf_tree_create(self._parent.size, _ptr(self._parent), _ptr(self._length),
                                  ctypes.byref(h)))
        self._h = h
        self.n_nodes = int(self._parent.size)
        self.n_tips = int(lib.uf_tree_tips(h))

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().uf_tree_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Table:
    """Owns a ``uf_table`` handle: CSR counts with samples as rows."""

    def __init__(self, indptr, indices, data, tree: Tree, n_features: int | None = None):
        lib = load()
        self._indptr = _host(indptr, np.int64)
        self._indices = _host(indices, np.int32)
        self._data = _host(data, np.float64)
        self.n_samples = int(self._indptr.size - 1)
        n_features = tree.n_tips if n_features is None else int(n_features)
        h = ctypes.c_void_p()
        _check(lib.uf_table_create(self.n_samples, n_features, _ptr(self._indptr),
                                   _ptr(self._indices), _ptr(self._data), tree.handle,
                                   ctypes.byref(h)))
        self._h = h
        self.tree = tree

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().uf_table_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def uf_tree_create(parent, length) -> Tree:
    return Tree(parent, length)


def uf_table_create(indptr, indices, data, tree: Tree, n_features: int | None = None) -> Table:
    return Table(indptr, indices, data, tree, n_features)


def _code_of(codes: dict, name: str, what: str) -> int:
    """The C enum value of a method or precision name."""
    try:
        return codes[name]
    except (KeyError, TypeError):
        raise ValueError(f"unknown {what} {name!r}; one of {', '.join(codes)}") from None


def _out_spec(out, n_values: int, out_fp32: bool):
    """(pointer, is_device, stream, keepalive) for an output buffer."""
    if out is None:
        arr = np.empty(n_values, dtype=np.float32 if out_fp32 else np.float64)
        return arr.ctypes.data, 0, None, arr
    if hasattr(out, "data_ptr"):  # torch tensor
        import torch
        want = torch.float32 if out_fp32 else torch.float64
        if out.dtype != want or not out.is_contiguous() or out.numel() < n_values:
            raise ValueError(f"output tensor must be contiguous {want} with >= {n_values} elements")
        if out.is_cuda:
            return out.data_ptr(), 1, torch.cuda.current_stream(out.device).cuda_stream, out
        return out.data_ptr(), 0, None, out
    arr = out
    want = np.float32 if out_fp32 else np.float64
    if arr.dtype != want or not arr.flags.c_contiguous or arr.size < n_values:
        raise ValueError(f"output array must be contiguous {want} with >= {n_values} elements")
    return arr.ctypes.data, 0, None, arr


def _on_device_of(buf):
    """Context in which a CUDA tensor's device is the current device (the C
    ABI writes device outputs on the current device); no-op otherwise."""
    if hasattr(buf, "is_cuda") and buf.is_cuda:
        import torch
        return torch.cuda.device(buf.device)
    return contextlib.nullcontext()


def uf_compute(tree: Tree, table: Table, method: str, alpha: float = 1.0, precision: str = "fp64",
               stripe_start: int = 0, stripe_stop: int | None = None, out=None,
               out_fp32: bool = False, stream=None):
    """Distances for stripes [stripe_start, stripe_stop) (default: all).

    Full range -> condensed vector of n(n-1)/2; other ranges ->
    (stop - start) x n stripe-major values.  Returns ``(out, Report)``.
    ``stream`` overrides the stream (an int handle) for device outputs."""
    lib = load()
    m_code, p_code = _code_of(METHODS, method, "method"), _code_of(PRECISIONS, precision, "precision")
    n = table.n_samples
    S = uf_stripe_count(n)
    stop = S if stripe_stop is None else int(stripe_stop)
    start = int(stripe_start)
    full = start == 0 and stop == S
    n_values = condensed_size(n) if full else max(stop - start, 0) * n
    ptr, is_dev, st, keep = _out_spec(out, n_values, out_fp32)
    if stream is not None:
        st = int(stream)
    rep = Report()
    with _on_device_of(out):
        _check(lib.uf_compute(tree.handle, table.handle, m_code, float(alpha),
                              p_code, start, stop, ctypes.c_void_p(ptr), is_dev,
                              int(bool(out_fp32)), ctypes.byref(rep),
                              ctypes.c_void_p(st) if st else None))
    if out is None and not full:
        keep = keep.reshape(max(stop - start, 0), n)
    return keep, rep


def uf_compute_batch(tree: Tree, tables, method: str, alpha: float = 1.0, precision: str = "fp64",
                     outs=None, stream=None):
    """Full-range condensed distances of many tables over one tree.
    Returns ``(outs, reports)``."""
    lib = load()
    m_code, p_code = _code_of(METHODS, method, "method"), _code_of(PRECISIONS, precision, "precision")
    nt = len(tables)
    if outs is None:
        outs = [None] * nt
    specs = [_out_spec(o, condensed_size(t.n_samples), False) for o, t in zip(outs, tables)]
    devs = {s[1] for s in specs}
    if len(devs) > 1:
        raise ValueError("outputs must be all host or all device buffers")
    is_dev = devs.pop() if devs else 0
    cuda_devs = {o.device for o in outs if hasattr(o, "is_cuda") and o.is_cuda}
    if len(cuda_devs) > 1:
        raise ValueError("device outputs must all be on one device")
    st = stream if stream is not None else next((s[2] for s in specs if s[2]), None)
    handles = (ctypes.c_void_p * nt)(*[t.handle.value for t in tables])
    ptrs = (ctypes.c_void_p * nt)(*[s[0] for s in specs])
    reps = (Report * max(nt, 1))()
    with _on_device_of(next((o for o in outs if hasattr(o, "is_cuda") and o.is_cuda), None)):
        _check(lib.uf_compute_batch(tree.handle, handles, nt, m_code, float(alpha),
                                    p_code, ptrs, is_dev, reps,
                                    ctypes.c_void_p(int(st)) if st else None))
    return [s[3] for s in specs], [reps[i] for i in range(nt)]


def uf_compute_ranges(tree: Tree, jobs, method: str, alpha: float = 1.0, precision: str = "fp64",
                      outs=None, out_fp32: bool = False, stream=None):
    """Many (table, stripe_start, stripe_stop) jobs over one tree in one call.
    Job t's output is the condensed matrix for the full range, else
    (stop - start) x n stripe-major values.  Returns ``(outs, reports)``."""
    lib = load()
    m_code, p_code = _code_of(METHODS, method, "method"), _code_of(PRECISIONS, precision, "precision")
    nj = len(jobs)
    if outs is None:
        outs = [None] * nj
    sizes = []
    for table, start, stop in jobs:
        full = start == 0 and stop == uf_stripe_count(table.n_samples)
        sizes.append(condensed_size(table.n_samples) if full else max(stop - start, 0) * table.n_samples)
    specs = [_out_spec(o, sz, out_fp32) for o, sz in zip(outs, sizes)]
    devs = {s[1] for s in specs}
    if len(devs) > 1:
        raise ValueError("outputs must be all host or all device buffers")
    is_dev = devs.pop() if devs else 0
    cuda_devs = {o.device for o in outs if hasattr(o, "is_cuda") and o.is_cuda}
    if len(cuda_devs) > 1:
        raise ValueError("device outputs must all be on one device")
    st = stream if stream is not None else next((s[2] for s in specs if s[2]), None)
    handles = (ctypes.c_void_p * nj)(*[t.handle.value for t, _, _ in jobs])
    starts = np.ascontiguousarray([int(a) for _, a, _ in jobs], dtype=np.int64)
    stops = np.ascontiguousarray([int(b) for _, _, b in jobs], dtype=np.int64)
    ptrs = (ctypes.c_void_p * nj)(*[s[0] for s in specs])
    reps = (Report * max(nj, 1))()
    with _on_device_of(next((o for o in outs if hasattr(o, "is_cuda") and o.is_cuda), None)):
        _check(lib.uf_compute_ranges(tree.handle, handles, _ptr(starts), _ptr(stops), nj, m_code, float(alpha),
                                     p_code, ptrs, is_dev, int(bool(out_fp32)), reps,
                                     ctypes.c_void_p(int(st)) if st else None))
    res = []
    for (table, start, stop), s, sz in zip(jobs, specs, sizes):
        keep = s[3]
        full = start == 0 and stop == uf_stripe_count(table.n_samples)
        if isinstance(keep, np.ndarray) and outs[len(res)] is None and not full:
            keep = keep.reshape(max(stop - start, 0), table.n_samples)
        res.append(keep)
    return res, [reps[i] for i in range(nj)]


def uf_probe_l2_atomics(nbytes: int = 16 << 20) -> float:
    """Random 64-bit atomic adds per second into a device array of nbytes on
    the current device (diagnostic: the ceiling of the region scatter's
    atomics)."""
    rate = ctypes.c_double(0.0)
    _check(load().uf_probe_l2_atomics(int(nbytes), ctypes.byref(rate)))
    return rate.value


def uf_compute_noalloc(tree: Tree, table: Table, method: str, alpha: float = 1.0,
                       precision: str = "fp64", out=None, stream=None):
    """Full-range condensed distances without any device allocation by the
    library: for callers that may not allocate device memory (their own
    memory manager owns the device heap, or the allocator may not be entered
    at that point).  ``out`` must be a CUDA float64 tensor of n(n-1)/2
    elements, written in place; the library works in its fixed 64 MiB area and
    raises UF_ENOMEM for problems that do not fit.  Returns ``out``."""
    import torch
    n = table.n_samples
    need = condensed_size(n)
    if out is None or not hasattr(out, "data_ptr") or not out.is_cuda:
        raise ValueError("out must be a CUDA torch tensor (device memory owned by the caller)")
    if out.dtype != torch.float64 or not out.is_contiguous() or out.numel() < need:
        raise ValueError(f"out must be a contiguous float64 tensor with >= {need} elements")
    st = int(stream) if stream is not None else torch.cuda.current_stream(out.device).cuda_stream
    m_code, p_code = _code_of(METHODS, method, "method"), _code_of(PRECISIONS, precision, "precision")
    with _on_device_of(out):
        _check(load().uf_compute_noalloc(tree.handle, table.handle, m_code, float(alpha),
                                         p_code, ctypes.c_void_p(out.data_ptr()),
                                         ctypes.c_void_p(st) if st else None))
    return out
