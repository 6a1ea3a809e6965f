"""Seeded synthetic workloads: Yule trees and sparse sample-by-feature tables.

This module only draws random inputs.  It holds none of the UniFrac
arithmetic, so both the CUDA path's tests and the oracle's tests may use it.

Trees (the recipe used for every workload):
  1. start from a root with two tips;
  2. repeatedly pick a uniformly random current tip and give it two children
     until there are ``n_tips`` tips;
  3. draw every branch length iid from an exponential with mean 0.1 (FP64);
  4. relabel the nodes in postorder, visiting children in creation order;
     tips take feature ids in the order they appear in that postorder.
The result is a parent array with ``parent[i] > i`` and the root last.

Tables are CSR with samples as rows and columns sorted, one column per tip.
Counts are ``1 + Poisson(lam)`` with ``lam ~ LogNormal(1, 1)`` per nonzero,
or ``max(1, round(LogNormal(1, 1.5)))`` for the heavy-tailed workloads.  A
sample left without any nonzero gets one uniformly random feature with
count 1.  All draws use numpy's PCG64 with the seeds listed in ``WORKLOADS``.
"""
from __future__ import annotations

import dataclasses
import hashlib
import os

import numpy as np

__all__ = ["Tree", "Table", "yule_tree", "table_iid", "table_prevalence", "pair_subset",
           "WORKLOADS", "workload", "batched_workload", "stripe_pairs_bruteforce"]


@dataclasses.dataclass
class Tree:
    parent: np.ndarray  # int64 [n_nodes], parent[i] > i, root = last node with -1
    length: np.ndarray  # float64 [n_nodes], length of the branch above each node

    @property
    def n_nodes(self) -> int:
        return int(self.parent.shape[0])

    @property
    def n_tips(self) -> int:
        has_child = np.zeros(self.n_nodes, dtype=bool)
        has_child[self.parent[:-1]] = True
        return int((~has_child).sum())


@dataclasses.dataclass
class Table:
    n_samples: int
    n_features: int
    indptr: np.ndarray   # int64 [n_samples + 1]
    indices: np.ndarray  # int32 [nnz]
    data: np.ndarray     # float64 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.indptr[-1])

    def dense(self) -> np.ndarray:
        out = np.zeros((self.n_samples, self.n_features), dtype=np.float64)
        rows = np.repeat(np.arange(self.n_samples), np.diff(self.indptr))
        out[rows, self.indices] = self.data
        return out

    @staticmethod
    def from_dense(counts: np.ndarray) -> "Table":
        counts = np.asarray(counts, dtype=np.float64)
        n, f = counts.shape
        rows, cols = np.nonzero(counts)
        indptr = np.zeros(n + 1, dtype=np.int64)
        np.cumsum(np.bincount(rows, minlength=n), out=indptr[1:])
        return Table(n, f, indptr, cols.astype(np.int32), counts[rows, cols].astype(np.float64))

    def digest(self) -> str:
        h = hashlib.sha256()
        for a in (self.indptr, self.indices, self.data):
            h.update(np.ascontiguousarray(a).tobytes())
        return h.hexdigest()[:16]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def yule_tree(n_tips: int, seed: int, mean_length: float = 0.1) -> Tree:
    """Seeded Yule tree with ``n_tips`` tips in postorder (see module doc)."""
    if n_tips < 2:
        raise ValueError("a Yule tree needs at least two tips")
    rng = _rng(seed)
    n_nodes = 2 * n_tips - 1
    left = [-1] * n_nodes
    right = [-1] * n_nodes
    left[0], right[0] = 1, 2
    tips = [1, 2]
    nxt = 3
    # one uniform per split picks which current tip splits
    picks = rng.random(n_tips - 2)
    for i in range(n_tips - 2):
        r = int(picks[i] * len(tips))
        t = tips[r]
        left[t], right[t] = nxt, nxt + 1
        tips[r] = nxt
        tips.append(nxt + 1)
        nxt += 2
    # postorder over creation ids, children in creation order
    order = []
    stack = [(0, False)]
    while stack:
        node, done = stack.pop()
        if done or left[node] < 0:
            order.append(node)
        else:
            stack.append((node, True))
            stack.append((right[node], False))
            stack.append((left[node], False))
    order_a = np.asarray(order, dtype=np.int64)
    new_id = np.empty(n_nodes, dtype=np.int64)
    new_id[order_a] = np.arange(n_nodes, dtype=np.int64)
    parent = np.full(n_nodes, -1, dtype=np.int64)
    left_a = np.asarray(left, dtype=np.int64)
    right_a = np.asarray(right, dtype=np.int64)
    internal = np.nonzero(left_a >= 0)[0]
    parent[new_id[left_a[internal]]] = new_id[internal]
    parent[new_id[right_a[internal]]] = new_id[internal]
    # the root's entry is drawn too; UniFrac ignores it (no branch above the root)
    length = rng.exponential(mean_length, size=n_nodes).astype(np.float64)
    return Tree(parent, length)


def _counts(rng: np.random.Generator, m: int, heavy: bool) -> np.ndarray:
    if heavy:
        return np.maximum(1.0, np.round(rng.lognormal(1.0, 1.5, size=m)))
    lam = rng.lognormal(1.0, 1.0, size=m)
    return 1.0 + rng.poisson(lam).astype(np.float64)


def _to_csr(n: int, f: int, rows: np.ndarray, cols: np.ndarray, vals: np.ndarray,
            rng: np.random.Generator) -> Table:
    present = np.zeros(n, dtype=bool)
    present[rows] = True
    empty = np.nonzero(~present)[0]
    if empty.size:
        rows = np.concatenate([rows, empty])
        cols = np.concatenate([cols, rng.integers(0, f, size=empty.size)])
        vals = np.concatenate([vals, np.ones(empty.size)])
    key = rows.astype(np.int64) * f + cols.astype(np.int64)
    order = np.argsort(key, kind="stable")
    rows, cols, vals = rows[order], cols[order], vals[order]
    indptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=indptr[1:])
    return Table(n, f, indptr, cols.astype(np.int32), vals.astype(np.float64))


def table_iid(n_samples: int, n_features: int, density: float, seed: int,
              heavy: bool = False) -> Table:
    """Every (sample, feature) is nonzero independently with ``density``."""
    rng = _rng(seed)
    per_row = rng.binomial(n_features, density, size=n_samples)
    rows, cols = [], []
    for k in range(n_samples):
        m = int(per_row[k])
        if m:
            c = rng.choice(n_features, size=m, replace=False)
            cols.append(np.asarray(c, dtype=np.int64))
            rows.append(np.full(m, k, dtype=np.int64))
    rows_a = np.concatenate(rows) if rows else np.zeros(0, np.int64)
    cols_a = np.concatenate(cols) if cols else np.zeros(0, np.int64)
    vals = _counts(rng, rows_a.size, heavy)
    return _to_csr(n_samples, n_features, rows_a, cols_a, vals, rng)


def table_prevalence(n_samples: int, n_features: int, beta_a: float, beta_b: float,
                     seed: int, heavy: bool = False) -> Table:
    """Feature f has prevalence ``p_f ~ Beta(a, b)``; each sample holds f
    independently with probability ``p_f``."""
    rng = _rng(seed)
    prev = rng.beta(beta_a, beta_b, size=n_features)
    per_col = rng.binomial(n_samples, prev)
    rows, cols = [], []
    for f in np.nonzero(per_col)[0]:
        m = int(per_col[f])
        r = rng.choice(n_samples, size=m, replace=False)
        rows.append(np.asarray(r, dtype=np.int64))
        cols.append(np.full(m, f, dtype=np.int64))
    rows_a = np.concatenate(rows) if rows else np.zeros(0, np.int64)
    cols_a = np.concatenate(cols) if cols else np.zeros(0, np.int64)
    vals = _counts(rng, rows_a.size, heavy)
    return _to_csr(n_samples, n_features, rows_a, cols_a, vals, rng)


def pair_subset(n_samples: int, n_pairs: int, seed: int = 12345):
    """``n_pairs`` distinct pairs i < j drawn uniformly without replacement
    (all pairs, in row-major order, when there are no more than that)."""
    total = n_samples * (n_samples - 1) // 2
    if total <= n_pairs:
        i, j = np.triu_indices(n_samples, k=1)
        return i.astype(np.int64), j.astype(np.int64)
    rng = _rng(seed)
    picked = np.unique(rng.integers(0, total, size=int(n_pairs * 1.3) + 16))
    while picked.size < n_pairs:
        picked = np.unique(np.concatenate([picked, rng.integers(0, total, size=n_pairs)]))
    picked = rng.permutation(picked)[:n_pairs]
    picked.sort()
    # condensed index -> (i, j), row-major upper triangle
    n = n_samples
    i = (n - 2 - np.floor(np.sqrt(-8.0 * picked + 4.0 * n * (n - 1) - 7) / 2.0 - 0.5)).astype(np.int64)
    start = n * i - i * (i + 1) // 2
    # guard the float estimate
    over = start > picked
    while over.any():
        i[over] -= 1
        start = n * i - i * (i + 1) // 2
        over = start > picked
    nxt = n * (i + 1) - (i + 1) * (i + 2) // 2
    under = nxt <= picked
    while under.any():
        i[under] += 1
        start = n * i - i * (i + 1) // 2
        nxt = n * (i + 1) - (i + 1) * (i + 2) // 2
        under = nxt <= picked
    j = picked - start + i + 1
    return i, j


def stripe_pairs_bruteforce(n: int):
    """Every (stripe s, column k) cell of the full stripe set with its pair
    (k, (k + s + 1) mod n): a plain enumeration used to check layouts."""
    cells = []
    for s in range(n // 2):
        for k in range(n):
            cells.append((s, k, k, (k + s + 1) % n))
    return cells


# workload name -> (tree tips, tree seed, table factory)
WORKLOADS = {
    # 1,024 tips, 64 samples, 10% iid nonzeros
    "yule1k_n64": dict(tips=1024, tree_seed=1, table=lambda t: table_iid(64, t, 0.10, seed=2)),
    # 50,000 tips, 2,048 samples, prevalence Beta(0.5, 20)
    "yule50k_n2048": dict(tips=50_000, tree_seed=3,
                          table=lambda t: table_prevalence(2048, t, 0.5, 20.0, seed=4)),
    # EMP-shaped: 300,000 tips, 25,000 samples, prevalence Beta(0.1, 19.9), heavy counts
    "yule300k_n25000": dict(tips=300_000, tree_seed=5,
                            table=lambda t: table_prevalence(25_000, t, 0.1, 19.9, seed=6, heavy=True)),
    # 113k-shaped: 500,000 tips, 113,000 samples, prevalence Beta(0.06, 19.94), heavy counts
    "yule500k_n113000": dict(tips=500_000, tree_seed=9,
                             table=lambda t: table_prevalence(113_000, t, 0.06, 19.94, seed=10, heavy=True)),
}


def _cache_dir() -> str:
    # generated workloads are cached beside this module (UF_SYNTH_CACHE overrides)
    d = os.environ.get("UF_SYNTH_CACHE", os.path.join(os.path.dirname(os.path.abspath(__file__)), "_cache"))
    os.makedirs(d, exist_ok=True)
    return d


def workload(name: str, cache: bool = True):
    """(Tree, Table) of a named workload, cached on disk by name."""
    spec = WORKLOADS[name]
    path = os.path.join(_cache_dir(), f"{name}.npz")
    if cache and os.path.exists(path):
        z = np.load(path)
        tree = Tree(z["parent"], z["length"])
        table = Table(int(z["n"]), int(z["f"]), z["indptr"], z["indices"], z["data"])
        return tree, table
    tree = yule_tree(spec["tips"], spec["tree_seed"])
    table = spec["table"](tree.n_tips)
    if cache:
        tmp = path + f".{os.getpid()}.tmp.npz"
        np.savez(tmp, parent=tree.parent, length=tree.length, n=table.n_samples,
                 f=table.n_features, indptr=table.indptr, indices=table.indices, data=table.data)
        os.replace(tmp, path)
    return tree, table


def batched_workload(n_tables: int = 64, tips: int = 100_000, lo: int = 200, hi: int = 5000,
                     density: float = 0.01):
    """Many independent tables of uneven sample counts over one shared tree:
    sample counts uniform on [lo, hi], iid nonzeros at ``density``; tree seed
    7, table t seed 8 + t, sample counts drawn with seed 7."""
    tree = yule_tree(tips, 7)
    sizes = _rng(7).integers(lo, hi + 1, size=n_tables)
    tables = [table_iid(int(sizes[t]), tree.n_tips, density, seed=8 + t) for t in range(n_tables)]
    return tree, tables
