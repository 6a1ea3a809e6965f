"""Pins for the FP64 oracle: facts fixed by the mathematics, not by the oracle.

Every check here is independent of ``oracle/uf_oracle.c``'s own code:
closed forms on two- and three-tip trees, textbook distances that UniFrac
reduces to on star trees, an independent root-path enumeration, weighted
unnormalized as an earth mover's distance (a transport LP), hand-worked
values (tests/golden/hand_small.txt) and invariants of the metric family.
The definitions are those of the paper's refs [1] and [3] (Sec. 1); the
paper prints no formula, so the readings are stated in the oracle header.
"""
import math
import os

import numpy as np
import pytest

import oracle
from synth import Table, Tree, table_iid, yule_tree

METHODS = ["unweighted", "weighted_unnormalized", "weighted_normalized", "generalized"]
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _pair(tree, table, method, alpha, i, j, lib=None):
    return oracle.pairs(tree, table, method, alpha, [i], [j], lib=lib)[0][0]


def two_tip_tree(a, b):
    # tips 0 and 1 under the root 2; the root's length must be ignored
    return Tree(np.array([2, 2, -1], dtype=np.int64), np.array([a, b, 0.77]))


def star_tree(n_tips, lengths=None):
    parent = np.full(n_tips + 1, n_tips, dtype=np.int64)
    parent[-1] = -1
    length = np.ones(n_tips + 1) if lengths is None else np.append(np.asarray(lengths, float), 0.0)
    length[-1] = 0.5  # ignored: no branch above the root
    return Tree(parent, length)


# ---------------------------------------------------------------- closed forms

def check_two_tip(lib=None, seed=0):
    rng = np.random.default_rng(seed)
    for _ in range(20):
        a, b = rng.uniform(0.05, 3.0, size=2)
        cx, cy = rng.integers(1, 50, size=2), rng.integers(1, 50, size=2)
        table = Table.from_dense(np.array([cx, cy], dtype=float))
        x, y = cx[0] / cx.sum(), cy[0] / cy.sum()
        alpha = float(rng.uniform(0.0, 1.0))
        s1, s2 = x + y, 2.0 - x - y
        exp = {
            "weighted_unnormalized": (a + b) * abs(x - y),
            "weighted_normalized": (a + b) * abs(x - y) / (a * (x + y) + b * (2 - x - y)),
            "generalized": abs(x - y) * (a * s1 ** (alpha - 1) + b * s2 ** (alpha - 1))
            / (a * s1 ** alpha + b * s2 ** alpha),
            "unweighted": 0.0,  # both samples hold both tips
        }
        tree = two_tip_tree(a, b)
        for m, e in exp.items():
            got = _pair(tree, table, m, alpha, 0, 1, lib)
            assert got == pytest.approx(e, rel=1e-13, abs=1e-15), (m, got, e)
        # presence: {A} vs {B} -> 1; {A} vs {A, B} -> b / (a + b)
        t2 = Table.from_dense(np.array([[3.0, 0.0], [0.0, 5.0], [2.0, 7.0]]))
        assert _pair(tree, t2, "unweighted", 0, 0, 1, lib) == pytest.approx(1.0, rel=1e-15)
        assert _pair(tree, t2, "unweighted", 0, 0, 2, lib) == pytest.approx(b / (a + b), rel=1e-14)


def test_two_tip_closed_forms():
    check_two_tip()


def check_three_tip(lib=None, seed=1):
    # ((A:a, B:b):c, C:e): unnormalized = a|dA| + b|dB| + c|dA + dB| + e|dC|
    rng = np.random.default_rng(seed)
    for _ in range(20):
        a, b, c, e = rng.uniform(0.05, 2.0, size=4)
        tree = Tree(np.array([2, 2, 4, 4, -1], dtype=np.int64), np.array([a, b, c, e, 1.3]))
        counts = rng.integers(0, 20, size=(2, 3)).astype(float)
        counts[:, 0] += 1
        table = Table.from_dense(counts)
        p = counts / counts.sum(axis=1, keepdims=True)
        d = p[0] - p[1]
        exp = a * abs(d[0]) + b * abs(d[1]) + c * abs(d[0] + d[1]) + e * abs(d[2])
        got = _pair(tree, table, "weighted_unnormalized", 0, 0, 1, lib)
        assert got == pytest.approx(exp, rel=1e-13, abs=1e-15)
        den = a * (p[0, 0] + p[1, 0]) + b * (p[0, 1] + p[1, 1]) + c * (p[0, 0] + p[0, 1] + p[1, 0] + p[1, 1]) \
            + e * (p[0, 2] + p[1, 2])
        got = _pair(tree, table, "weighted_normalized", 0, 0, 1, lib)
        assert got == pytest.approx(exp / den, rel=1e-13, abs=1e-15)


def test_three_tip_closed_form():
    check_three_tip()


# ----------------------------------------------------------- textbook cases

def check_star_textbook(lib=None, seed=2):
    rng = np.random.default_rng(seed)
    n_tips, n = 12, 9
    counts = rng.integers(0, 6, size=(n, n_tips)).astype(float) * (rng.random((n, n_tips)) < 0.5)
    counts[:, 0] += 1.0
    counts[3] = counts[4]        # two identical samples
    table = Table.from_dense(counts)
    tree = star_tree(n_tips)
    p = counts / counts.sum(axis=1, keepdims=True)
    pres = counts > 0
    for i in range(n):
        for j in range(i + 1, n):
            inter = np.logical_and(pres[i], pres[j]).sum()
            union = np.logical_or(pres[i], pres[j]).sum()
            jaccard = 1.0 - inter / union
            l1 = np.abs(p[i] - p[j]).sum()
            bray = np.abs(counts[i] / counts[i].sum() - counts[j] / counts[j].sum()).sum() / 2.0
            # Canberra distance of the relative abundances (0/0 terms dropped)
            both = pres[i] | pres[j]
            canberra = (np.abs(p[i] - p[j])[both] / (p[i] + p[j])[both]).sum()
            assert _pair(tree, table, "unweighted", 0, i, j, lib) == pytest.approx(jaccard, rel=1e-14, abs=1e-16)
            assert _pair(tree, table, "weighted_unnormalized", 0, i, j, lib) == pytest.approx(l1, rel=1e-13, abs=1e-16)
            assert _pair(tree, table, "weighted_normalized", 0, i, j, lib) == pytest.approx(bray, rel=1e-13, abs=1e-16)
            assert _pair(tree, table, "generalized", 1.0, i, j, lib) == pytest.approx(bray, rel=1e-13, abs=1e-16)
            # generalized(0) weighs every present branch equally: Canberra over the union's size
            assert _pair(tree, table, "generalized", 0.0, i, j, lib) == pytest.approx(
                canberra / union, rel=1e-13, abs=1e-16)


def test_star_tree_textbook_distances():
    check_star_textbook()


def test_star_tree_against_scipy():
    spatial = pytest.importorskip("scipy.spatial.distance")
    rng = np.random.default_rng(3)
    counts = rng.integers(0, 9, size=(6, 10)).astype(float)
    counts[:, 1] += 1
    table = Table.from_dense(counts)
    tree = star_tree(10)
    p = counts / counts.sum(axis=1, keepdims=True)
    for i in range(6):
        for j in range(i + 1, 6):
            assert _pair(tree, table, "unweighted", 0, i, j) == pytest.approx(
                spatial.jaccard(counts[i] > 0, counts[j] > 0), rel=1e-14)
            assert _pair(tree, table, "weighted_normalized", 0, i, j) == pytest.approx(
                spatial.braycurtis(p[i], p[j]), rel=1e-13)
            assert _pair(tree, table, "weighted_unnormalized", 0, i, j) == pytest.approx(
                spatial.cityblock(p[i], p[j]), rel=1e-13)
            union = np.logical_or(counts[i] > 0, counts[j] > 0).sum()
            assert _pair(tree, table, "generalized", 0.0, i, j) == pytest.approx(
                spatial.canberra(p[i], p[j]) / union, rel=1e-13)


# --------------------------------------------------- independent formulation

def path_enumeration(tree, table, method, alpha, i, j):
    """UniFrac from root paths: a tip's path lists the branches to the root;
    a sample's mass on a branch sums over the tips whose path uses it."""
    parent = tree.parent
    n_nodes = parent.size
    has_child = np.zeros(n_nodes, bool)
    has_child[parent[:-1]] = True
    tips = np.nonzero(~has_child)[0]
    counts = table.dense()
    mass = [dict(), dict()]
    for side, k in enumerate((i, j)):
        tot = counts[k].sum()
        for f, node in enumerate(tips):
            c = counts[k, f]
            if c == 0:
                continue
            v = node
            while parent[v] != -1:
                mass[side][v] = mass[side].get(v, 0.0) + c / tot
                v = parent[v]
    num = den = 0.0
    for v in range(n_nodes - 1):
        l = tree.length[v]
        a, b = mass[0].get(v, 0.0), mass[1].get(v, 0.0)
        pa, pb = v in mass[0], v in mass[1]
        if method == "unweighted":
            num += l * (pa != pb)
            den += l * (pa or pb)
        elif method in ("weighted_unnormalized", "weighted_normalized"):
            num += l * abs(a - b)
            den += l * (a + b)
        else:
            s = a + b
            if s > 0:
                num += l * s ** alpha * abs(a - b) / s
                den += l * s ** alpha
    if method == "weighted_unnormalized":
        return num
    return 0.0 if den == 0 else num / den


def random_small_tree(rng, n_tips, unary=0, zero_len=0):
    """Random topology with optional unary nodes and zero-length branches,
    in an arbitrary children-before-parents order."""
    # build by random merges, then relabel by a random topological order
    nodes = list(range(n_tips))
    parent = {}
    nxt = n_tips
    while len(nodes) > 1:
        a, b = rng.choice(len(nodes), 2, replace=False)
        x, y = nodes[a], nodes[b]
        parent[x] = nxt
        parent[y] = nxt
        nodes = [z for t, z in enumerate(nodes) if t not in (a, b)] + [nxt]
        nxt += 1
    root = nodes[0]
    for _ in range(unary):
        cands = [v for v in parent]
        v = cands[rng.integers(len(cands))]
        parent[nxt] = parent[v]
        parent[v] = nxt
        nxt += 1
    total = nxt
    parent[root] = -1
    # topological order children-before-parents with random tie breaks
    children = {v: [] for v in range(total)}
    for v, p in parent.items():
        if p != -1:
            children[p].append(v)
    order = []
    pending = {v: len(children[v]) for v in range(total)}
    ready = [v for v in range(total) if pending[v] == 0]
    while ready:
        v = ready.pop(rng.integers(len(ready)))
        order.append(v)
        p = parent[v]
        if p != -1:
            pending[p] -= 1
            if pending[p] == 0:
                ready.append(p)
    new = {v: t for t, v in enumerate(order)}
    par = np.array([new[parent[v]] if parent[v] != -1 else -1 for v in order], dtype=np.int64)
    length = rng.exponential(0.3, size=total)
    zl = rng.choice(total - 1, size=min(zero_len, total - 1), replace=False)
    length[zl] = 0.0
    return Tree(par, length)


def random_table_for(rng, tree, n, density=0.4):
    f = tree.n_tips
    counts = rng.integers(1, 9, size=(n, f)).astype(float) * (rng.random((n, f)) < density)
    for k in range(n):
        if counts[k].sum() == 0:
            counts[k, rng.integers(f)] = 1.0
    return Table.from_dense(counts)


def check_path_enumeration(lib=None, seed=4, cases=12):
    rng = np.random.default_rng(seed)
    for c in range(cases):
        tree = random_small_tree(rng, int(rng.integers(2, 14)), unary=int(rng.integers(0, 3)),
                                 zero_len=int(rng.integers(0, 3)))
        table = random_table_for(rng, tree, int(rng.integers(2, 7)))
        alpha = float(rng.choice([0.0, 0.5, 1.0, rng.uniform()]))
        n = table.n_samples
        ii, jj = np.triu_indices(n, 1)
        for m in METHODS:
            got = oracle.pairs(tree, table, m, alpha, ii, jj, lib=lib)[0]
            exp = np.array([path_enumeration(tree, table, m, alpha, a, b) for a, b in zip(ii, jj)])
            assert np.allclose(got, exp, rtol=1e-14, atol=1e-14), (c, m, got, exp)


def test_path_enumeration_matches():
    check_path_enumeration()


# ----------------------------------------------------- earth mover's distance

def tip_path_distances(tree):
    """Path length between every two tips: the smallest sum of the two climbs
    to a common ancestor (the lowest one; ties only through zero lengths).
    A climb from u adds the length of the branch above each node it leaves,
    so the root's length never enters."""
    n = tree.n_nodes
    has_child = np.zeros(n, bool)
    has_child[tree.parent[:-1]] = True
    tips = np.nonzero(~has_child)[0]
    climbs = []
    for u in tips:
        up, d, v = {int(u): 0.0}, 0.0, int(u)
        while tree.parent[v] != -1:
            d += tree.length[v]
            v = int(tree.parent[v])
            up[v] = d
        climbs.append(up)
    T = len(tips)
    D = np.zeros((T, T))
    for f in range(T):
        for g in range(T):
            common = climbs[f].keys() & climbs[g].keys()
            D[f, g] = min(climbs[f][a] + climbs[g][a] for a in common)
    return D


def has_children(tree):
    has = np.zeros(tree.n_nodes, bool)
    has[tree.parent[:-1]] = True
    return has


def tree_depth(tree, u):
    """Sum of the lengths of the branches from node u up to the root."""
    d = 0.0
    while tree.parent[u] != -1:
        d += tree.length[u]
        u = int(tree.parent[u])
    return d


def earth_movers(D, p, q):
    """Earth mover's distance between tip distributions p and q under the
    ground distance D: the cheapest transport plan, as a linear program."""
    linprog = pytest.importorskip("scipy.optimize").linprog
    src, dst = np.nonzero(p)[0], np.nonzero(q)[0]
    a, b = len(src), len(dst)
    A = np.zeros((a + b, a * b))
    for r in range(a):
        A[r, r * b:(r + 1) * b] = 1.0      # all of p[src[r]] leaves
    for c in range(b):
        A[a + c, c::b] = 1.0               # all of q[dst[c]] arrives
    res = linprog(D[np.ix_(src, dst)].ravel(), A_eq=A, b_eq=np.concatenate([p[src], q[dst]]),
                  bounds=(0, None), method="highs")
    assert res.status == 0, res.message
    return res.fun


def check_earth_movers(lib=None, seed=8, cases=10):
    # weighted unnormalized UniFrac is the earth mover's distance between the
    # two samples' relative abundances over the tips, with path length on the
    # tree as the ground distance: a transport LP with no tree walk at all
    rng = np.random.default_rng(seed)
    for c in range(cases):
        tree = random_small_tree(rng, int(rng.integers(2, 12)), unary=int(rng.integers(0, 3)),
                                 zero_len=int(rng.integers(0, 3)))
        f = tree.n_tips
        counts = rng.integers(1, 9, size=(4, f)).astype(float) * (rng.random((4, f)) < 0.5)
        for k in range(4):
            if counts[k].sum() == 0:
                counts[k, rng.integers(f)] = 1.0
        table = Table.from_dense(counts)
        P = counts / counts.sum(axis=1, keepdims=True)
        D = tip_path_distances(tree)
        ii, jj = np.triu_indices(4, 1)
        got = oracle.pairs(tree, table, "weighted_unnormalized", 0.0, ii, jj, lib=lib)[0]
        for g, a, b in zip(got, ii, jj):
            exp = earth_movers(D, P[a], P[b])
            assert g == pytest.approx(exp, rel=1e-8, abs=1e-10), (c, a, b, g, exp)
        # the normalized denominator separates into per-sample terms: each
        # tip's relative abundance times its depth (its climb to the root)
        depth = np.array([tree_depth(tree, int(u)) for u in np.nonzero(~has_children(tree))[0]])
        den = oracle.pairs(tree, table, "weighted_normalized", 0.0, ii, jj, lib=lib)[2]
        exp = (P[ii] + P[jj]) @ depth
        assert np.allclose(den, exp, rtol=1e-13, atol=1e-15), (c, den, exp)


def test_earth_movers_distance():
    check_earth_movers()


# ------------------------------------------------------------- hand-worked

def load_hand_small():
    tree = Tree(np.array([2, 2, 4, 4, -1], dtype=np.int64), np.array([1.0, 2.0, 3.0, 4.0, 5.0]))
    table = Table.from_dense(np.array([[1.0, 1.0, 2.0], [3.0, 0.0, 1.0], [0.0, 2.0, 0.0]]))
    rows = []
    with open(os.path.join(GOLDEN, "hand_small.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split(None, 4)
            rows.append((parts[0], float(parts[1]), int(parts[2]), int(parts[3]),
                         eval(parts[4], {"sqrt": math.sqrt})))
    return tree, table, rows


def check_hand_small(lib=None):
    tree, table, rows = load_hand_small()
    for method, alpha, i, j, exp in rows:
        got = _pair(tree, table, method, alpha, i, j, lib)
        assert got == pytest.approx(exp, rel=1e-14), (method, alpha, i, j, got, exp)


def test_hand_worked_values():
    check_hand_small()


def check_zero_lengths(lib=None):
    # every branch of length zero: den == 0 for every pair, so d == 0
    tree = Tree(np.array([2, 2, 4, 4, -1], dtype=np.int64), np.zeros(5))
    table = Table.from_dense(np.array([[1.0, 0.0, 2.0], [0.0, 3.0, 1.0]]))
    for m in METHODS:
        assert _pair(tree, table, m, 0.5, 0, 1, lib) == 0.0
    # a zero-length branch contributes nothing: (A:0, B:b) two-tip tree
    tree = two_tip_tree(0.0, 2.0)
    t2 = Table.from_dense(np.array([[3.0, 0.0], [0.0, 5.0], [2.0, 7.0]]))
    assert _pair(tree, t2, "unweighted", 0, 0, 1, lib) == 1.0
    assert _pair(tree, t2, "unweighted", 0, 0, 2, lib) == pytest.approx(1.0, rel=1e-15)


def test_zero_lengths():
    check_zero_lengths()


# --------------------------------------------------------------- invariants

def check_invariants(lib=None, seed=5):
    rng = np.random.default_rng(seed)
    tree = yule_tree(40, seed=11)
    tbl = table_iid(10, tree.n_tips, 0.3, seed=12)
    counts = tbl.dense()
    counts[7] = counts[2]  # an identical pair
    table = Table.from_dense(counts)
    n = table.n_samples
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    ii, jj = ii.ravel(), jj.ravel()
    for m in METHODS:
        for alpha in ([0.0, 0.5, 1.0] if m == "generalized" else [0.0]):
            D = oracle.pairs(tree, table, m, alpha, ii, jj, lib=lib)[0].reshape(n, n)
            assert np.all(np.diag(D) == 0.0)
            assert np.array_equal(D, D.T)
            assert D[2, 7] == 0.0
            assert np.all(D >= 0)
            if m != "weighted_unnormalized":
                assert np.all(D <= 1.0 + 1e-15)
            if m in ("unweighted", "weighted_unnormalized"):
                for a in range(n):
                    for b in range(n):
                        assert np.all(D[a, b] <= D[a, :] + D[:, b] + 1e-12)
            # permuting samples permutes the matrix
            perm = rng.permutation(n)
            Dp = oracle.pairs(tree, Table.from_dense(counts[perm]), m, alpha, ii, jj, lib=lib)[0].reshape(n, n)
            assert np.allclose(Dp, D[np.ix_(perm, perm)], rtol=1e-14, atol=1e-15)
            # scaling one sample's counts changes nothing
            c2 = counts.copy()
            c2[4] *= 3.0
            Ds = oracle.pairs(tree, Table.from_dense(c2), m, alpha, ii, jj, lib=lib)[0].reshape(n, n)
            assert np.allclose(Ds, D, rtol=1e-13, atol=1e-15)
            # scaling every length by c scales unnormalized by c, the rest not at all
            t2 = Tree(tree.parent, tree.length * 2.5)
            Dl = oracle.pairs(t2, table, m, alpha, ii, jj, lib=lib)[0].reshape(n, n)
            factor = 2.5 if m == "weighted_unnormalized" else 1.0
            assert np.allclose(Dl, D * factor, rtol=1e-13, atol=1e-15)


def test_invariants():
    check_invariants()


def subdivide(tree, v, frac):
    """Insert a unary node on the branch above v, splitting its length."""
    n = tree.n_nodes
    # new node goes right after v in the order: indices > v shift by one
    parent = np.empty(n + 1, dtype=np.int64)
    length = np.empty(n + 1)
    remap = np.arange(n) + (np.arange(n) > v)
    for u in range(n):
        p = tree.parent[u]
        parent[remap[u]] = -1 if p == -1 else remap[p]
        length[remap[u]] = tree.length[u]
    parent[v] = v + 1
    length[v] = tree.length[v] * frac
    parent[v + 1] = remap[tree.parent[v]]
    length[v + 1] = tree.length[v] * (1 - frac)
    return Tree(parent, length)


def check_structural(lib=None, seed=6):
    rng = np.random.default_rng(seed)
    tree = yule_tree(30, seed=13)
    table = table_iid(6, tree.n_tips, 0.3, seed=14)
    n = table.n_samples
    ii, jj = np.triu_indices(n, 1)
    for m in METHODS:
        alpha = 0.5
        D = oracle.pairs(tree, table, m, alpha, ii, jj, lib=lib)[0]
        # a unary node splitting a branch changes nothing
        for v in rng.choice(tree.n_nodes - 1, size=4, replace=False):
            D2 = oracle.pairs(subdivide(tree, int(v), 0.3), table, m, alpha, ii, jj, lib=lib)[0]
            assert np.allclose(D2, D, rtol=1e-13, atol=1e-15)
    # generalized(alpha = 1) is weighted normalized
    a = oracle.pairs(tree, table, "generalized", 1.0, ii, jj, lib=lib)[0]
    b = oracle.pairs(tree, table, "weighted_normalized", 0.0, ii, jj, lib=lib)[0]
    assert np.allclose(a, b, rtol=1e-13, atol=1e-15)
    # generalized(alpha = 0) has the unweighted denominator: sum of l over s > 0
    g0 = oracle.pairs(tree, table, "generalized", 0.0, ii, jj, lib=lib)[2]
    uw = oracle.pairs(tree, table, "unweighted", 0.0, ii, jj, lib=lib)[2]
    assert np.allclose(g0, uw, rtol=1e-14)


def test_structural_invariants():
    check_structural()


def prune(tree, keep_tip):
    """Drop the tips not in keep_tip and every internal node left childless."""
    n = tree.n_nodes
    has_child = np.zeros(n, bool)
    has_child[tree.parent[:-1]] = True
    tips = np.nonzero(~has_child)[0]
    alive = np.zeros(n, bool)
    alive[tips[keep_tip]] = True
    for v in range(n - 1):  # children before parents
        if alive[v]:
            alive[tree.parent[v]] = True
    new = np.cumsum(alive) - 1
    kept = np.nonzero(alive)[0]
    parent = np.array([new[tree.parent[v]] if tree.parent[v] != -1 else -1 for v in kept], np.int64)
    return Tree(parent, tree.length[kept].copy())


def test_removing_absent_tips():
    # tips absent from both samples (and the branches only they use) do not matter
    tree = yule_tree(40, seed=15)
    rng = np.random.default_rng(7)
    counts = rng.integers(1, 9, size=(2, tree.n_tips)).astype(float)
    absent = rng.random(tree.n_tips) < 0.5
    absent[0] = False
    counts[:, absent] = 0.0
    table = Table.from_dense(counts)
    small = prune(tree, ~absent)
    table_s = Table.from_dense(counts[:, ~absent])
    assert small.n_tips == int((~absent).sum())
    for m in METHODS:
        a = _pair(tree, table, m, 0.5, 0, 1)
        b = _pair(small, table_s, m, 0.5, 0, 1)
        assert a == pytest.approx(b, rel=1e-13)


# --------------------------------------------------------------- validation

def test_validation_codes():
    good = two_tip_tree(1.0, 2.0)
    t = Table.from_dense(np.array([[1.0, 2.0], [3.0, 0.0]]))
    assert oracle.check_tree(good) == "OK"
    assert oracle.check_tree(Tree(np.array([2, 2, 0]), np.ones(3))) == "ETREE"      # no root
    assert oracle.check_tree(Tree(np.array([2, 0, -1]), np.ones(3))) == "ETREE"     # parent < child
    assert oracle.check_tree(Tree(np.array([2, 2, -1]), np.array([1.0, -1.0, 0]))) == "ETREE"
    assert oracle.check_tree(Tree(np.array([2, 2, -1]), np.array([1.0, np.nan, 0]))) == "ETREE"
    assert oracle.check_table(good, t) == "OK"
    bad = Table(2, 2, np.array([0, 2, 2]), np.array([0, 1], np.int32), np.array([1.0, 1.0]))
    assert oracle.check_table(good, bad) == "ETABLE"  # empty sample
    bad = Table(1, 2, np.array([0, 2]), np.array([1, 0], np.int32), np.array([1.0, 1.0]))
    assert oracle.check_table(good, bad) == "ETABLE"  # unsorted indices
    bad = Table(1, 2, np.array([0, 1]), np.array([0], np.int32), np.array([-1.0]))
    assert oracle.check_table(good, bad) == "ETABLE"  # negative count
    bad = Table(1, 3, np.array([0, 1]), np.array([0], np.int32), np.array([1.0]))
    assert oracle.check_table(good, bad) == "ETABLE"  # features != tips
    with pytest.raises(oracle.OracleError):
        oracle.pairs(good, t, "generalized", 1.5, [0], [1])


# ------------------------------------------------------- striped vs pairwise

@pytest.mark.parametrize("n", [2, 3, 4, 5, 8, 9])
def test_striped_loop_matches_pairwise(n):
    tree = yule_tree(25, seed=21)
    table = table_iid(n, tree.n_tips, 0.3, seed=22 + n)
    S = n // 2
    for m in METHODS:
        _, _, dist, _ = oracle.striped(tree, table, m, 0.5, 0, S)
        for s in range(S):
            for k in range(n):
                j = (k + s + 1) % n
                exp = oracle.pairs(tree, table, m, 0.5, [min(k, j)], [max(k, j)])[0][0]
                assert dist[s, k] == pytest.approx(exp, rel=1e-13, abs=1e-15)
        # stripe ranges are independent subproblems
        if S >= 2:
            a = oracle.striped(tree, table, m, 0.5, 0, 1)[2]
            b = oracle.striped(tree, table, m, 0.5, 1, S)[2]
            assert np.array_equal(np.vstack([a, b]), dist)
