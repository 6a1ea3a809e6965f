"""Pins for the oracle's further Striped UniFrac family members.

The paper names the family (Sec. 1) without formulas.  The members built
here are unweighted unnormalized (the unweighted numerator alone) and the
variance-adjusted weighted UniFrac of Chang, Luan & Sun (BMC
Bioinformatics 12:118, 2011), unnormalized and normalized: each branch term
is divided by sqrt(m_v (m - m_v)), m_v the two samples' counts below v and m
their totals (branches with m_v = 0 or m_v = m add nothing; the readings
are stated in the oracle's header).  Every check is independent of the
oracle's code: closed forms on two- and three-tip trees, a symmetric
difference on a star tree, hand-worked values (tests/golden/hand_variants.txt),
an independent root-path enumeration and invariants.
"""
import math
import os

import numpy as np
import pytest

import oracle
from synth import Table, Tree, table_iid, yule_tree
from tests.test_oracle_pins import (_pair, random_small_tree, random_table_for, star_tree, subdivide,
                                    two_tip_tree)

VARIANTS = ["unweighted_unnormalized", "vaw_weighted_unnormalized", "vaw_weighted_normalized"]
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def check_variant_two_tip(lib=None, seed=30):
    rng = np.random.default_rng(seed)
    for _ in range(20):
        a, b = rng.uniform(0.05, 3.0, size=2)
        cx, cy = rng.integers(1, 50, size=2).astype(float), rng.integers(1, 50, size=2).astype(float)
        table = Table.from_dense(np.array([cx, cy]))
        x, y = cx[0] / cx.sum(), cy[0] / cy.sum()
        tree = two_tip_tree(a, b)
        # both branches have m_v (m - m_v) = (cx0 + cy0)(cx1 + cy1) and |dp| = |x - y|
        q = math.sqrt((cx[0] + cy[0]) * (cx[1] + cy[1]))
        assert _pair(tree, table, "vaw_weighted_unnormalized", 0, 0, 1, lib) == pytest.approx(
            (a + b) * abs(x - y) / q, rel=1e-13, abs=1e-16)
        # the common weight cancels: the normalized form is plain weighted normalized
        assert _pair(tree, table, "vaw_weighted_normalized", 0, 0, 1, lib) == pytest.approx(
            (a + b) * abs(x - y) / (a * (x + y) + b * (2 - x - y)), rel=1e-13, abs=1e-16)
        assert _pair(tree, table, "unweighted_unnormalized", 0, 0, 1, lib) == 0.0
        t2 = Table.from_dense(np.array([[3.0, 0.0], [0.0, 5.0], [2.0, 7.0]]))
        assert _pair(tree, t2, "unweighted_unnormalized", 0, 0, 1, lib) == pytest.approx(a + b, rel=1e-15)
        assert _pair(tree, t2, "unweighted_unnormalized", 0, 0, 2, lib) == pytest.approx(b, rel=1e-15)
        # {A} vs {B}: each branch holds all counts of one sample only, m_v (m - m_v) = T0 T1
        d = _pair(tree, t2, "vaw_weighted_unnormalized", 0, 0, 1, lib)
        assert d == pytest.approx((a + b) / math.sqrt(3.0 * 5.0), rel=1e-14)


def test_variant_two_tip_closed_forms():
    check_variant_two_tip()


def check_variant_three_tip(lib=None, seed=31):
    # ((A:a, B:b):c, C:e), counts X, Y: m_A, m_B, m_C, m_P = m_A + m_B, m = m_P + m_C
    rng = np.random.default_rng(seed)
    for _ in range(20):
        a, b, c, e = rng.uniform(0.05, 2.0, size=4)
        tree = Tree(np.array([2, 2, 4, 4, -1], dtype=np.int64), np.array([a, b, c, e, 1.3]))
        counts = rng.integers(1, 20, size=(2, 3)).astype(float)
        table = Table.from_dense(counts)
        T = counts.sum(axis=1)
        p = counts / T[:, None]
        m = T.sum()
        mA, mB, mC = counts.sum(axis=0)
        mP = mA + mB
        dA, dB, dC = p[0] - p[1]
        sA, sB, sC = p[0] + p[1]
        num = (a * abs(dA) / math.sqrt(mA * (m - mA)) + b * abs(dB) / math.sqrt(mB * (m - mB))
               + c * abs(dA + dB) / math.sqrt(mP * mC) + e * abs(dC) / math.sqrt(mC * (m - mC)))
        den = (a * sA / math.sqrt(mA * (m - mA)) + b * sB / math.sqrt(mB * (m - mB))
               + c * (sA + sB) / math.sqrt(mP * mC) + e * sC / math.sqrt(mC * (m - mC)))
        assert _pair(tree, table, "vaw_weighted_unnormalized", 0, 0, 1, lib) == pytest.approx(num, rel=1e-13)
        assert _pair(tree, table, "vaw_weighted_normalized", 0, 0, 1, lib) == pytest.approx(num / den, rel=1e-13)


def test_variant_three_tip_closed_form():
    check_variant_three_tip()


def check_variant_star(lib=None, seed=32):
    # star tree, unit lengths: unweighted unnormalized = size of the symmetric
    # difference of the two samples' feature sets
    rng = np.random.default_rng(seed)
    n_tips, n = 12, 8
    counts = rng.integers(0, 6, size=(n, n_tips)).astype(float) * (rng.random((n, n_tips)) < 0.5)
    counts[:, 0] += 1.0
    table = Table.from_dense(counts)
    tree = star_tree(n_tips)
    pres = counts > 0
    for i in range(n):
        for j in range(i + 1, n):
            sym = float(np.logical_xor(pres[i], pres[j]).sum())
            assert _pair(tree, table, "unweighted_unnormalized", 0, i, j, lib) == sym


def test_variant_star_symmetric_difference():
    check_variant_star()


def load_hand_variants():
    tree = Tree(np.array([2, 2, 4, 4, -1], dtype=np.int64), np.array([1.0, 2.0, 3.0, 4.0, 5.0]))
    table = Table.from_dense(np.array([[1.0, 1.0, 2.0], [3.0, 0.0, 1.0], [0.0, 2.0, 0.0], [1.0, 1.0, 0.0]]))
    rows = []
    with open(os.path.join(GOLDEN, "hand_variants.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split(None, 3)
            rows.append((parts[0], int(parts[1]), int(parts[2]), eval(parts[3], {"sqrt": math.sqrt})))
    return tree, table, rows


def check_hand_variants(lib=None):
    tree, table, rows = load_hand_variants()
    assert len(rows) == 9
    for method, i, j, exp in rows:
        got = _pair(tree, table, method, 0.0, i, j, lib)
        assert got == pytest.approx(exp, rel=1e-14), (method, i, j, got, exp)


def test_hand_worked_variant_values():
    check_hand_variants()


def path_enumeration_variant(tree, table, method, i, j):
    """The variants from root paths: a sample's count on a branch sums over
    the tips whose path to the root uses it."""
    parent = tree.parent
    n_nodes = parent.size
    has_child = np.zeros(n_nodes, bool)
    has_child[parent[:-1]] = True
    tips = np.nonzero(~has_child)[0]
    counts = table.dense()
    cnt = [dict(), dict()]
    for side, k in enumerate((i, j)):
        for f, node in enumerate(tips):
            c = counts[k, f]
            if c == 0:
                continue
            v = node
            while parent[v] != -1:
                cnt[side][v] = cnt[side].get(v, 0.0) + c
                v = parent[v]
    TA, TB = counts[i].sum(), counts[j].sum()
    num = den = 0.0
    for v in range(n_nodes - 1):
        l = tree.length[v]
        ca, cb = cnt[0].get(v, 0.0), cnt[1].get(v, 0.0)
        if method == "unweighted_unnormalized":
            num += l * ((ca > 0) != (cb > 0))
            continue
        mv, rest = ca + cb, TA + TB - ca - cb
        if mv > 0 and rest > 0:
            w = 1.0 / math.sqrt(mv * rest)
            num += l * w * abs(ca / TA - cb / TB)
            den += l * w * (ca / TA + cb / TB)
    if method != "vaw_weighted_normalized":
        return num
    return 0.0 if den == 0 else num / den


def check_variant_paths(lib=None, seed=33, cases=12):
    rng = np.random.default_rng(seed)
    for c in range(cases):
        tree = random_small_tree(rng, int(rng.integers(2, 14)), unary=int(rng.integers(0, 3)),
                                 zero_len=int(rng.integers(0, 3)))
        table = random_table_for(rng, tree, int(rng.integers(2, 7)))
        n = table.n_samples
        ii, jj = np.triu_indices(n, 1)
        for m in VARIANTS:
            got = oracle.pairs(tree, table, m, 0.0, ii, jj, lib=lib)[0]
            exp = np.array([path_enumeration_variant(tree, table, m, a, b) for a, b in zip(ii, jj)])
            assert np.allclose(got, exp, rtol=1e-13, atol=1e-15), (c, m, got, exp)


def test_variant_path_enumeration():
    check_variant_paths()


def check_variant_invariants(lib=None, seed=34):
    rng = np.random.default_rng(seed)
    tree = yule_tree(40, seed=35)
    counts = table_iid(10, tree.n_tips, 0.3, seed=36).dense()
    counts[7] = counts[2]
    table = Table.from_dense(counts)
    n = table.n_samples
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    ii, jj = ii.ravel(), jj.ravel()
    for m in VARIANTS:
        D = oracle.pairs(tree, table, m, 0.0, ii, jj, lib=lib)[0].reshape(n, n)
        assert np.all(np.diag(D) == 0.0) and np.array_equal(D, D.T) and D[2, 7] == 0.0
        assert np.all(D >= 0)
        if m == "vaw_weighted_normalized":
            assert np.all(D <= 1.0 + 1e-15)
        if m == "unweighted_unnormalized":  # a weighted Hamming distance on the branches
            for a in range(n):
                assert np.all(D[a, :][:, None] <= D[a, :][None, :] + D + 1e-12)
        perm = rng.permutation(n)
        Dp = oracle.pairs(tree, Table.from_dense(counts[perm]), m, 0.0, ii, jj, lib=lib)[0].reshape(n, n)
        assert np.allclose(Dp, D[np.ix_(perm, perm)], rtol=1e-14, atol=1e-15)
        # every length x c: both unnormalized forms x c, the normalized one unchanged
        Dl = oracle.pairs(Tree(tree.parent, tree.length * 2.5), table, m, 0.0, ii, jj, lib=lib)[0].reshape(n, n)
        assert np.allclose(Dl, D * (1.0 if m == "vaw_weighted_normalized" else 2.5), rtol=1e-13, atol=1e-15)
        # every sample's counts x c: m_v and m - m_v scale by c, so the weights by 1/c
        Dc = oracle.pairs(tree, Table.from_dense(counts * 4.0), m, 0.0, ii, jj, lib=lib)[0].reshape(n, n)
        factor = {"unweighted_unnormalized": 1.0, "vaw_weighted_unnormalized": 0.25,
                  "vaw_weighted_normalized": 1.0}[m]
        assert np.allclose(Dc, D * factor, rtol=1e-13, atol=1e-16)
        # a unary node splitting a branch changes nothing (both halves see the same m_v)
        iu, ju = np.triu_indices(n, 1)
        Du = oracle.pairs(tree, table, m, 0.0, iu, ju, lib=lib)[0]
        for v in rng.choice(tree.n_nodes - 1, size=3, replace=False):
            D2 = oracle.pairs(subdivide(tree, int(v), 0.4), table, m, 0.0, iu, ju, lib=lib)[0]
            assert np.allclose(D2, Du, rtol=1e-13, atol=1e-15)
    # unweighted unnormalized is the unweighted numerator
    iu, ju = np.triu_indices(n, 1)
    uu = oracle.pairs(tree, table, "unweighted_unnormalized", 0.0, iu, ju, lib=lib)[0]
    num = oracle.pairs(tree, table, "unweighted", 0.0, iu, ju, lib=lib)[1]
    assert np.allclose(uu, num, rtol=1e-15)


def test_variant_invariants():
    check_variant_invariants()


@pytest.mark.parametrize("n", [2, 3, 5, 8])
def test_variant_striped_loop_matches_pairwise(n):
    tree = yule_tree(25, seed=41)
    table = table_iid(n, tree.n_tips, 0.3, seed=42 + n)
    S = n // 2
    for m in VARIANTS:
        _, _, dist, _ = oracle.striped(tree, table, m, 0.0, 0, S)
        for s in range(S):
            for k in range(n):
                j = (k + s + 1) % n
                exp = oracle.pairs(tree, table, m, 0.0, [min(k, j)], [max(k, j)])[0][0]
                assert dist[s, k] == pytest.approx(exp, rel=1e-13, abs=1e-15)
