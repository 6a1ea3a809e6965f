"""Helpers shared by the GPU tests: tolerances and oracle comparison."""
import numpy as np

import oracle

METHODS = ["unweighted", "weighted_unnormalized", "weighted_normalized", "generalized"]
# further members of the family (unweighted unnormalized, variance-adjusted weighted)
VARIANTS = ["unweighted_unnormalized", "vaw_weighted_unnormalized", "vaw_weighted_normalized"]
# methods whose distance is an unbounded numerator: the mixed tolerance scales with max(1, |d|)
UNBOUNDED = ("weighted_unnormalized", "unweighted_unnormalized", "vaw_weighted_unnormalized")

# FP64 path: 1e-10 relative (exact zeros stay within 1e-15); mixed path: 1e-5
# absolute, scaled by max(1, |d|) for the unbounded (unnormalized) methods.
FP64_RTOL, FP64_ATOL = 1e-10, 1e-15
MIXED_ATOL = 1e-5


def tolerance_ok(got, exp, method, precision):
    got = np.asarray(got, dtype=np.float64)
    exp = np.asarray(exp, dtype=np.float64)
    if precision == "fp64":
        return np.abs(got - exp) <= FP64_RTOL * np.abs(exp) + FP64_ATOL
    scale = np.maximum(1.0, np.abs(exp)) if method in UNBOUNDED else 1.0
    return np.abs(got - exp) <= MIXED_ATOL * scale


# every comparison's errors, for the precision report printed after a run
# (tests/conftest.py): (what, method, precision, values, max_abs, max_rel,
# max_scaled, max_abs_at_zero)
PRECISION_LOG = []

# relative errors are reported only where the oracle's distance is at least
# this large; where it is exactly 0 (identical samples) the absolute error is
# reported in a column of its own
REL_FLOOR = 1e-12


def record_errors(got, exp, method, precision, what=""):
    got = np.asarray(got, dtype=np.float64)
    exp = np.asarray(exp, dtype=np.float64)
    if got.size == 0:
        return
    diff = np.abs(got - exp)
    big = np.abs(exp) >= REL_FLOOR
    rel = float((diff[big] / np.abs(exp[big])).max()) if big.any() else 0.0
    zero = exp == 0
    at_zero = float(diff[zero].max()) if zero.any() else 0.0
    scaled = diff / np.maximum(1.0, np.abs(exp))
    PRECISION_LOG.append((what, method, precision, int(got.size), float(diff.max()), rel,
                          float(scaled.max()), at_zero))


def precision_summary():
    """Lines of the precision report: per method and precision, the largest
    absolute, relative (where the oracle's |d| >= REL_FLOOR), max(1, |d|)-scaled
    error, and the largest absolute error where the oracle gives exactly 0."""
    agg = {}
    for _, method, precision, n, a, r, sc, z in PRECISION_LOG:
        v = agg.setdefault((method, precision), [0, 0, 0.0, 0.0, 0.0, 0.0])
        v[0] += 1
        v[1] += n
        v[2], v[3], v[4], v[5] = max(v[2], a), max(v[3], r), max(v[4], sc), max(v[5], z)
    lines = [f"{'method':<24}{'precision':<10}{'checks':>7}{'values':>12}{'max abs':>11}{'max rel':>11}"
             f"{'max scaled':>12}{'abs at d=0':>12}"]
    for (method, precision), (c, n, a, r, sc, z) in sorted(agg.items()):
        lines.append(f"{method:<24}{precision:<10}{c:>7}{n:>12}{a:>11.2e}{r:>11.2e}{sc:>12.2e}{z:>12.2e}")
    lines.append(f"(max rel over oracle values |d| >= {REL_FLOOR:g}; abs at d=0 over identical-sample pairs)")
    return lines


def assert_close(got, exp, method, precision, what=""):
    record_errors(got, exp, method, precision, what)
    ok = tolerance_ok(got, exp, method, precision)
    if not ok.all():
        bad = np.nonzero(~ok)[0]
        i = bad[np.argmax(np.abs(np.asarray(got)[bad] - np.asarray(exp)[bad]))]
        raise AssertionError(f"{what} {method}/{precision}: {bad.size} of {ok.size} values out of "
                             f"tolerance; worst at {i}: got {got[i]!r} expected {exp[i]!r}")


def condensed_index(n, i, j):
    i, j = np.minimum(i, j), np.maximum(i, j)
    return n * i - i * (i + 1) // 2 + (j - i - 1)


def oracle_condensed(tree, table, method, alpha):
    return oracle.condensed(tree, table, method, alpha)
