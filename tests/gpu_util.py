"""Helpers shared by the GPU tests: tolerances and oracle comparison."""
import numpy as np

import oracle

METHODS = ["unweighted", "weighted_unnormalized", "weighted_normalized", "generalized"]

# FP64 path: 1e-10 relative (exact zeros stay within 1e-15); mixed path: 1e-5
# absolute, scaled by max(1, |d|) for the unbounded weighted_unnormalized.
FP64_RTOL, FP64_ATOL = 1e-10, 1e-15
MIXED_ATOL = 1e-5


def tolerance_ok(got, exp, method, precision):
    got = np.asarray(got, dtype=np.float64)
    exp = np.asarray(exp, dtype=np.float64)
    if precision == "fp64":
        return np.abs(got - exp) <= FP64_RTOL * np.abs(exp) + FP64_ATOL
    scale = np.maximum(1.0, np.abs(exp)) if method == "weighted_unnormalized" else 1.0
    return np.abs(got - exp) <= MIXED_ATOL * scale


def assert_close(got, exp, method, precision, what=""):
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
