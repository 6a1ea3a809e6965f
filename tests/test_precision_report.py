"""The GPU tests' comparison helper on the CPU: tolerances, and the error
record behind the precision report printed after a GPU test run."""
import numpy as np
import pytest

from tests import gpu_util


@pytest.fixture()
def clean_log():
    saved = list(gpu_util.PRECISION_LOG)
    gpu_util.PRECISION_LOG.clear()
    yield gpu_util.PRECISION_LOG
    gpu_util.PRECISION_LOG[:] = saved


def test_tolerances(clean_log):
    exp = np.array([0.0, 0.25, 1.0, 40.0])
    gpu_util.assert_close(exp + 9e-6, exp, "weighted_normalized", "mixed")
    with pytest.raises(AssertionError):
        gpu_util.assert_close(exp + 2e-5, exp, "weighted_normalized", "mixed")
    # the unbounded method's tolerance scales with max(1, |d|)
    gpu_util.assert_close(exp + np.array([0, 0, 0, 3e-4]), exp, "weighted_unnormalized", "mixed")
    gpu_util.assert_close(exp * (1 + 5e-11), exp, "generalized", "fp64")
    with pytest.raises(AssertionError):
        gpu_util.assert_close(exp * (1 + 5e-10), exp, "generalized", "fp64")


def test_error_record_and_summary(clean_log):
    exp = np.array([0.0, 0.5, 2.0, 0.0])
    got = exp + np.array([0.0, 1e-7, 4e-6, 0.0])
    gpu_util.assert_close(got, exp, "weighted_unnormalized", "mixed", "case a")
    gpu_util.assert_close(got[:2], exp[:2], "weighted_unnormalized", "mixed", "case b")
    gpu_util.assert_close(np.zeros(0), np.zeros(0), "unweighted", "mixed", "empty")
    assert len(clean_log) == 2
    what, method, precision, n, a, r, sc, z = clean_log[0]
    assert (what, method, precision, n) == ("case a", "weighted_unnormalized", "mixed", 4)
    assert a == pytest.approx(4e-6) and r == pytest.approx(2e-6) and sc == pytest.approx(2e-6)
    assert z == 0.0
    lines = gpu_util.precision_summary()
    assert len(lines) == 3 and lines[0].split()[:2] == ["method", "precision"]
    row = lines[1].split()
    assert row[:4] == ["weighted_unnormalized", "mixed", "2", "6"]
    assert float(row[4]) == pytest.approx(4e-6)


def test_relative_error_ignores_oracle_zeros(clean_log):
    # an oracle zero enters the absolute column only; relative errors are
    # taken where |d| >= REL_FLOOR
    exp = np.array([0.0, 1e-14, 0.5])
    got = np.array([1e-16, 1e-14 + 1e-24, 0.5 * (1 + 1e-12)])
    gpu_util.assert_close(got, exp, "weighted_normalized", "fp64", "zeros")
    _, _, _, _, a, r, _, z = clean_log[0]
    assert z == pytest.approx(1e-16)
    assert r == pytest.approx(1e-12, rel=1e-3)
    assert a == pytest.approx(1e-16)
