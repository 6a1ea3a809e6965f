"""Pins of the downstream agreement helpers (Mantel statistic, principal
coordinates, Procrustes disparity) against closed forms; CPU only."""
import numpy as np
import pytest

from paper_2005_05826_gb300 import downstream as ds


def euclid_condensed(x):
    d = np.sqrt(((x[:, None, :] - x[None, :, :]) ** 2).sum(-1))
    i, j = np.triu_indices(len(x), 1)
    return d[i, j]


def test_square_roundtrip_and_bad_length():
    c = np.arange(1.0, 11.0)  # n = 5
    d = ds.square(c)
    assert d.shape == (5, 5) and np.all(np.diag(d) == 0) and np.all(d == d.T)
    i, j = np.triu_indices(5, 1)
    np.testing.assert_array_equal(d[i, j], c)
    with pytest.raises(ValueError):
        ds.square(np.ones(7))


def test_mantel_identity_affine_and_independent():
    rng = np.random.default_rng(1)
    a = euclid_condensed(rng.normal(size=(40, 3)))
    r, p = ds.mantel(a, a, permutations=199, seed=2)
    assert r == pytest.approx(1.0, abs=1e-12)
    assert p == pytest.approx(1 / 200)
    r2, _ = ds.mantel(a, 2.5 * a + 3.0, permutations=0)
    assert r2 == pytest.approx(1.0, abs=1e-12)  # Pearson is affine invariant
    b = euclid_condensed(rng.normal(size=(40, 3)))
    r3, p3 = ds.mantel(a, b, permutations=199, seed=3)
    assert abs(r3) < 0.3 and p3 > 0.01  # unrelated point sets


def test_pcoa_recovers_euclidean_configuration():
    rng = np.random.default_rng(4)
    x = rng.normal(size=(30, 3)) * np.array([5.0, 2.0, 0.5])
    coords, w = ds.pcoa(euclid_condensed(x), k=5)
    # three positive eigenvalues: those of the centred Gram matrix
    xc = x - x.mean(axis=0)
    np.testing.assert_allclose(np.sort(w)[::-1], np.sort(np.linalg.eigvalsh(xc.T @ xc))[::-1], rtol=1e-9)
    assert coords.shape == (30, 3)
    assert ds.procrustes(xc, coords) < 1e-20  # same configuration up to rotation / reflection


def test_procrustes_rotation_invariance_and_mismatch():
    rng = np.random.default_rng(5)
    x = rng.normal(size=(25, 4))
    q, _ = np.linalg.qr(rng.normal(size=(4, 4)))
    assert ds.procrustes(x, 3.0 * x @ q + 1.0) < 1e-20
    assert ds.procrustes(x, rng.normal(size=(25, 4))) > 0.1
