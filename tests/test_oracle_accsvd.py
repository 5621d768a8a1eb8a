"""Pins for the Appendix's accurate SVD: relative accuracy on graded matrices against a
60-digit mpmath SVD, factor orthogonality, reconstruction."""
import numpy as np
import pytest

from oracle.accsvd import accurate_svd

mp = pytest.importorskip("mpmath")


def _reference(M):
    mp.mp.dps = 60
    sv = np.array([float(x) for x in mp.svd_r(mp.matrix(M.tolist()), compute_uv=False)])
    return np.sort(sv)[::-1]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_two_sided_graded_relative_accuracy(seed):
    rng = np.random.default_rng(seed)
    n = 12
    G = rng.standard_normal((n, n))
    d1 = np.logspace(0, -7, n)
    d2 = np.logspace(0, -7, n)[rng.permutation(n)]
    M = d1[:, None] * G * d2[None, :]
    ref = _reference(M)
    A, lam, B = accurate_svd(M)
    assert np.max(np.abs(np.sort(lam)[::-1] - ref) / ref) < 1e-12
    assert np.abs(A.T @ A - np.eye(n)).max() < 1e-13
    assert np.abs(B @ B.T - np.eye(n)).max() < 1e-13
    assert np.abs((A * lam) @ B - M).max() < 1e-14


def test_plain_lapack_is_worse_on_the_same_matrix():
    """The matrix family above is one where the recursion matters (documents the need)."""
    rng = np.random.default_rng(1)
    n = 12
    G = rng.standard_normal((n, n))
    d1 = np.logspace(0, -7, n)
    d2 = np.logspace(0, -7, n)[rng.permutation(n)]
    M = d1[:, None] * G * d2[None, :]
    ref = _reference(M)
    plain = np.linalg.svd(M, compute_uv=False)
    A, lam, B = accurate_svd(M)
    assert np.max(np.abs(plain - ref) / ref) > 100 * np.max(np.abs(np.sort(lam)[::-1] - ref) / ref)


def test_no_refinement_when_well_conditioned():
    rng = np.random.default_rng(4)
    M = rng.standard_normal((8, 10))
    A, lam, B = accurate_svd(M)
    A0, lam0, B0 = np.linalg.svd(M, full_matrices=False)
    assert np.array_equal(lam, lam0)


def test_rank_deficient_and_rectangular():
    rng = np.random.default_rng(5)
    M = rng.standard_normal((9, 3)) @ rng.standard_normal((3, 6))
    A, lam, B = accurate_svd(M)
    assert lam.size == 6
    assert np.abs((A * lam) @ B - M).max() < 1e-13
    assert np.all(lam[3:] < 1e-12 * lam[0])
