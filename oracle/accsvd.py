"""Accurate recursive SVD (the paper's Appendix) -- test infrastructure.

Steps, in the Appendix's order and notation (M = A Lambda B):
 1. SVD of M by a standard routine (here LAPACK through numpy).
 2. With singular values lambda_1 >= ... >= lambda_n, find the first p with
    lambda_p / lambda_1 < eps (eps = 1e-4 in the paper).
 3. If there is none, return A, Lambda, B.
 4. Otherwise form X = A^T M B^T restricted to the rows and columns p..n.
 5. Recurse on X, giving A~, Lambda~, B~.
 6. Rotate: A[:, p..n] <- A[:, p..n] A~, B[p..n, :] <- B~ B[p..n, :], lambda_p..n <- lambda~.
 7. Return.
Readings: the refined sub-block is indices p..n (the Appendix's step 4 says n-p, its step 6
sums k = p..n; the latter is taken), p >= 2 so the recursion terminates; an all-zero X ends it.
"""
from __future__ import annotations

import numpy as np

EPS = 1e-4


def accurate_svd(M, eps=EPS):
    A, lam, B = np.linalg.svd(M, full_matrices=False)
    n = lam.size
    if n <= 1 or lam[0] == 0.0:
        return A, lam, B
    small = np.nonzero(lam / lam[0] < eps)[0]
    if small.size == 0:
        return A, lam, B
    p = int(small[0])                       # 0-based first index of the refined block
    X = A[:, p:].T @ M @ B[p:, :].T
    if not np.any(X):
        lam = lam.copy()
        lam[p:] = 0.0
        return A, lam, B
    At, lt, Bt = accurate_svd(X, eps)
    A = A.copy()
    B = B.copy()
    lam = lam.copy()
    A[:, p:] = A[:, p:] @ At
    B[p:, :] = Bt @ B[p:, :]
    lam[p:] = lt
    return A, lam, B
