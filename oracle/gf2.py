"""Gaussian elimination over F_2 (plain, for small dense matrices).

Used by the generator-picture sum of Sec. 3.2 (a representative error and a basis of
the trivial errors) and by the closed-form pins (rank of H).
"""
from __future__ import annotations

import numpy as np


def row_reduce(A: np.ndarray):
    """Reduced row echelon form of A over F_2.  Returns (R, pivot_columns)."""
    R = (np.asarray(A, dtype=np.uint8) & 1).copy()
    rows, cols = R.shape
    pivots = []
    r = 0
    for c in range(cols):
        if r >= rows:
            break
        hit = np.nonzero(R[r:, c])[0]
        if hit.size == 0:
            continue
        k = r + hit[0]
        if k != r:
            R[[r, k]] = R[[k, r]]
        for i in range(rows):
            if i != r and R[i, c]:
                R[i] ^= R[r]
        pivots.append(c)
        r += 1
    return R, pivots


def rank(A: np.ndarray) -> int:
    return len(row_reduce(A)[1])


def solve(A: np.ndarray, b: np.ndarray):
    """One solution x of A x = b over F_2, or None if the system is inconsistent."""
    A = np.asarray(A, dtype=np.uint8)
    aug = np.concatenate([A, np.asarray(b, dtype=np.uint8).reshape(-1, 1)], axis=1)
    R, piv = row_reduce(aug)
    n = A.shape[1]
    if n in piv:
        return None
    x = np.zeros(n, dtype=np.uint8)
    for i, c in enumerate(piv):
        x[c] = R[i, n]
    return x


def kernel(A: np.ndarray) -> np.ndarray:
    """Basis of {x : A x = 0} over F_2, as rows of a (n - rank) x n matrix."""
    A = np.asarray(A, dtype=np.uint8)
    n = A.shape[1]
    R, piv = row_reduce(A)
    free = [c for c in range(n) if c not in piv]
    basis = np.zeros((len(free), n), dtype=np.uint8)
    for k, f in enumerate(free):
        basis[k, f] = 1
        for i, c in enumerate(piv):
            basis[k, c] = R[i, f]
    return basis
