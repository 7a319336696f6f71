"""Exact rational solve of a small Hines system -- test infrastructure only.

Gaussian elimination with partial pivoting on the dense matrix in
``fractions.Fraction`` arithmetic: no rounding at all, so it pins the FP64
oracle to the plain definition x = A^{-1} b (Section 2: A[i][i] = d[i],
A[i][p[i]] = A[p[i]][i] = u[i]).  Inputs are taken as exact rationals
(floats are converted exactly).  Only for tiny systems (N <= ~40).
"""
from __future__ import annotations

from fractions import Fraction


def dense_matrix(p, d, u):
    n = len(d)
    A = [[Fraction(0)] * n for _ in range(n)]
    for i in range(n):
        A[i][i] = Fraction(d[i])
    for i in range(1, n):
        A[i][p[i]] = Fraction(u[i])
        A[p[i]][i] = Fraction(u[i])
    return A


def solve(p, d, u, b):
    """Exact x with A x = b, as a list of Fractions."""
    A = dense_matrix(p, d, u)
    n = len(A)
    M = [row[:] + [Fraction(b[i])] for i, row in enumerate(A)]
    for k in range(n):
        piv = max(range(k, n), key=lambda r: abs(M[r][k]))
        if M[piv][k] == 0:
            raise ZeroDivisionError("singular matrix")
        M[k], M[piv] = M[piv], M[k]
        for r in range(k + 1, n):
            if M[r][k] != 0:
                f = M[r][k] / M[k][k]
                for c in range(k, n + 1):
                    M[r][c] -= f * M[k][c]
    x = [Fraction(0)] * n
    for k in range(n - 1, -1, -1):
        s = M[k][n] - sum(M[k][c] * x[c] for c in range(k + 1, n))
        x[k] = s / M[k][k]
    return x
