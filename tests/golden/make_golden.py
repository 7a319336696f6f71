"""Writes tests/golden/tiny_systems.txt: small Hines systems with their exact
rational solutions.  Calls only oracle.exact (exact Fraction elimination on
the dense matrix, the plain definition x = A^{-1} b of Section 2).

Each system is a cell tree in Hines numbering (p[0] = -1, p[i] < i) with
integer axial coefficients a_i, leak terms s_i = 1/10, d_i = s_i + sum of the
a at i, u_i = -a_i and an integer right-hand side.

Run:  python tests/golden/make_golden.py
"""
import os
import sys
from fractions import Fraction

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
from oracle import exact  # noqa: E402

SYSTEMS = {
    # a root branch of 3 compartments with two child branches of 2 compartments (a "Y")
    "y_tree": [-1, 0, 1, 2, 3, 2, 5],
    # an unbranched cable: Hines with p[i] = i - 1 is the Thomas algorithm
    "chain5": [-1, 0, 1, 2, 3],
    # a child attached to the middle of a chain
    "mid_attach": [-1, 0, 1, 2, 1, 4],
    # one soma compartment with four single-compartment dendrites
    "star": [-1, 0, 0, 0, 0],
    # two branch levels, ternary split at the root branch end
    "ternary": [-1, 0, 1, 1, 1, 4, 5, 4, 7],
}


def coefficients(p):
    n = len(p)
    a = [Fraction(0)] + [Fraction((i % 3) + 1) for i in range(1, n)]
    s = [Fraction(1, 10)] * n
    d = list(s)
    for i in range(1, n):
        d[i] += a[i]
        d[p[i]] += a[i]
    u = [Fraction(0)] + [-a[i] for i in range(1, n)]
    b = [Fraction(((7 * i) % 5) - 2) for i in range(n)]
    return d, u, b


def main():
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tiny_systems.txt")
    with open(out, "w") as f:
        f.write("# Exact solutions of small Hines systems (Section 2: A[i][i] = d[i],\n")
        f.write("# A[i][p[i]] = A[p[i]][i] = u[i]), written by tests/golden/make_golden.py\n")
        f.write("# with oracle.exact (exact rational Gaussian elimination).\n")
        f.write("# name | p | d | u | b | x  (fractions num/den, comma separated)\n")
        for name, p in SYSTEMS.items():
            d, u, b = coefficients(p)
            x = exact.solve(p, d, u, b)
            fmt = lambda v: ",".join(str(t) for t in v)  # noqa: E731
            f.write(f"{name} | {fmt(p)} | {fmt(d)} | {fmt(u)} | {fmt(b)} | {fmt(x)}\n")
    print("wrote", out)


if __name__ == "__main__":
    main()
