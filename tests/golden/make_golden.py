"""Writes the closed-form fixtures used by tests/test_oracle.py.

Nothing here runs the oracle or the GPU library: every number is a formula.

kn_trace.txt   -- K_n (complete graph, ones off the diagonal): A^2 = (n-2)A +
                  (n-1)I, so trace(A^3) = n(n-1)(n-2).
amg_galerkin.txt -- 7-point Laplacian (diag 6, off -1) on a g^3 grid and the
                  piecewise-constant 2x2x2 aggregation R (M = g/2 aggregates per
                  side).  (R^T A R)(I,J) sums A over aggregate pairs: diagonal
                  8*6 - 24 = 24 (12 internal edges, both directions), faces
                  -4 (4 crossing edges); at level l this compounds to 6*4^l and
                  -4^l.  R^T A has, per aggregate, its 8 own points plus 4
                  outside neighbours through each face with a neighbour inside
                  the grid: nnz = 8 M^3 + 24 M^3 - 24 M^2 = 32 M^3 - 24 M^2.
                  R^T A R is the 7-point pattern on M^3: 7 M^3 - 6 M^2.
"""
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    with open(os.path.join(HERE, "kn_trace.txt"), "w") as fh:
        fh.write("# n  trace(A^3) for K_n = n(n-1)(n-2)\n")
        for n in range(3, 10):
            fh.write(f"{n} {n * (n - 1) * (n - 2)}\n")
    with open(os.path.join(HERE, "amg_galerkin.txt"), "w") as fh:
        fh.write("# fine_side coarse_level diag off nnz(R^T A) nnz(R^T A R)\n")
        for g0 in (8, 16, 128):
            g, lvl = g0, 0
            while g >= 4:
                M = g // 2
                lvl += 1
                fh.write(f"{g} {lvl} {6 * 4 ** lvl} {-(4 ** lvl)} "
                         f"{32 * M ** 3 - 24 * M ** 2} {7 * M ** 3 - 6 * M ** 2}\n")
                g = M


if __name__ == "__main__":
    main()
