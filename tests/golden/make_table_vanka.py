"""Writes table_vanka_oracle.txt: the oracle's FGMRES iteration counts on the AL column of
Table vanka (Sec. 5.2.3), the stored values the GPU solve is compared with.

Configuration of that column: 2D multi-sinker problem (Sec. 5.2: omega 0.1, delta 200,
beta 10, mu_max = DR^(1/2), mu_min = DR^(-1/2)), [Q2]^2 x P1disc on a 128^2 quadrilateral
mesh, 4 mesh levels, 5 smoothing steps, the P2 preconditioner with gamma = 100, F-cycle,
iterations to a 1e6 residual reduction; 1, 6 and 24 sinkers at DR 1e4, 1e6, 1e8, 1e10.
Sinker centres are seeded (seed 0), so the counts are this oracle's, not the paper's (its
centres are random): the paper's printed column is kept beside them for comparison.

Calls only oracle/ and the input generator.  Run from the repository root:
    python tests/golden/make_table_vanka.py
(about six minutes on one core).
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.mg import Hierarchy  # noqa: E402
from oracle.stokes import StokesSolver  # noqa: E402
from synthetic import problems as P  # noqa: E402

SINKERS = (1, 6, 24)
DRS = (1e4, 1e6, 1e8, 1e10)
PRINTED = {1: (4, 6, 8, 9), 6: (10, 14, 16, 16), 24: (9, 15, 20, 25)}   # Table vanka, AL column


def counts(sinkers, dr):
    pb = P.sinker_problem(2, 128, 4, sinkers, 0.1, 200.0, dr, 10.0, 100.0, 0)
    H = Hierarchy(2, pb.n, pb.mu, pb.gamma, steps=5, W="Mp_mu", cycle="F")
    return StokesSolver(H, schur="P2").solve(pb.f, pb.u_bc, rtol=1e-6)[2]


def main():
    lines = ["# Oracle FGMRES iteration counts, AL column of Table vanka (Sec. 5.2.3): 2D 128^2,",
             "# 4 levels, 5 smoothing steps, P2 with gamma 100, F-cycle, 1e6 residual reduction,",
             "# sinker centres from seed 0.  Written by tests/golden/make_table_vanka.py (oracle only).",
             "# columns: sinkers DR oracle_iterations paper_iterations"]
    for s in SINKERS:
        for j, dr in enumerate(DRS):
            its = counts(s, dr)
            lines.append(f"{s} {dr:.0e} {its} {PRINTED[s][j]}")
            print(lines[-1], flush=True)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "table_vanka_oracle.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
