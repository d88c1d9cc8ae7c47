"""Writes sinker2d_128_oracle.txt: the oracle's FGMRES iteration counts on the 2D 128^2
multi-sinker configuration, the stored values the GPU's FP64 solve must reproduce.

Configuration: 2D multi-sinker problem (Sec. 5.2: 8 sinkers from seed 0, omega 0.1,
delta 200, beta 10, DR 1e6 with mu_max = 1e3, mu_min = 1e-3), [Q2]^2 x P1disc on 128^2
quadrilaterals, 5 mesh levels (coarse 8^2), GMRES(5) vertex-star smoothing, V-cycle, the P1
preconditioner of Eq. (precond) (two cycles per iteration), FGMRES to a 1e-8 relative
residual, gamma 1, 1e2 and 1e4.

Calls only oracle/ and the input generator.  Run from the repository root:
    python tests/golden/make_sinker2d_128.py
(a few minutes on one core).
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.mg import Hierarchy  # noqa: E402
from oracle.stokes import StokesSolver  # noqa: E402
from synthetic import problems as P  # noqa: E402

GAMMAS = (1.0, 1e2, 1e4)


def counts(gamma):
    pb = P.sinker_problem(2, 128, 5, 8, 0.1, 200.0, 1e6, 10.0, gamma, 0)
    H = Hierarchy(2, pb.n, pb.mu, pb.gamma, steps=5)
    return StokesSolver(H).solve(pb.f, pb.u_bc, rtol=1e-8)[2]


def main():
    lines = ["# Oracle FGMRES iteration counts, 2D 128^2 multi-sinker (8 sinkers, seed 0, DR 1e6),",
             "# 5 levels, GMRES(5) star smoothing, V-cycle, P1, rtol 1e-8.",
             "# Written by tests/golden/make_sinker2d_128.py (oracle only).",
             "# columns: gamma oracle_iterations"]
    for g in GAMMAS:
        lines.append(f"{g:.0e} {counts(g)}")
        print(lines[-1], flush=True)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "sinker2d_128_oracle.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
