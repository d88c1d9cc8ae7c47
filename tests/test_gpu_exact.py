"""The exact-A preconditioner on the GPU (Sec. 3, Table exacttopleft): a context with one
level has no multigrid, and its (1,1) block solve is the dense inverse of A_gamma on the
mesh, so FGMRES with the block factorisation of Eq. (precond) runs with A-hat = A_gamma.

The oracle solves the same systems with a sparse LU of A_gamma (StokesSolver(exact_A=True));
the two exact solves differ only by rounding, so the iteration counts are the oracle's, and
through the oracle's CPU pin (tests/test_oracle_pins.py) they keep Table exacttopleft's
pattern: P1 = P2 at gamma = 0, counts falling with gamma, within one of the printed counts at
gamma = 1e3."""
import numpy as np
import pytest

from gpu_helpers import rel, torch  # noqa: F401
from oracle.mg import Hierarchy
from oracle.stokes import StokesSolver
from synthetic import problems as P

from paper_2107_00820_gb300 import Context, alstokes as A  # noqa: E402

pytestmark = pytest.mark.gpu

CELLS = [(var, g, dr) for var in ("P1", "P2") for g in (0.0, 10.0, 1e3) for dr in (1e4, 1e6, 1e8)]


def _solve_both(n, var, gamma, dr, rtol=1e-6):
    """(oracle count, GPU solve, GPU solution's true residual in the oracle's system)."""
    from test_gpu_parity import _true_residual
    pb = P.sinker_problem(2, n, 1, 8, 0.1, 200.0, dr, 10.0, gamma, 0)
    W = "Mp_mu" if var == "P2" else "Mp"
    H = Hierarchy(2, pb.n, [pb.mu[0]], gamma, smoother="richardson", steps=1, W=W)
    s = StokesSolver(H, var, exact_A=True)
    _, _, its, _ = s.solve(pb.f, pb.u_bc, rtol=rtol)
    ctx = Context(2, pb.n, 1, pb.mu, gamma, rtol=rtol, maxit=300,
                  schur=A.ALS_SCHUR_P2 if var == "P2" else A.ALS_SCHUR_P1)
    u, p, info = ctx.solve(pb.f, pb.u_bc)
    ctx.close()
    return its, info, _true_residual(s, pb, u, p)


@pytest.mark.parametrize("var,gamma,dr", CELLS, ids=lambda v: str(v))
def test_table_exacttopleft_16(var, gamma, dr):
    """All 18 cells of Table exacttopleft's layout at 2D 16^2 (1e6 residual reduction):
    identical iteration counts, and the GPU solution's true residual meets the tolerance
    (at rtol 1e-6 two valid iterates may differ by cond * 1e-6 in the solution)."""
    its, info, res = _solve_both(16, var, gamma, dr)
    assert info.converged and info.iterations == its, (info.iterations, its)
    assert res <= 1.5e-6, res


@pytest.mark.parametrize("var,gamma,dr", [("P1", 1e3, 1e8), ("P2", 10.0, 1e6), ("P1", 0.0, 1e4)])
def test_table_exacttopleft_32(var, gamma, dr):
    """Three cells at 2D 32^2 (7,938 free velocity dofs: a dense inverse of 504 MB)."""
    its, info, res = _solve_both(32, var, gamma, dr)
    assert info.converged and info.iterations == its, (info.iterations, its)
    assert res <= 1.5e-6, res
