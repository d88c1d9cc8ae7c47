"""Newton's method for the viscoplastic rheology on the GPU (als_newton_solve, Sec. 5.3.1)
against the oracle's Newton iteration (oracle/newton.py, pinned on the CPU by finite
differences of the residual, the rheology's closed forms and the quadratic tail).

The GPU evaluates the linearised coefficient at every level's Gauss points from the finest
iterate with its own kernel, re-runs the setup with it, solves each step with its FP64
FGMRES, and backtracks on the residual norm it evaluates itself; the oracle does each of
these with assembled matrices.  In FP64 the two iterations must take the same steps: the
same number of Newton steps, the same FGMRES count per step (within one where a step's
tolerance is crossed by a hair), residual norms that agree to round-off relative to the
first, and the same converged solution."""
import numpy as np
import pytest

from gpu_helpers import rel, torch  # noqa: F401
from oracle.fem import Mesh
from oracle.newton import ViscoplasticProblem

from paper_2107_00820_gb300 import Context, alstokes as A  # noqa: E402

pytestmark = pytest.mark.gpu


def _problem(d, n, levels, tau_y, gamma):
    m = Mesh(d, n)
    x = m.node_coords()
    if d == 2:
        uD = np.stack([np.sin(np.pi * x[:, 0]) * np.cos(np.pi * x[:, 1]),
                       -np.cos(np.pi * x[:, 0]) * np.sin(np.pi * x[:, 1])])
    else:
        uD = np.stack([np.sin(np.pi * x[:, 0]) * np.cos(np.pi * x[:, 1]),
                       -np.cos(np.pi * x[:, 0]) * np.sin(np.pi * x[:, 1]),
                       np.zeros(m.N)])
    f = np.zeros((m.ncells, 3 ** d, d))
    f[..., d - 1] = -1.0
    return ViscoplasticProblem(d, n, levels, f, uD, 1.0, tau_y, gamma), f, uD.reshape(-1)


def _context(d, n, levels, gamma, **opt):
    nm = 3 if d == 2 else 6
    iu = np.triu_indices(nm)
    C = (2.0 * np.eye(nm))[iu]
    coeffs, mus = [], []
    for lvl in range(levels):
        nc = (n // 2 ** (levels - 1 - lvl)) ** d
        coeffs.append(np.ascontiguousarray(np.broadcast_to(C, (nc, 3 ** d, len(C)))))
        mus.append(np.ones((nc, 3 ** d)))
    return Context(d, n, levels, coeffs, gamma, mu_eff=mus, schur=A.ALS_SCHUR_P2, maxit=300, **opt)


@pytest.mark.parametrize("d,n,levels,tau_y", [(2, 8, 2, 1.0), (2, 16, 3, 0.3), (3, 4, 2, 1.0)])
def test_newton_matches_the_oracle(d, n, levels, tau_y):
    gamma = 1e2
    pb, f, uD = _problem(d, n, levels, tau_y, gamma)
    uo, po, hist_o, lin_o = pb.solve(rtol=1e-10, maxit=30)
    ctx = _context(d, n, levels, gamma)
    u, p, info = ctx.newton_solve(f, uD, mu_ref=1.0, tau_y=tau_y, rtol=1e-10, maxit=30)
    hist, lin = ctx.newton_history()
    assert info.converged == 1
    assert info.iterations == len(lin_o), (info.iterations, len(lin_o))
    assert all(abs(a - b) <= 1 for a, b in zip(lin[1:], lin_o)), (lin[1:], lin_o)
    assert np.allclose(hist, hist_o, rtol=1e-6, atol=1e-9 * hist_o[0]), (hist, hist_o)
    assert rel(u, uo) <= 1e-8 and rel(p, po) <= 1e-7, (rel(u, uo), rel(p, po))
    # the converged iterate is a zero of the oracle's residual
    Ru, Rp = pb.residual(u, p)
    assert np.sqrt(Ru @ Ru + Rp @ Rp) <= 1e-9 * hist_o[0]


def test_newton_mixed_mode_converges_to_the_same_solution():
    """The FP32 cycle inside the linear solves (mixed mode): the same converged solution
    (the Newton residual is evaluated in FP64), in at most two more Newton steps."""
    pb, f, uD = _problem(2, 16, 3, 1.0, 1e2)
    uo, po, hist_o, lin_o = pb.solve(rtol=1e-10, maxit=30)
    ctx = _context(2, 16, 3, 1e2, mode=A.ALS_MODE_MIXED)
    u, p, info = ctx.newton_solve(f, uD, mu_ref=1.0, tau_y=1.0, rtol=1e-10, maxit=30)
    assert info.converged == 1 and info.iterations <= len(lin_o) + 2
    assert rel(u, uo) <= 1e-7 and rel(p, po) <= 1e-7, (rel(u, uo), rel(p, po))


def test_newton_refuses_a_scalar_context():
    pb, f, uD = _problem(2, 8, 2, 1.0, 1e2)
    m = Mesh(2, 8)
    ctx = Context(2, 8, 2, [np.ones((16, 9)), np.ones((64, 9))], 1e2, schur=A.ALS_SCHUR_P2)
    with pytest.raises(A.ALSError) as e:
        ctx.newton_solve(f, uD)
    assert e.value.status == A.ALS_EINVAL
    assert m.ncells == 64
