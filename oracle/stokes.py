"""FP64 oracle: AL block preconditioner and FGMRES for the augmented Stokes system.

TEST INFRASTRUCTURE ONLY (see oracle/fem.py).  Follows:
  * Eq. (augstokessys): [[A + gamma B^T W^-1 B, B^T], [B, 0]] [u; p] =
    [r1 + gamma B^T W^-1 r2; r2] with W = M_p;
  * Eq. (precond): P = [[I, -A^-1 B^T], [0, I]] diag(A^-1, -S^-1) [[I, 0], [-B A^-1, I]],
    applied literally right to left, so the (1,1) approximation (a multigrid
    cycle) is applied twice per preconditioner application ("full");
    the factorisation types that keep only some factors, with the same
    blocks: "upper" = [[A, B^T], [0, -S]]^-1, "lower" = [[A, 0], [B, -S]]^-1,
    "diag" = diag(A^-1, -S^-1), one (1,1) application each;
  * Eq. (P1P2): P1: S_gamma^-1 = M_p(1/mu)^-1 + gamma M_p^-1;
    P2: S_gamma^-1 = (1 + gamma) M_p(1/mu)^-1, both block diagonal (one
    (d+1)x(d+1) block per cell, Sec. 5.1);
  * flexible GMRES (Sec. 5.1), right preconditioned, classical Gram-Schmidt
    applied twice, no restart, relative residual test on the l2 norm.

Dirichlet data are lifted: r1 = F - A u_D and r2 = -B u_D on the
interior rows; boundary rows carry the identity (Firedrake/PETSc convention).
The pressure is fixed up to a constant; the constant mode (1 on the
constant-basis slot of every cell) is projected out after each
preconditioner application and the final pressure has zero mean.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .mg import Hierarchy


def schur_blocks(level, variant="P1"):
    """Per-cell (d+1)x(d+1) blocks of S_gamma^-1 (Eq. (P1P2)).

    P1 pairs (S_hat, W) = (M_p(1/mu), M_p), P2 pairs (M_p(1/mu), M_p(1/mu)):
    the level's augmentation weight W must match the variant.
    """
    m = level.mesh
    if (variant == "P1") != (level.W == "Mp"):
        raise ValueError(f"{variant} needs W = {'M_p' if variant == 'P1' else 'M_p(1/mu)'}")
    inv_mu = np.linalg.inv(level.Mp_mu_blocks)
    inv_M = np.linalg.inv(m.M_elem)
    if variant == "P1":
        return inv_mu + level.gamma * inv_M[None]
    if variant == "P2":
        return (1.0 + level.gamma) * inv_mu
    raise ValueError(variant)


def pressure_nullvector(level):
    m = level.mesh
    n = np.zeros(m.npres)
    n[:: m.npres // m.ncells] = 1.0             # pressure coefficients per cell: d + 1 at k = 2
    return n


class StokesSolver:
    """Block-preconditioned FGMRES on the augmented system (Secs. 3, 5.1)."""

    def __init__(self, hierarchy: Hierarchy, schur="P1", exact_A=False, fact="full"):
        if fact not in ("full", "upper", "lower", "diag"):
            raise ValueError(fact)
        self.fact = fact
        self.H = hierarchy
        self.fine = lv = hierarchy.levels[-1]
        self.nu, self.np_ = lv.mesh.nu, lv.mesh.npres
        self.Sinv = sp.block_diag(list(schur_blocks(lv, schur)), format="csr")
        self.nvec = pressure_nullvector(lv)
        self.exact_A = exact_A
        if exact_A:
            import scipy.sparse.linalg as spla
            self._lu = spla.splu(lv.A.tocsc())

    # system operator K = [[A_gamma, B^T], [B, 0]] with Dirichlet identity rows
    def matvec(self, x):
        lv = self.fine
        u, p = x[: self.nu], x[self.nu:]
        return np.concatenate([lv.A @ u + lv.Bt @ p, lv.B @ u])

    def Ahat_inv(self, f):
        if self.exact_A:
            return self._lu.solve(f)
        return self.H.cycle(f)

    def project(self, p):
        n = self.nvec
        return p - (n @ p) / (n @ n) * n

    def precondition(self, x):
        lv = self.fine
        f, g = x[: self.nu], x[self.nu:]
        if self.fact == "full":
            z1 = self.Ahat_inv(f)
            z2 = -(self.Sinv @ (g - lv.B @ z1))
            x1 = z1 - self.Ahat_inv(lv.Bt @ z2)
        elif self.fact == "upper":
            z2 = -(self.Sinv @ g)
            x1 = self.Ahat_inv(f - lv.Bt @ z2)
        elif self.fact == "lower":
            x1 = self.Ahat_inv(f)
            z2 = -(self.Sinv @ (g - lv.B @ x1))
        else:
            x1 = self.Ahat_inv(f)
            z2 = -(self.Sinv @ g)
        return np.concatenate([x1, self.project(z2)])

    def fgmres(self, rhs, rtol=1e-8, maxit=300):
        beta = np.linalg.norm(rhs)
        hist = [beta]
        n = rhs.shape[0]
        if beta == 0.0:
            return np.zeros(n), 0, hist
        V = np.zeros((maxit + 1, n))
        Z = np.zeros((maxit, n))
        H = np.zeros((maxit + 1, maxit))
        V[0] = rhs / beta
        k_done = 0
        y = np.zeros(0)
        for k in range(maxit):
            Z[k] = self.precondition(V[k])
            w = self.matvec(Z[k])
            h = V[: k + 1] @ w
            w = w - V[: k + 1].T @ h
            h2 = V[: k + 1] @ w
            w = w - V[: k + 1].T @ h2
            H[: k + 1, k] = h + h2
            H[k + 1, k] = np.linalg.norm(w)
            V[k + 1] = w / H[k + 1, k] if H[k + 1, k] > 0 else 0.0
            e1 = np.zeros(k + 2)
            e1[0] = beta
            Hk = H[: k + 2, : k + 1]
            y = np.linalg.lstsq(Hk, e1, rcond=None)[0]
            res = np.linalg.norm(e1 - Hk @ y)
            hist.append(res)
            k_done = k + 1
            if res <= rtol * beta:
                break
        return Z[:k_done].T @ y, k_done, hist

    def rhs(self, f_qp, u_bc, r2=None):
        """Lifted, augmented right-hand side (Eq. (augstokessys))."""
        lv = self.fine
        bd = lv.bdof
        uD = np.where(bd, np.asarray(u_bc, float).reshape(-1), 0.0)
        F = lv.load_vector(f_qp)
        r1 = F - lv.A_raw @ uD
        r2_tot = -(lv.B_raw @ uD) if r2 is None else np.asarray(r2, float) - lv.B_raw @ uD
        winv_r2 = np.linalg.solve(lv.W_blocks, r2_tot.reshape(lv.mesh.ncells, -1)[:, :, None])[:, :, 0]
        rhs1 = r1 + lv.gamma * (lv.B_raw.T @ winv_r2.reshape(-1))
        rhs1[bd] = 0.0
        return np.concatenate([rhs1, r2_tot]), uD

    def solve(self, f_qp, u_bc, r2=None, rtol=1e-8, maxit=300):
        b, uD = self.rhs(f_qp, u_bc, r2)
        x, its, hist = self.fgmres(b, rtol, maxit)
        u = x[: self.nu] + uD
        p = x[self.nu:].copy()
        npr = self.fine.mesh.npres // self.fine.mesh.ncells
        p[::npr] -= p[::npr].mean()
        return u, p, its, hist


def direct_solve(level, f_qp, u_bc, r2=None):
    """Sparse direct solve of the augmented system with a zero-mean pressure
    constraint (a Lagrange multiplier on the constant mode)."""
    import scipy.sparse.linalg as spla
    solver = StokesSolver.__new__(StokesSolver)
    solver.fine = level
    solver.nu, solver.np_ = level.mesh.nu, level.mesh.npres
    b, uD = StokesSolver.rhs(solver, f_qp, u_bc, r2)
    n = pressure_nullvector(level)
    K = sp.bmat([[level.A, level.Bt, None],
                 [level.B, None, sp.csr_matrix(n[:, None])],
                 [None, sp.csr_matrix(n[None, :]), None]], format="csc")
    x = spla.spsolve(K, np.concatenate([b, [0.0]]))
    u = x[: level.mesh.nu] + uD
    p = x[level.mesh.nu: -1]
    return u, p
