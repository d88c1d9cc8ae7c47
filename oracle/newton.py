"""FP64 oracle: Newton's method for Stokes flow with the viscoplastic rheology of Sec. 5.3.

TEST INFRASTRUCTURE ONLY (see oracle/fem.py).  Follows Sec. 5.3.1:

  * effective viscosity mu(eps_II) = mu_ref tau_y / (2 mu_ref eps_II + tau_y), with
    eps_II = sqrt(eps : eps / 2) the second invariant of the strain rate eps(u);
  * the nonlinear problem -div(2 mu(eps_II(u)) eps(u)) + grad p = f, -div u = 0 in the weak
    form of Sec. 2 ([Q2]^d x P1disc, 3^d Gauss points, Dirichlet rows replaced);
  * each Newton step solves the linearised Stokes system whose viscous coefficient is the
    fourth-order tensor 2 mu [I - (eps (x) tau)_sym / (2 eps_II max(tau_y, tau_II))], with
    the right-hand side the negative nonlinear residual.  The paper's stress-velocity variant
    carries tau as an extra unknown whose update formula it cites but does not state; the
    standard Newton method it names as the alternative takes tau = 2 mu eps of the current
    iterate, which is what this module does (tau_II = 2 mu eps_II < tau_y, so the max is tau_y);
  * the AL preconditioner of every linearised system uses the scalar prefactor mu for the
    weighted pressure mass (Sec. 5.3.2), with the P2 pairing (W = M_p(1/mu));
  * coarse levels are rediscretised (Sec. 5.1): their coefficients are evaluated at their own
    Gauss points from the finest-level iterate.

A backtracking line search on the residual norm (halving the step) globalises the iteration;
the paper does not state its globalisation.
"""
from __future__ import annotations

import numpy as np

from .fem import Level, Mesh, lagrange_q2, lagrange_q2_deriv, mandel_pairs
from .mg import Hierarchy
from .stokes import StokesSolver


# ---------------------------------------------------------------------------
# rheology
# ---------------------------------------------------------------------------
def second_invariant(E):
    """eps_II = sqrt(E : E / 2) for strain tensors E (..., d, d)."""
    return np.sqrt(0.5 * np.einsum("...kl,...kl->...", E, E))


def viscosity(eII, mu_ref, tau_y):
    """Effective viscosity of Sec. 5.3.1."""
    return mu_ref * tau_y / (2.0 * mu_ref * eII + tau_y)


def mandel_vector(E):
    """Mandel vector of symmetric tensors E (..., d, d): diagonal, then sqrt2 off-diagonal."""
    d = E.shape[-1]
    return np.stack([w * E[..., k, l] for (k, l), w in mandel_pairs(d)], -1)


def newton_tensor(E, mu_ref, tau_y, T=None):
    """The linearised viscous coefficient at each point, in packed Mandel form, and mu.

    C = 2 mu [I - (eps (x) tau)_sym / (2 eps_II max(tau_y, tau_II))]; T is the stress
    variable (default 2 mu eps, the standard Newton method).  In Mandel vectors
    (e, t) the operator (eps (x) tau)_sym : d eps is (e t^T + t e^T) / 2 acting on d e.
    Returns (C packed upper triangle row-major (..., m(m+1)/2), mu (...))."""
    eII = second_invariant(E)
    mu = viscosity(eII, mu_ref, tau_y)
    if T is None:
        T = 2.0 * mu[..., None, None] * E
    e, t = mandel_vector(E), mandel_vector(T)
    tII = second_invariant(T)
    denom = 2.0 * eII * np.maximum(tau_y, tII)
    scale = np.divide(1.0, denom, out=np.zeros_like(denom), where=denom > 0)
    m = e.shape[-1]
    sym = 0.5 * (e[..., :, None] * t[..., None, :] + t[..., :, None] * e[..., None, :])
    C = 2.0 * mu[..., None, None] * (np.eye(m) - scale[..., None, None] * sym)
    iu = np.triu_indices(m)
    return C[..., iu[0], iu[1]], mu


# ---------------------------------------------------------------------------
# strain rates of a finest-level velocity, at any level's Gauss points
# ---------------------------------------------------------------------------
def strain_at_qp(mesh: Mesh, u):
    """eps(u_h) at the mesh's own Gauss points: (ncells, nq, d, d)."""
    return np.einsum("cj,qjkl->cqkl", u[mesh.cell_dofs], mesh.strain_basis)


def strain_at_points(mesh: Mesh, u, cells, xi):
    """eps(u_h) at reference points xi (npts, d) of the given cells (npts,): (npts, d, d)."""
    d, mi = mesh.d, mesh.ref.mi
    L = lagrange_q2(xi)                       # (npts, d, 3)
    dL = lagrange_q2_deriv(xi)
    grad = np.ones((xi.shape[0], mi.shape[0], d))
    for k in range(d):
        for j in range(d):
            grad[:, :, j] *= (dL if j == k else L)[:, k, mi[:, k]]
    grad *= (2.0 / np.array(mesh.h))[None, None, :]
    U = u[mesh.cell_dofs[cells]].reshape(len(cells), d, -1)        # component-major
    G = np.einsum("pai,pij->paj", U, grad)                          # d u_a / d x_j
    return 0.5 * (G + np.swapaxes(G, 1, 2))


def strain_on_level(fine: Mesh, u, level_mesh: Mesh):
    """eps(u_h) of the finest-level velocity at the Gauss points of another level."""
    d = fine.d
    h_l, h_f = np.array(level_mesh.h), np.array(fine.h)
    x = (level_mesh.cells[:, None, :] + 0.5 * (1.0 + level_mesh.ref.xq[None])) * h_l
    x = x.reshape(-1, d)
    c = np.minimum(np.floor(x / h_f).astype(np.int64), np.array(fine.n) - 1)
    xi = 2.0 * (x / h_f - c) - 1.0
    stride = np.cumprod((1,) + fine.n[:-1])
    E = strain_at_points(fine, u, (c * stride).sum(1), xi)
    return E.reshape(level_mesh.ncells, level_mesh.ref.nq, d, d)


# ---------------------------------------------------------------------------
# the nonlinear problem
# ---------------------------------------------------------------------------
class ViscoplasticProblem:
    """-div(2 mu(eps_II) eps(u)) + grad p = f, -div u = 0 on (0,1)^d with u = u_D on the
    boundary, on an n^d mesh with a `levels`-level hierarchy for the linearised solves."""

    def __init__(self, d, n, levels, f_qp, u_bc, mu_ref, tau_y, gamma):
        self.d, self.n, self.L = d, n, levels
        self.mu_ref, self.tau_y, self.gamma = float(mu_ref), float(tau_y), float(gamma)
        self.meshes = [Mesh(d, n // 2 ** (levels - 1 - l)) for l in range(levels)]
        self.fine = m = self.meshes[-1]
        self.f_qp = np.asarray(f_qp, float)
        self.bdof = m.boundary_dof
        self.uD = np.where(self.bdof, np.asarray(u_bc, float).reshape(-1), 0.0)
        # the body-force load vector, with the empty-coefficient level only for its tables
        self.F = Level(d, n, np.ones((m.ncells, m.ref.nq)), 0.0).load_vector(self.f_qp)

    def residual(self, u, p):
        """(R_u, R_p) = (A(u) u + B^T p - F, B u) with Dirichlet rows of R_u set to 0."""
        m = self.fine
        E = strain_at_qp(m, u)
        mu = viscosity(second_invariant(E), self.mu_ref, self.tau_y)
        loc = np.einsum("q,cq,cqkl,qjkl->cj", 2.0 * m.wdet, mu, E, m.strain_basis)
        P = np.asarray(p).reshape(m.ncells, self.d + 1)
        loc = loc + P @ m.B_elem
        Ru = np.zeros(m.nu)
        np.add.at(Ru, m.cell_dofs, loc)
        Ru -= self.F
        Ru[self.bdof] = 0.0
        Rp = (u[m.cell_dofs] @ m.B_elem.T).reshape(-1)
        return Ru, Rp

    def linearisation(self, u):
        """Hierarchy of the linearised operator at u (tensor C and mu on every level)."""
        Cs, mus = [], []
        for lm in self.meshes:
            E = strain_at_qp(lm, u) if lm is self.fine else strain_on_level(self.fine, u, lm)
            C, mu = newton_tensor(E, self.mu_ref, self.tau_y)
            Cs.append(C)
            mus.append(mu)
        return Cs, mus

    def newton_step(self, u, p, rtol=1e-12, steps=5):
        """Solve [J B^T; B 0] [du; dp] = -[R_u; R_p] by AL-preconditioned FGMRES (Sec. 5.3)."""
        Cs, mus = self.linearisation(u)
        H = Hierarchy(self.d, self.n, Cs, self.gamma, kind="tensor", mu_eff=mus, steps=steps, W="Mp_mu")
        s = StokesSolver(H, schur="P2")
        lv = H.levels[-1]
        Ru, Rp = self.residual(u, p)
        r2 = -Rp
        winv_r2 = np.linalg.solve(lv.W_blocks, r2.reshape(lv.mesh.ncells, -1)[:, :, None])[:, :, 0]
        rhs1 = -Ru + self.gamma * (lv.B_raw.T @ winv_r2.reshape(-1))
        rhs1[self.bdof] = 0.0
        x, its, _ = s.fgmres(np.concatenate([rhs1, r2]), rtol=rtol, maxit=300)
        return x[: lv.mesh.nu], x[lv.mesh.nu:], its

    def norm(self, u, p):
        Ru, Rp = self.residual(u, p)
        return float(np.sqrt(Ru @ Ru + Rp @ Rp))

    def solve(self, u0=None, p0=None, rtol=1e-10, maxit=30):
        """Newton with backtracking; returns (u, p, residual-norm history, linear iterations)."""
        m = self.fine
        u = self.uD.copy() if u0 is None else np.asarray(u0, float).copy()
        u[self.bdof] = self.uD[self.bdof]
        p = np.zeros(m.npres) if p0 is None else np.asarray(p0, float).copy()
        hist = [self.norm(u, p)]
        lin = []
        for _ in range(maxit):
            if hist[-1] <= rtol * hist[0]:
                break
            # linear tolerance: an absolute target of 1e-12 of the first residual, which
            # keeps the steps exact to well below the Newton tolerance without asking
            # FGMRES for more than FP64 allows once the residual itself is small
            eta = min(1e-2, max(1e-12, 1e-12 * hist[0] / hist[-1]))
            du, dp, its = self.newton_step(u, p, rtol=eta)
            lin.append(its)
            alpha = 1.0
            for _ in range(12):
                r = self.norm(u + alpha * du, p + alpha * dp)
                if r < (1.0 - 1e-4 * alpha) * hist[-1]:
                    break
                alpha *= 0.5
            u, p = u + alpha * du, p + alpha * dp
            hist.append(r)
        return u, p, hist, lin
