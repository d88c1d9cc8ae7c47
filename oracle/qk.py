"""FP64 oracle for higher orders: [Q_k]^d x P_(k-1)^disc, scalar viscosity.

TEST INFRASTRUCTURE ONLY (see oracle/fem.py).  The same definitions as the
k = 2 oracle, written for any order k >= 2, so that the higher-order study of
Sec. 5.2.2 (Table k) has a reference before any kernel exists for it:

  * velocity: continuous Q_k, nodal basis on k + 1 equispaced nodes per axis and
    cell, node lattice of k n + 1 nodes per direction, x fastest;
  * pressure: discontinuous P_(k-1), the monomials xi^alpha (|alpha| <= k - 1) in
    reference coordinates, ordered by total degree (for k = 2: {1, xi_0, .., xi_(d-1)},
    the basis of oracle/fem.py); C(k - 1 + d, d) of them per cell;
  * (k + 1)^d Gauss points per cell (exact for the degree-2k products of the
    viscous and mass terms);
  * A_gamma = A + gamma B^T M_p^-1 B (Sec. 3, Eq. (augstokessys), W = M_p), Dirichlet
    rows and columns replaced by the identity;
  * vertex stars (Sec. 4.1, Eq. (viim)): the free nodes strictly inside star(v),
    (2k - 1)^d of them for an interior vertex;
  * P_H: coarse Q_k basis evaluated at the fine nodes; P~ = P_H - sum_K E_K A_K^-1
    E_K^T G P_H over the coarse-cell interiors (Eq. (Ptilde), the reading of
    oracle/mg.py); restriction by transposition.

Reading: the paper states dim V_i = (k - 1)^d for the star spaces (Sec. 5.2.2, the
paragraph before Table k); the free nodes strictly inside a 2x2(x2)-cell star of
Q_k number (2k - 1)^d per component, which is the space the smoother inverts for
k = 2 as well (3^d nodes), so (2k - 1)^d is used.
"""
from __future__ import annotations

import itertools
from functools import cached_property

import numpy as np
import scipy.sparse as sp

from .fem import assemble, dirichlet_rows_cols, multi_index, multi_index_grid


# ---------------------------------------------------------------------------
# 1D tables
# ---------------------------------------------------------------------------
def lagrange_nodes(k):
    return np.linspace(-1.0, 1.0, k + 1)


def lagrange_1d(k, xi):
    """Values (len(xi), k + 1) of the degree-k Lagrange polynomials on equispaced nodes."""
    t = lagrange_nodes(k)
    xi = np.atleast_1d(np.asarray(xi, float))
    out = np.ones((len(xi), k + 1))
    for a in range(k + 1):
        for b in range(k + 1):
            if b != a:
                out[:, a] *= (xi - t[b]) / (t[a] - t[b])
    return out


def lagrange_1d_deriv(k, xi):
    """Derivatives (len(xi), k + 1): product rule over the factors of each polynomial."""
    t = lagrange_nodes(k)
    xi = np.atleast_1d(np.asarray(xi, float))
    out = np.zeros((len(xi), k + 1))
    for a in range(k + 1):
        for m in range(k + 1):
            if m == a:
                continue
            term = np.full(len(xi), 1.0 / (t[a] - t[m]))
            for b in range(k + 1):
                if b != a and b != m:
                    term = term * (xi - t[b]) / (t[a] - t[b])
            out[:, a] += term
    return out


def pressure_exponents(d, k):
    """Exponent tuples alpha with |alpha| <= k - 1, by total degree, then e_0 before e_1 .."""
    al = [a for a in itertools.product(range(k), repeat=d) if sum(a) <= k - 1]
    return sorted(al, key=lambda a: (sum(a), [-v for v in a]))


class RefElementK:
    """Reference tables on [-1, 1]^d for Q_k velocities and P_(k-1) pressures."""

    def __init__(self, d, k):
        self.d, self.k = d, k
        self.mi = multi_index(d, k + 1)              # node / point multi-indices, x fastest
        self.nb = self.mi.shape[0]                   # (k + 1)^d
        g, w = np.polynomial.legendre.leggauss(k + 1)
        self.gauss_pts, self.gauss_wts = g, w
        self.nq = self.nb
        self.xq = g[self.mi]                         # (nq, d)
        self.wq = np.prod(w[self.mi], axis=1)
        L = lagrange_1d(k, g)                        # L[q, a]
        dL = lagrange_1d_deriv(k, g)
        self.phi = np.ones((self.nq, self.nb))
        self.dphi = np.ones((self.nq, self.nb, d))
        for ax in range(d):
            qa = self.mi[:, ax][:, None]
            aa = self.mi[:, ax][None, :]
            self.phi *= L[qa, aa]
            for j in range(d):
                self.dphi[:, :, j] *= (dL if j == ax else L)[qa, aa]
        self.alpha = pressure_exponents(d, k)
        self.npr = len(self.alpha)
        self.psi = np.stack([np.prod(self.xq ** np.array(a)[None, :], axis=1) for a in self.alpha], -1)


class MeshK:
    """Uniform mesh of (0, 1)^d with n[ax] cells per direction and its Q_k lattice."""

    def __init__(self, d, n, k):
        self.d, self.k = d, k
        self.n = (int(n),) * d if np.isscalar(n) else tuple(int(v) for v in n)
        self.h = tuple(1.0 / v for v in self.n)
        self.nn = tuple(k * v + 1 for v in self.n)
        self.N = int(np.prod(self.nn))
        self.ncells = int(np.prod(self.n))
        self.ref = RefElementK(d, k)
        self.detJ = float(np.prod([hk / 2.0 for hk in self.h]))
        self.stride = np.cumprod((1,) + self.nn[:-1])

    @cached_property
    def cells(self):
        return multi_index_grid(self.n)

    @cached_property
    def cell_nodes(self):
        g = self.k * self.cells[:, None, :] + self.ref.mi[None, :, :]
        return (g * self.stride).sum(-1)

    @cached_property
    def cell_dofs(self):
        return np.concatenate([a * self.N + self.cell_nodes for a in range(self.d)], axis=1)

    @cached_property
    def nodes(self):
        return multi_index_grid(self.nn)

    @cached_property
    def boundary_node(self):
        m = np.zeros(self.N, bool)
        for ax in range(self.d):
            m |= (self.nodes[:, ax] == 0) | (self.nodes[:, ax] == self.nn[ax] - 1)
        return m

    @cached_property
    def boundary_dof(self):
        return np.tile(self.boundary_node, self.d)

    @property
    def nu(self):
        return self.d * self.N

    @property
    def npres(self):
        return self.ref.npr * self.ncells

    def node_index(self, multi):
        return (np.asarray(multi) * self.stride).sum(-1)

    def node_coords(self):
        return self.nodes * (np.array(self.h) / self.k)

    @cached_property
    def grad_phi(self):
        return self.ref.dphi * (2.0 / np.array(self.h))[None, None, :]

    @cached_property
    def wdet(self):
        return self.ref.wq * self.detJ

    @cached_property
    def strain_basis(self):
        d, nb = self.d, self.ref.nb
        g = self.grad_phi
        e = np.zeros((self.ref.nq, d * nb, d, d))
        for al in range(d):
            cols = slice(al * nb, (al + 1) * nb)
            e[:, cols, al, :] += 0.5 * g
            e[:, cols, :, al] += 0.5 * g
        return e

    @cached_property
    def div_basis(self):
        g = self.grad_phi
        return np.concatenate([g[:, :, al] for al in range(self.d)], axis=1)

    @cached_property
    def B_elem(self):
        """[B_K]_(p, j) = -(psi_p, div phi_j)_K."""
        return -np.einsum("q,qa,qj->aj", self.wdet, self.ref.psi, self.div_basis)

    @cached_property
    def M_elem(self):
        return np.einsum("q,qa,qb->ab", self.wdet, self.ref.psi, self.ref.psi)

    def AL_elem(self, gamma):
        B = self.B_elem
        return gamma * B.T @ np.linalg.solve(self.M_elem, B)

    def A_elem(self, mu):
        """(2 mu eps(phi_j) : eps(phi_i))_K for every cell; mu sampled at the Gauss points."""
        e = self.strain_basis
        ee = np.einsum("qikl,qjkl->qij", e, e)
        return np.einsum("q,cq,qij->cij", 2.0 * self.wdet, mu, ee)


class LevelK:
    """Assembled FP64 operators of one level (scalar mu at the Gauss points).

    W = "Mp": augmentation weight M_p (the P1 pairing); "Mp_mu": M_p(1/mu) in the
    augmentation too, gamma B_K^T M_K(1/mu)^-1 B_K per cell (the P2 pairing, Eq. (P1P2)).
    """

    def __init__(self, d, n, k, mu, gamma, W="Mp"):
        self.mesh = m = MeshK(d, n, k)
        self.gamma = float(gamma)
        self.mu = np.asarray(mu, float)
        self.bdof = m.boundary_dof
        self.free = ~self.bdof
        self.W = W
        dofs = m.cell_dofs
        pdofs = np.arange(m.npres).reshape(m.ncells, m.ref.npr)
        self.Mp_mu_blocks = np.einsum("q,cq,qa,qb->cab", m.wdet, 1.0 / self.mu, m.ref.psi, m.ref.psi)
        if W == "Mp":
            G_elem = m.AL_elem(gamma)
            self.W_blocks = np.broadcast_to(m.M_elem, (m.ncells,) + m.M_elem.shape)
        elif W == "Mp_mu":
            Bk = m.B_elem
            G_elem = gamma * np.einsum("aj,cab,bk->cjk", Bk, np.linalg.inv(self.Mp_mu_blocks), Bk)
            self.W_blocks = self.Mp_mu_blocks
        else:
            raise ValueError(W)
        self.A_raw = assemble(m, m.A_elem(self.mu), dofs, dofs, (m.nu, m.nu))
        self.G_raw = assemble(m, G_elem, dofs, dofs, (m.nu, m.nu))
        self.B_raw = assemble(m, m.B_elem, pdofs, dofs, (m.npres, m.nu))
        f = sp.diags(self.free.astype(float))
        self.A = dirichlet_rows_cols((self.A_raw + self.G_raw).tocsr(), self.bdof)
        self.G = (f @ self.G_raw @ f).tocsr()
        self.B = (self.B_raw @ f).tocsr()
        self.Bt = self.B.T.tocsr()

    def load_vector(self, f_qp):
        """F_(alpha,i) = sum_q w |J| f_alpha(x_q) phi_i(x_q); f_qp: (ncells, nq, d)."""
        m = self.mesh
        F = np.zeros(m.nu)
        loc = np.einsum("q,cqa,qi->cai", m.wdet, f_qp, m.ref.phi)
        np.add.at(F, m.cell_dofs, loc.reshape(m.ncells, -1))
        return F

    def gauss_points(self):
        """Physical Gauss points (ncells, nq, d)."""
        m = self.mesh
        return (m.cells[:, None, :] + 0.5 * (1.0 + m.ref.xq[None])) * np.array(m.h)


# ---------------------------------------------------------------------------
# vertex stars, transfers
# ---------------------------------------------------------------------------
def star_nodes_k(mesh: MeshK, vertex):
    """Free nodes strictly inside star(v): lattice offsets -(k-1) .. k-1 from k v."""
    k, out = mesh.k, []
    for o in multi_index(mesh.d, 2 * k - 1):
        g = k * np.asarray(vertex) + (o - (k - 1))
        if np.all(g > 0) and np.all(g < np.array(mesh.nn) - 1):
            out.append(int(mesh.node_index(g)))
    return np.array(out, dtype=np.int64)


def star_dofs_k(mesh: MeshK, vertex):
    nodes = star_nodes_k(mesh, vertex)
    return np.concatenate([a * mesh.N + nodes for a in range(mesh.d)])


def all_vertices_k(mesh: MeshK):
    return multi_index_grid(tuple(v + 1 for v in mesh.n))


def star_patches_k(level: LevelK):
    from .mg import PatchSet
    m = level.mesh
    return PatchSet(level.A, [star_dofs_k(m, v) for v in all_vertices_k(m)])


def prolongation_1d_k(nc, k):
    """Coarse Q_k basis on nc cells evaluated at the fine Q_k nodes (2 nc cells)."""
    nf_nodes, nc_nodes = 2 * k * nc + 1, k * nc + 1
    P = np.zeros((nf_nodes, nc_nodes))
    for f in range(nf_nodes):
        x = f / (2.0 * k * nc)
        c = min(int(x * nc), nc - 1)
        xi = 2.0 * (x * nc - c) - 1.0
        P[f, k * c: k * c + k + 1] += lagrange_1d(k, [xi])[0]
    P[np.abs(P) < 1e-15] = 0.0
    return P


def standard_prolongation_k(coarse: MeshK, fine: MeshK):
    """P_H on velocity vectors, fine Dirichlet rows and coarse Dirichlet columns zeroed."""
    P = sp.csr_matrix(np.ones((1, 1)))
    for ax in range(coarse.d):            # x fastest => kron(P_z, kron(P_y, P_x))
        P = sp.kron(sp.csr_matrix(prolongation_1d_k(coarse.n[ax], coarse.k)), P, format="csr")
    P = sp.block_diag([P] * coarse.d, format="csr")
    rf = sp.diags((~fine.boundary_dof).astype(float))
    cf = sp.diags((~coarse.boundary_dof).astype(float))
    return (rf @ P @ cf).tocsr()


def coarse_cell_interiors_k(coarse: MeshK, fine: MeshK):
    """Free fine dofs strictly inside each coarse cell = star of the fine vertex 2K + 1."""
    return [star_dofs_k(fine, 2 * K + 1) for K in coarse.cells]


def robust_prolongation_k(coarse: MeshK, fine_level: LevelK):
    """P~ = P_H - sum_K E_K A_K^-1 E_K^T G P_H with G = gamma B^T M_p^-1 B (fine)."""
    from .mg import PatchSet
    fine = fine_level.mesh
    PH = standard_prolongation_k(coarse, fine)
    ps = PatchSet(fine_level.A, coarse_cell_interiors_k(coarse, fine))
    rows, cols, vals = [], [], []
    for _, idx, _, inv in ps.groups.values():
        for j in range(idx.shape[0]):
            rows.append(np.repeat(idx[j], idx.shape[1]))
            cols.append(np.tile(idx[j], idx.shape[1]))
            vals.append(inv[j].ravel())
    Ablk = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=fine_level.A.shape).tocsr()
    return (PH - Ablk @ (fine_level.G @ PH)).tocsr(), PH


def two_level_error(fine: LevelK, coarse: LevelK, smoother="star", transfer="robust", steps=2, tau=0.25):
    """Dense error propagation of one two-level cycle on the free dofs: Richardson
    pre/post smoothing with D^-1 (the star PSC operator, or point Jacobi), the exact
    coarse solve on the rediscretised coarse operator, prolongation P~ or P_H and its
    transpose as restriction (Sec. 4)."""
    A = fine.A.toarray()
    n = A.shape[0]
    if smoother == "star":
        ps = star_patches_k(fine)
        Dinv = np.stack([ps.apply(e) for e in np.eye(n)], 1)
    else:
        Dinv = np.diag(1.0 / np.diag(A))
    S = np.eye(n) - tau * Dinv @ A
    if transfer == "robust":
        P = robust_prolongation_k(coarse.mesh, fine)[0].toarray()
    else:
        P = standard_prolongation_k(coarse.mesh, fine.mesh).toarray()
    Ac = coarse.A.toarray()
    fc = coarse.free
    Pf = P[:, fc]
    C = np.eye(n) - Pf @ np.linalg.solve(Ac[np.ix_(fc, fc)], Pf.T @ A)
    E = np.linalg.matrix_power(S, steps) @ C @ np.linalg.matrix_power(S, steps)
    f = fine.free
    return E[np.ix_(f, f)]


class HierarchyK:
    """Levels 0 (coarsest) .. L-1 of order k with the gamma-robust cycle of Sec. 4: s steps of
    GMRES right-preconditioned by the star PSC operator (smoother "gmres"), or of damped
    Richardson on it ("richardson", damping tau, default 2^-d), or point Jacobi ("jacobi",
    the negative control); robust (or standard) prolongation, its transpose as restriction,
    exact coarse solve; cycle "V" or "F" (the paper's 3D runs use an F-cycle, Table linear;
    the F-cycle is the recursion of oracle/mg.py: the coarse correction is an F-cycle from
    zero, then a V-cycle from its result).  The interface the oracle's Stokes solver uses
    (levels, cycle)."""

    def __init__(self, d, n, k, mus, gamma, steps=5, smoother="gmres", transfer="robust", W="Mp", cycle="V",
                 tau=None):
        import scipy.linalg as sla
        if cycle not in ("V", "F"):
            raise ValueError(cycle)
        if smoother not in ("gmres", "richardson", "jacobi"):
            raise ValueError(smoother)
        L = len(mus)
        self.d, self.k, self.L, self.steps, self.smoother = d, k, L, steps, smoother
        self.cycle_type = cycle
        self.tau = tau if tau is not None else (2.0 ** -d if smoother == "richardson" else 1.0)
        self.levels = []
        for lvl in range(L):
            f = 2 ** (L - 1 - lvl)
            nl = tuple(v // f for v in ((n,) * d if np.isscalar(n) else n))
            self.levels.append(LevelK(d, nl, k, mus[lvl], gamma, W))
        self.patches = [None] + [star_patches_k(lv) if smoother != "jacobi" else None for lv in self.levels[1:]]
        self.P = [None]
        for lvl in range(1, L):
            if transfer == "robust":
                self.P.append(robust_prolongation_k(self.levels[lvl - 1].mesh, self.levels[lvl])[0])
            else:
                self.P.append(standard_prolongation_k(self.levels[lvl - 1].mesh, self.levels[lvl].mesh))
        A0 = self.levels[0].A
        self.coarse_free = np.flatnonzero(self.levels[0].free)
        self._chol = sla.cho_factor(A0[self.coarse_free][:, self.coarse_free].toarray(), lower=True)

    def Dinv(self, lvl):
        if self.smoother == "jacobi":
            dg = self.levels[lvl].A.diagonal()
            return lambda r: r / dg
        return self.patches[lvl].apply

    def coarse_solve(self, b):
        import scipy.linalg as sla
        x = np.zeros_like(b)
        x[self.coarse_free] = sla.cho_solve(self._chol, b[self.coarse_free])
        return x

    def smooth(self, lvl, x, b):
        from .mg import smooth_gmres, smooth_richardson
        A = self.levels[lvl].A
        if self.smoother == "richardson":
            return smooth_richardson(A, self.Dinv(lvl), x, b, self.steps, self.tau)
        return smooth_gmres(A, self.Dinv(lvl), x, b, self.steps)

    def vcycle(self, b, lvl=None, x0=None):
        lvl = self.L - 1 if lvl is None else lvl
        if lvl == 0:
            return self.coarse_solve(b)
        A = self.levels[lvl].A
        x = self.smooth(lvl, np.zeros_like(b) if x0 is None else x0.copy(), b)
        ec = self.vcycle(self.P[lvl].T @ (b - A @ x), lvl - 1)
        x = x + self.P[lvl] @ ec
        return self.smooth(lvl, x, b)

    def fcycle(self, b, lvl=None):
        lvl = self.L - 1 if lvl is None else lvl
        if lvl == 0:
            return self.coarse_solve(b)
        A = self.levels[lvl].A
        x = self.smooth(lvl, np.zeros_like(b), b)
        bc = self.P[lvl].T @ (b - A @ x)
        ec = self.fcycle(bc, lvl - 1)
        if lvl - 1 > 0:
            ec = self.vcycle(bc, lvl - 1, x0=ec)
        x = x + self.P[lvl] @ ec
        return self.smooth(lvl, x, b)

    def cycle(self, b):
        return self.fcycle(b) if self.cycle_type == "F" else self.vcycle(b)
