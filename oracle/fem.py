"""FP64 oracle: the [Q2]^d x P1^disc discretisation of the (augmented) Stokes system.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
CPU restatement of what the GPU library computes; only the tests, the smoke
check and the CPU-baseline leg of the benchmark may import it.  It shares no
code with the CUDA path and never reads anything the CUDA path produced.

Everything here is the textbook definition written out with NumPy/SciPy:
full 3^d Gauss quadrature, explicit element matrices, global assembly with
scipy.sparse, Dirichlet rows/columns replaced by the identity.

Paper passages followed:
  * weak form and operators, Sec. 2, Eq. (stokessys): [A]_ij = (2 mu eps(phi_i), eps(phi_j)),
    [B]_ij = -(psi_i, div phi_j);
  * pressure mass matrices, Eq. (inv-visc-mass): [M_p(1/mu)]_ij = (mu^-1 psi_i, psi_j);
  * augmented system, Sec. 3, Eq. (augstokessys): A_gamma = A + gamma B^T W^-1 B with W = M_p;
  * tensor viscosity, Eq. (stokes-lin): the stress is C : eps(u) with a 4th-order C;
  * spaces V_h^k x Q_h^(k-1) with k = 2 (Sec. 4), on uniform quad/hex meshes of (0,1)^d.

Conventions (shared with the C ABI as a data contract, not as code):
  * node lattice (2n_k+1 nodes per direction), node index x-fastest;
  * velocity vector = d blocks of N nodal values (component-major);
  * pressure basis on each cell: {1, xi_0, .., xi_(d-1)} in reference coordinates
    xi in [-1,1]^d, pressure vector laid out [cell][d+1];
  * tensor coefficients in Mandel notation, upper triangle row-major:
    2D (e00, e11, sqrt2 e01) -> 6 entries; 3D (e00, e11, e22, sqrt2 e12,
    sqrt2 e02, sqrt2 e01) -> 21 entries.
"""
from __future__ import annotations

import itertools
import math
from functools import cached_property

import numpy as np
import scipy.sparse as sp

GAUSS_PTS = np.array([-math.sqrt(0.6), 0.0, math.sqrt(0.6)])
GAUSS_WTS = np.array([5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0])


def lagrange_q2(xi):
    """The three quadratic Lagrange polynomials on the nodes -1, 0, 1."""
    xi = np.asarray(xi, float)
    return np.stack([0.5 * xi * (xi - 1.0), 1.0 - xi * xi, 0.5 * xi * (xi + 1.0)], -1)


def lagrange_q2_deriv(xi):
    xi = np.asarray(xi, float)
    return np.stack([xi - 0.5, -2.0 * xi, xi + 0.5], -1)


def multi_index(d, m=3):
    """All d-tuples over range(m), first entry fastest; shape (m^d, d)."""
    idx = np.array(list(itertools.product(range(m), repeat=d)))
    return idx[:, ::-1].copy()


def mandel_size(d):
    return 3 if d == 2 else 6


def mandel_pairs(d):
    """(k, l) tensor index and weight of each Mandel component."""
    if d == 2:
        return [((0, 0), 1.0), ((1, 1), 1.0), ((0, 1), math.sqrt(2.0))]
    return [((0, 0), 1.0), ((1, 1), 1.0), ((2, 2), 1.0),
            ((1, 2), math.sqrt(2.0)), ((0, 2), math.sqrt(2.0)), ((0, 1), math.sqrt(2.0))]


def unpack_mandel(c_packed, d):
    """Upper-triangle row-major packed Mandel matrices -> full (.., m, m)."""
    m = mandel_size(d)
    iu = np.triu_indices(m)
    full = np.zeros(c_packed.shape[:-1] + (m, m))
    full[..., iu[0], iu[1]] = c_packed
    full[..., iu[1], iu[0]] = c_packed
    return full


class RefElement:
    """Reference tables on [-1,1]^d: Q2 basis, derivatives, P1 pressure basis."""

    def __init__(self, d):
        self.d = d
        self.mi = multi_index(d)                    # node / point multi-indices
        self.nb = self.mi.shape[0]                  # 3^d
        self.nq = self.nb
        self.xq = GAUSS_PTS[self.mi]                # (nq, d) reference points
        self.wq = np.prod(GAUSS_WTS[self.mi], axis=1)
        L = lagrange_q2(GAUSS_PTS)                  # L[q, a]
        dL = lagrange_q2_deriv(GAUSS_PTS)
        self.phi = np.ones((self.nq, self.nb))
        self.dphi = np.ones((self.nq, self.nb, d))  # reference derivatives
        for k in range(d):
            qk = self.mi[:, k][:, None]
            ak = self.mi[:, k][None, :]
            self.phi *= L[qk, ak]
            for j in range(d):
                self.dphi[:, :, j] *= (dL if j == k else L)[qk, ak]
        self.psi = np.concatenate([np.ones((self.nq, 1)), self.xq], axis=1)  # (nq, d+1)


class Mesh:
    """Uniform mesh of (0,1)^d with n[k] cells per direction and its Q2 lattice."""

    def __init__(self, d, n):
        self.d = d
        self.n = (int(n),) * d if np.isscalar(n) else tuple(int(v) for v in n)
        self.h = tuple(1.0 / v for v in self.n)
        self.nn = tuple(2 * v + 1 for v in self.n)
        self.N = int(np.prod(self.nn))
        self.ncells = int(np.prod(self.n))
        self.ref = RefElement(d)
        self.detJ = float(np.prod([hk / 2.0 for hk in self.h]))
        self.stride = np.cumprod((1,) + self.nn[:-1])

    # --- index bookkeeping ---------------------------------------------------
    @cached_property
    def cells(self):
        return multi_index_grid(self.n)

    @cached_property
    def cell_nodes(self):
        """(ncells, 3^d) global node of each local node."""
        g = 2 * self.cells[:, None, :] + self.ref.mi[None, :, :]
        return (g * self.stride).sum(-1)

    @cached_property
    def cell_dofs(self):
        """(ncells, d*3^d) global velocity dofs, local order component-major."""
        return np.concatenate([a * self.N + self.cell_nodes for a in range(self.d)], axis=1)

    @cached_property
    def nodes(self):
        return multi_index_grid(self.nn)

    @cached_property
    def boundary_node(self):
        m = np.zeros(self.N, bool)
        for k in range(self.d):
            m |= (self.nodes[:, k] == 0) | (self.nodes[:, k] == self.nn[k] - 1)
        return m

    @cached_property
    def boundary_dof(self):
        return np.tile(self.boundary_node, self.d)

    @property
    def nu(self):
        return self.d * self.N

    @property
    def npres(self):
        return (self.d + 1) * self.ncells

    def node_index(self, multi):
        return (np.asarray(multi) * self.stride).sum(-1)

    def node_coords(self):
        return self.nodes * (np.array(self.h) / 2.0)

    # --- physical tables -----------------------------------------------------
    @cached_property
    def grad_phi(self):
        """(nq, nb, d) physical derivatives (affine, axis-aligned cells)."""
        return self.ref.dphi * (2.0 / np.array(self.h))[None, None, :]

    @cached_property
    def wdet(self):
        return self.ref.wq * self.detJ

    @cached_property
    def strain_basis(self):
        """eps(phi_(alpha,a)) at each point: (nq, d*nb, d, d)."""
        d, nb = self.d, self.ref.nb
        g = self.grad_phi
        e = np.zeros((self.ref.nq, d * nb, d, d))
        for al in range(d):
            cols = slice(al * nb, (al + 1) * nb)
            e[:, cols, al, :] += 0.5 * g
            e[:, cols, :, al] += 0.5 * g
        return e

    @cached_property
    def mandel_basis(self):
        """Mandel vectors of eps(phi_i): (nq, d*nb, m)."""
        e = self.strain_basis
        return np.stack([w * e[:, :, k, l] for (k, l), w in mandel_pairs(self.d)], -1)

    @cached_property
    def div_basis(self):
        """div phi_(alpha,a) = d phi_a / d x_alpha: (nq, d*nb)."""
        g = self.grad_phi
        return np.concatenate([g[:, :, al] for al in range(self.d)], axis=1)

    # --- element matrices ----------------------------------------------------
    @cached_property
    def B_elem(self):
        """[B_K]_(a, j) = -(psi_a, div phi_j)_K, shape (d+1, d*nb)."""
        return -np.einsum("q,qa,qj->aj", self.wdet, self.ref.psi, self.div_basis)

    @cached_property
    def M_elem(self):
        """[M_K]_ab = (psi_a, psi_b)_K."""
        return np.einsum("q,qa,qb->ab", self.wdet, self.ref.psi, self.ref.psi)

    def Mmu_elem(self, mu):
        """[M_K(1/mu)]_ab = (mu^-1 psi_a, psi_b)_K for every cell: (ncells, d+1, d+1)."""
        return np.einsum("q,cq,qa,qb->cab", self.wdet, 1.0 / mu, self.ref.psi, self.ref.psi)

    def AL_elem(self, gamma):
        """gamma B_K^T M_K^-1 B_K (the same on every cell of a uniform mesh)."""
        B = self.B_elem
        return gamma * B.T @ np.linalg.solve(self.M_elem, B)

    def A_elem(self, coeff, kind="scalar", cells=None):
        """Viscous element matrices (2 mu eps_i : eps_j) or (C eps_j) : eps_i."""
        if kind == "scalar":
            e = self.strain_basis
            ee = np.einsum("qikl,qjkl->qij", e, e)
            return np.einsum("q,cq,qij->cij", 2.0 * self.wdet, coeff, ee)
        mv = self.mandel_basis
        C = unpack_mandel(coeff, self.d)
        return np.einsum("q,qim,cqmn,qjn->cij", self.wdet, mv, C, mv)

    def Agamma_elem(self, coeff, gamma, kind="scalar"):
        return self.A_elem(coeff, kind) + self.AL_elem(gamma)[None]


def multi_index_grid(n):
    """All multi-indices of a box of shape n, first index fastest."""
    grids = np.meshgrid(*[np.arange(v) for v in n], indexing="ij")
    d = len(n)
    return np.stack([g.transpose(*reversed(range(d))).reshape(-1) for g in grids], -1)


# ---------------------------------------------------------------------------
# global assembly
# ---------------------------------------------------------------------------
def assemble(mesh, Ke, row_dofs, col_dofs, shape, chunk=4096):
    """sum_K scatter of element matrices Ke (ncells, r, c) into a CSR matrix."""
    out = sp.csr_matrix(shape)
    nc = Ke.shape[0] if Ke.ndim == 3 else mesh.ncells
    for s in range(0, nc, chunk):
        e = slice(s, min(nc, s + chunk))
        K = Ke[e] if Ke.ndim == 3 else np.broadcast_to(Ke, (e.stop - e.start,) + Ke.shape)
        r = np.repeat(row_dofs[e][:, :, None], K.shape[2], axis=2)
        c = np.repeat(col_dofs[e][:, None, :], K.shape[1], axis=1)
        out = out + sp.coo_matrix((K.ravel(), (r.ravel(), c.ravel())), shape=shape).tocsr()
    return out.tocsr()


def dirichlet_rows_cols(A, bdof):
    """Zero the Dirichlet rows and columns and put 1 on their diagonal."""
    f = sp.diags((~bdof).astype(float))
    return (f @ A @ f + sp.diags(bdof.astype(float))).tocsr()


class Level:
    """One multigrid level: mesh, coefficients and assembled FP64 operators.

    Level operators are obtained by rediscretising on the level's mesh with the
    level's own coefficient samples (Sec. 5.1).
    """

    def __init__(self, d, n, coeff, gamma, kind="scalar", mu_eff=None, W="Mp"):
        self.mesh = m = Mesh(d, n)
        self.gamma = float(gamma)
        self.kind = kind
        self.W = W
        self.coeff = np.asarray(coeff, float)
        self.mu = self.coeff if kind == "scalar" else np.asarray(mu_eff, float)
        bd = m.boundary_dof
        self.bdof = bd
        self.free = ~bd
        dofs = m.cell_dofs
        nu = m.nu
        pdofs = np.arange(m.npres).reshape(m.ncells, d + 1)
        # unconstrained operators
        self.A_raw = assemble(m, m.A_elem(self.coeff, kind), dofs, dofs, (nu, nu))
        self.Mp_mu_blocks = m.Mmu_elem(self.mu)
        if W == "Mp":            # W = M_p: the same AL block on every cell
            G_elem = m.AL_elem(gamma)
        elif W == "Mp_mu":       # W = M_p(1/mu): gamma B_K^T M_K(1/mu)^-1 B_K per cell
            Bk = m.B_elem
            G_elem = gamma * np.einsum("aj,cab,bk->cjk", Bk, np.linalg.inv(self.Mp_mu_blocks), Bk)
        else:
            raise ValueError(W)
        self.G_raw = assemble(m, G_elem, dofs, dofs, (nu, nu))
        self.B_raw = assemble(m, m.B_elem, pdofs, dofs, (m.npres, nu))
        self.Agam_raw = (self.A_raw + self.G_raw).tocsr()
        # Dirichlet-constrained forms: identity rows/cols for A, masked columns for B
        f = sp.diags(self.free.astype(float))
        self.A = dirichlet_rows_cols(self.Agam_raw, bd)
        self.G = (f @ self.G_raw @ f).tocsr()
        self.B = (self.B_raw @ f).tocsr()
        self.Bt = self.B.T.tocsr()
        self.W_blocks = (np.broadcast_to(m.M_elem, (m.ncells,) + m.M_elem.shape)
                         if W == "Mp" else self.Mp_mu_blocks)

    def load_vector(self, f_qp):
        """F_(alpha,i) = sum_q w |J| f_alpha(x_q) phi_i(x_q)."""
        m = self.mesh
        F = np.zeros(m.nu)
        loc = np.einsum("q,cqa,qi->cai", m.wdet, f_qp, m.ref.phi)  # (ncells, d, nb)
        np.add.at(F, m.cell_dofs, loc.reshape(m.ncells, -1))
        return F

    def apply_Agamma(self, x):
        return self.A @ x


def cell_local_apply(mesh, coeff, gamma, x, cells, kind="scalar"):
    """(A_gamma,K x_K) for a subset of cells, without any global assembly."""
    Ke = mesh.Agamma_elem(coeff[cells], gamma, kind)
    return np.einsum("cij,cj->ci", Ke, x[mesh.cell_dofs[cells]])
