"""FP64 oracle: the gamma-robust multigrid V-cycle for A_gamma.

TEST INFRASTRUCTURE ONLY (see oracle/fem.py).  Plain restatement of Sec. 4:

  * PSC smoother (Sec. 4.1): u <- u + tau D^-1 r with
    D^-1 = sum_i I_i A_i^-1 I_i^*, A_i the restriction of the assembled
    A_(h,gamma) to V_i;
  * vertex-star space decomposition, Eq. (viim): V_i = {v in V_h : supp v in
    star(v_i)}, for every vertex v_i of the mesh.  On a Q2 lattice these are
    the free dofs at the 3^d nodes within one half-cell of the vertex;
  * the relaxation is the GMRES-accelerated PSC iteration of Fig. (algo-outline)
    ("GMRES -> Block Jacobi"): s GMRES steps right-preconditioned by D^-1
    (the reading taken for the unstated preconditioning side); a damped
    Richardson variant and a point-Jacobi negative control are also here;
  * standard prolongation P_H = nested Q2 interpolation (coarse basis
    functions evaluated at the fine nodes), Sec. 4.2;
  * robust prolongation, Eq. (Ptilde): P~ u_H = P_H u_H - u~ with u~ in V^_h
    solving a_(h,gamma)(u~, v^) = gamma (Pi div P_H u_H, Pi div v^) for all v^
    in V^_h (the AL-term right-hand side), V^_h = functions supported in one
    coarse cell; restriction is its transpose;
  * the coarsest level is solved by a dense Cholesky factorisation (the paper
    uses a sparse direct solver there, Sec. 5.1).

Patch matrices are taken from the ASSEMBLED matrix, as in Sec. 5.1.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .fem import Level, Mesh, multi_index, multi_index_grid


# ---------------------------------------------------------------------------
# vertex stars
# ---------------------------------------------------------------------------
def star_nodes(mesh: Mesh, vertex):
    """Free Q2 nodes in the interior of star(v): offsets -1, 0, 1 half-cells.

    A node at offset o from the vertex lies strictly inside the star iff
    |o_k| <= 1 in every direction; it is free iff it is not on the boundary.
    Order: offsets x-fastest.
    """
    out = []
    for o in multi_index(mesh.d):
        g = 2 * np.asarray(vertex) + (o - 1)
        if np.all(g > 0) and np.all(g < np.array(mesh.nn) - 1):
            out.append(int(mesh.node_index(g)))
    return np.array(out, dtype=np.int64)


def star_dofs(mesh: Mesh, vertex):
    nodes = star_nodes(mesh, vertex)
    return np.concatenate([a * mesh.N + nodes for a in range(mesh.d)])


def all_vertices(mesh: Mesh):
    return multi_index_grid(tuple(v + 1 for v in mesh.n))


def extract_blocks(A, index_sets):
    """Dense A[idx, idx] for every index set (same length within a group)."""
    A = A.tocsr()
    out = []
    for idx in index_sets:
        out.append(A[idx][:, idx].toarray())
    return out


class PatchSet:
    """Index sets and FP64 inverses of dense local problems, grouped by size."""

    def __init__(self, A, index_sets):
        self.groups = {}
        by_size = {}
        for i, idx in enumerate(index_sets):
            by_size.setdefault(len(idx), []).append(i)
        for size, ids in by_size.items():
            idx = np.stack([index_sets[i] for i in ids])
            blocks = np.stack(extract_blocks(A, [index_sets[i] for i in ids]))
            inv = np.empty_like(blocks)
            for j, Ab in enumerate(blocks):
                c = sla.cho_factor(Ab, lower=True)
                inv[j] = sla.cho_solve(c, np.eye(size))
            self.groups[size] = (np.array(ids), idx, blocks, inv)
        self.index_sets = index_sets

    def apply(self, r):
        """sum_i I_i A_i^-1 I_i^T r."""
        z = np.zeros_like(r)
        for _, idx, _, inv in self.groups.values():
            y = np.einsum("pij,pj->pi", inv, r[idx])
            np.add.at(z, idx, y)
        return z

    def local_solve(self, r):
        """Per-set solutions A_i^-1 r[idx_i], as a dict id -> vector."""
        out = {}
        for ids, idx, _, inv in self.groups.values():
            y = np.einsum("pij,pj->pi", inv, r[idx])
            for i, v in zip(ids, y):
                out[int(i)] = v
        return out


def star_patches(level: Level):
    m = level.mesh
    sets = [star_dofs(m, v) for v in all_vertices(m)]
    return PatchSet(level.A, sets)


# ---------------------------------------------------------------------------
# transfers
# ---------------------------------------------------------------------------
def prolongation_1d(nc):
    """Coarse Q2 basis on nc cells evaluated at the fine Q2 nodes (2nc cells).

    Row f = fine node at x = f/(4 nc); the coarse cell containing it and the
    three quadratic Lagrange polynomials of that cell give the weights.
    """
    nf_nodes, nc_nodes = 4 * nc + 1, 2 * nc + 1
    P = np.zeros((nf_nodes, nc_nodes))
    for f in range(nf_nodes):
        x = f / (4.0 * nc)
        c = min(int(x * nc), nc - 1)
        xi = 2.0 * (x * nc - c) - 1.0             # reference coordinate in the coarse cell
        vals = [0.5 * xi * (xi - 1.0), 1.0 - xi * xi, 0.5 * xi * (xi + 1.0)]
        for a in range(3):
            P[f, 2 * c + a] += vals[a]
    P[np.abs(P) < 1e-15] = 0.0
    return P


def standard_prolongation(coarse: Mesh, fine: Mesh):
    """P_H on velocity vectors, with fine Dirichlet rows and coarse Dirichlet columns zeroed."""
    P = sp.csr_matrix(np.ones((1, 1)))
    for k in range(coarse.d):            # x fastest => kron(P_z, kron(P_y, P_x))
        P = sp.kron(sp.csr_matrix(prolongation_1d(coarse.n[k])), P, format="csr")
    P = sp.block_diag([P] * coarse.d, format="csr")
    rf = sp.diags((~fine.boundary_dof).astype(float))
    cf = sp.diags((~coarse.boundary_dof).astype(float))
    return (rf @ P @ cf).tocsr()


def coarse_cell_interiors(coarse: Mesh, fine: Mesh):
    """int(K): free fine dofs strictly inside each coarse cell = star of the
    fine vertex at the cell's centre."""
    return [star_dofs(fine, 2 * K + 1) for K in coarse.cells]


def robust_prolongation(coarse: Mesh, fine_level: Level):
    """P~ = P_H - sum_K E_K A_K^-1 E_K^T G P_H with G = gamma B^T M_p^-1 B (fine)."""
    fine = fine_level.mesh
    PH = standard_prolongation(coarse, fine)
    sets = coarse_cell_interiors(coarse, fine)
    ps = PatchSet(fine_level.A, sets)
    rows, cols, vals = [], [], []
    for ids, idx, _, inv in ps.groups.values():
        for j in range(idx.shape[0]):
            r = np.repeat(idx[j], idx.shape[1])
            c = np.tile(idx[j], idx.shape[1])
            rows.append(r); cols.append(c); vals.append(inv[j].ravel())
    Ablk = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=fine_level.A.shape).tocsr()
    return (PH - Ablk @ (fine_level.G @ PH)).tocsr(), PH, ps


# ---------------------------------------------------------------------------
# smoothers
# ---------------------------------------------------------------------------
def smooth_richardson(A, Dinv, x, b, steps, tau):
    for _ in range(steps):
        x = x + tau * Dinv(b - A @ x)
    return x


def smooth_gmres(A, Dinv, x, b, steps):
    """s steps of GMRES on A x = b from x, right-preconditioned by Dinv.

    Minimises ||b - A x||_2 over x0 + Dinv K_s(A Dinv, r0); classical
    Gram-Schmidt, one pass; least squares on the small Hessenberg matrix.
    """
    r0 = b - A @ x
    beta = np.linalg.norm(r0)
    if beta == 0.0:
        return x
    V = [r0 / beta]
    Z = []
    H = np.zeros((steps + 1, steps))
    for j in range(steps):
        z = Dinv(V[j])
        w = A @ z
        Vm = np.stack(V, 1)
        h = Vm.T @ w
        w = w - Vm @ h
        H[: j + 1, j] = h
        H[j + 1, j] = np.linalg.norm(w)
        Z.append(z)
        V.append(w / H[j + 1, j] if H[j + 1, j] > 0 else np.zeros_like(w))
    e1 = np.zeros(steps + 1)
    e1[0] = beta
    y = np.linalg.lstsq(H, e1, rcond=None)[0]
    return x + np.stack(Z, 1) @ y


# ---------------------------------------------------------------------------
# hierarchy and V-cycle
# ---------------------------------------------------------------------------
class Hierarchy:
    """Levels 0 (coarsest) .. L-1 (finest) with smoother and transfer data.

    smoother: "gmres" (default), "richardson" or "jacobi" (point Jacobi,
    the standard-multigrid negative control); transfer: "robust" or "standard";
    cycle: "V" (default) or "F" (what the paper ran, Sec. 5.1).
    """

    def __init__(self, d, n, coeffs, gamma, kind="scalar", mu_eff=None,
                 smoother="gmres", steps=5, tau=None, transfer="robust", W="Mp", cycle="V"):
        L = len(coeffs)
        self.d, self.L = d, L
        self.levels = []
        for lvl in range(L):
            f = 2 ** (L - 1 - lvl)
            nl = tuple(v // f for v in ((n,) * d if np.isscalar(n) else n))
            me = None if mu_eff is None else mu_eff[lvl]
            self.levels.append(Level(d, nl, coeffs[lvl], gamma, kind, me, W))
        self.smoother, self.steps, self.transfer = smoother, steps, transfer
        if cycle not in ("V", "F"):
            raise ValueError(cycle)
        self.cycle_type = cycle
        self.tau = tau if tau is not None else (2.0 ** -d if smoother == "richardson" else 1.0)
        self.patches = [None] + [star_patches(lv) if smoother != "jacobi" else None
                                 for lv in self.levels[1:]]
        self.P = [None]
        self.PH = [None]
        self.interiors = [None]
        for lvl in range(1, L):
            if transfer == "robust":
                Pt, PH, ps = robust_prolongation(self.levels[lvl - 1].mesh, self.levels[lvl])
            else:
                PH = standard_prolongation(self.levels[lvl - 1].mesh, self.levels[lvl].mesh)
                Pt, ps = PH, None
            self.P.append(Pt)
            self.PH.append(PH)
            self.interiors.append(ps)
        A0 = self.levels[0].A
        self.coarse_free = np.flatnonzero(self.levels[0].free)
        self.coarse_chol = sla.cho_factor(A0[self.coarse_free][:, self.coarse_free].toarray(),
                                          lower=True)

    def Dinv(self, lvl):
        if self.smoother == "jacobi":
            dg = self.levels[lvl].A.diagonal()
            return lambda r: r / dg
        return self.patches[lvl].apply

    def coarse_solve(self, b):
        x = np.zeros_like(b)
        x[self.coarse_free] = sla.cho_solve(self.coarse_chol, b[self.coarse_free])
        return x

    def smooth(self, lvl, x, b):
        A = self.levels[lvl].A
        if self.smoother == "gmres":
            return smooth_gmres(A, self.Dinv(lvl), x, b, self.steps)
        return smooth_richardson(A, self.Dinv(lvl), x, b, self.steps, self.tau)

    def vcycle(self, b, lvl=None, x0=None):
        """One V-cycle for A_(lvl) x = b from x = x0 (default 0) (Sec. 4, Fig. algo-outline)."""
        lvl = self.L - 1 if lvl is None else lvl
        if lvl == 0:
            return self.coarse_solve(b)
        A = self.levels[lvl].A
        x = np.zeros_like(b) if x0 is None else x0.copy()
        x = self.smooth(lvl, x, b)
        r = b - A @ x
        bc = self.P[lvl].T @ r
        ec = self.vcycle(bc, lvl - 1)
        x = x + self.P[lvl] @ ec
        return self.smooth(lvl, x, b)

    def fcycle(self, b, lvl=None):
        """One F-cycle for A_(lvl) x = b from x = 0.

        The paper runs an F-cycle (Sec. 5.1) without defining it; this is the
        textbook recursion: as the V-cycle, but the coarse correction is an
        F-cycle on level lvl-1 from zero followed by a V-cycle on level lvl-1
        started from that result.  On the coarsest level both are the exact
        solve, so one solve is done.
        """
        lvl = self.L - 1 if lvl is None else lvl
        if lvl == 0:
            return self.coarse_solve(b)
        A = self.levels[lvl].A
        x = self.smooth(lvl, np.zeros_like(b), b)
        r = b - A @ x
        bc = self.P[lvl].T @ r
        ec = self.fcycle(bc, lvl - 1)
        if lvl - 1 > 0:
            ec = self.vcycle(bc, lvl - 1, x0=ec)
        x = x + self.P[lvl] @ ec
        return self.smooth(lvl, x, b)

    def cycle(self, b):
        """The configured multigrid cycle (V or F) on the finest level from 0."""
        return self.fcycle(b) if self.cycle_type == "F" else self.vcycle(b)
