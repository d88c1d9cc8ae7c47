"""Cell-local evaluations of the oracle's operators, for sampled outputs at full size.

Test infrastructure only.  At the workloads' full sizes (823,875 velocity dofs on the
3D 32^3 mesh) the oracle's assembled matrices and hierarchy take far longer than a test
may, but every output of one operator step depends on a handful of cells:

  * a row of A_gamma x (Secs. 2-3, Eqs. stokessys/augstokessys) on the 2^d cells around
    its node;
  * the vertex-star patch matrix A_v (Sec. 4.1, Eq. viim) on the 2^d cells around v;
  * an entry of z = sum_v I_v A_v^-1 I_v^T r on the <= 2^d stars that hold its node;
  * an entry of P~ e_c (Eq. Ptilde) on the one coarse cell that holds its node;
  * an entry of P~^T r_f on the coarse cells around its coarse node.

This module evaluates those outputs one by one from the oracle's element matrices
(`oracle.fem.Mesh`) and its 1D coarse-to-fine weights (`oracle.mg.prolongation_1d`),
with the same Dirichlet conventions as the assembled oracle (identity rows and
columns for A, zeroed fine rows and coarse columns for P_H).  Every evaluation also
returns the sum of the absolute values of its terms, which bounds the rounding error
of any summation order (a running-error scale), so the tests can state elementwise
tolerances that no index, sign or layout mistake can meet.

`tests/test_local_oracle.py` checks every function here against the assembled oracle
on small meshes before the GPU tests use it at full size.
"""
from __future__ import annotations

import itertools

import numpy as np

from oracle.fem import Mesh, multi_index, unpack_mandel
from oracle.mg import prolongation_1d


class LocalLevel:
    """One level of the hierarchy, evaluated cell by cell (no global assembly)."""

    def __init__(self, d, n, coeff, gamma, kind="scalar", mu_eff=None, W="Mp"):
        self.m = m = Mesh(d, n)
        self.d = d
        self.n = np.array(m.n)
        self.nn = np.array(m.nn)
        self.nb = 3 ** d
        self.coeff = np.asarray(coeff, float)
        self.kind = kind
        self.gamma = float(gamma)
        self.W = W
        self.mu = self.coeff if kind == "scalar" else np.asarray(mu_eff, float)
        self.cstride = np.cumprod((1,) + tuple(m.n[:-1]))
        self.free_node = ~m.boundary_node
        self.free_dof = np.tile(self.free_node, d)
        self.mi = multi_index(d)                       # local node / star offset multi-indices
        self._G_const = m.AL_elem(gamma) if W == "Mp" else None
        self._patch_cache = {}

    # --- bookkeeping --------------------------------------------------------
    def cell_id(self, c):
        return int((np.asarray(c) * self.cstride).sum())

    def node_id(self, g):
        return int(self.m.node_index(np.asarray(g)))

    def node_multi(self, node):
        return self.m.nodes[node]

    def cells_of_node(self, g):
        """(cell id, local node index) of every cell whose closure holds node g."""
        per_dim = []
        for k in range(self.d):
            per_dim.append([c for c in (g[k] // 2 - 1, g[k] // 2)
                            if 0 <= c < self.n[k] and 2 * c <= g[k] <= 2 * c + 2])
        out = []
        for c in itertools.product(*per_dim):
            loc = sum(int(g[k] - 2 * c[k]) * 3 ** k for k in range(self.d))
            out.append((self.cell_id(c), loc))
        return out

    # --- element matrices ---------------------------------------------------
    def G_elem(self, cells):
        """gamma B_K^T W_K^-1 B_K on the given cells (W = M_p or M_p(1/mu))."""
        cells = np.asarray(cells)
        if self.W == "Mp":
            return np.broadcast_to(self._G_const, (len(cells),) + self._G_const.shape)
        Bk = self.m.B_elem
        Winv = np.linalg.inv(self.m.Mmu_elem(self.mu[cells]))
        return self.gamma * np.einsum("aj,cab,bk->cjk", Bk, Winv, Bk)

    def Agamma_elem(self, cells):
        cells = np.asarray(cells)
        if self.kind == "tensor":
            # the oracle's tensor element matrix (C eps(phi_j)) : eps(phi_i), contracted
            # pairwise (optimize=True) instead of in one nested loop: same terms, faster
            m = self.m
            C = unpack_mandel(self.coeff[cells], self.d)
            A = np.einsum("q,qim,cqmn,qjn->cij", m.wdet, m.mandel_basis, C, m.mandel_basis, optimize=True)
        else:
            A = self.m.A_elem(self.coeff[cells], self.kind)
        return A + self.G_elem(cells)

    # --- a1/a2: rows of A_gamma x -------------------------------------------
    def apply_rows(self, x, dofs):
        """(A_gamma x)_i and sum_j |A_ij x_j| for the given dofs (Dirichlet form:
        identity rows at boundary dofs, zero boundary columns elsewhere)."""
        N, nb = self.m.N, self.nb
        xf = np.where(self.free_dof, x, 0.0)
        val, scale = np.zeros(len(dofs)), np.zeros(len(dofs))
        for s, i in enumerate(dofs):
            a, node = divmod(int(i), N)
            if not self.free_node[node]:
                val[s], scale[s] = x[i], abs(x[i])
                continue
            cl = self.cells_of_node(self.node_multi(node))
            cells = [c for c, _ in cl]
            Ke = self.Agamma_elem(cells)
            rows = np.array([a * nb + loc for _, loc in cl])
            terms = Ke[np.arange(len(cl)), rows, :] * xf[self.m.cell_dofs[cells]]
            val[s], scale[s] = terms.sum(), np.abs(terms).sum()
        return val, scale

    # --- a3: vertex-star patch matrices -------------------------------------
    def patch(self, v):
        """(P, keep, gdofs) for vertex v (multi-index in 0..n):
        P    : (d 3^d)^2 patch matrix, dofs component-major, star offsets (-1,0,1)^d
               x-fastest; rows/columns of absent or boundary nodes are zero;
        keep : positions of the free dofs (the star space V_v), in that order;
        gdofs: global dof of every kept position."""
        key = tuple(int(t) for t in v)
        if key in self._patch_cache:
            return self._patch_cache[key]
        d, nb = self.d, self.nb
        v = np.asarray(key)
        P = np.zeros((d * nb, d * nb))
        around = [v - 1 + np.array(s) for s in itertools.product((0, 1), repeat=d)]
        around = [c for c in around if np.all(c >= 0) and np.all(c < self.n)]
        Kes = self.Agamma_elem([self.cell_id(c) for c in around])
        for c, Ke in zip(around, Kes):
            g = 2 * c + self.mi                        # nodes of the cell
            o = g - 2 * v + 1                          # offsets from the vertex, shifted to 0..2
            inside = np.all((o >= 0) & (o <= 2), axis=1)
            loc = np.flatnonzero(inside)
            pos = (o[inside] * (3 ** np.arange(d))).sum(1)
            ld = np.concatenate([a * nb + loc for a in range(d)])
            pd = np.concatenate([a * nb + pos for a in range(d)])
            P[np.ix_(pd, pd)] += Ke[np.ix_(ld, ld)]
        g_all = 2 * v + self.mi - 1
        free = np.all(g_all > 0, axis=1) & np.all(g_all < self.nn - 1, axis=1)
        keep = np.array([a * nb + p for a in range(d) for p in range(nb) if free[p]], dtype=np.int64)
        gdofs = np.array([(k // nb) * self.m.N + self.node_id(g_all[k % nb]) for k in keep], dtype=np.int64)
        P[np.ix_(~np.isin(np.arange(d * nb), keep), np.arange(d * nb))] = 0.0
        P[np.ix_(np.arange(d * nb), ~np.isin(np.arange(d * nb), keep))] = 0.0
        out = (P, keep, gdofs)
        self._patch_cache[key] = out
        return out

    def patch_inverse(self, v):
        """(inv of A_v on the kept dofs, keep, gdofs, cond_2(A_v))."""
        key = ("inv",) + tuple(int(t) for t in v)
        if key not in self._patch_cache:
            P, keep, gdofs = self.patch(v)
            Av = P[np.ix_(keep, keep)]
            self._patch_cache[key] = (np.linalg.inv(Av), keep, gdofs, np.linalg.cond(Av))
        return self._patch_cache[key]

    # --- a4: the star smoother z = sum_v I_v A_v^-1 I_v^T r -------------------
    def vertices_of_node(self, g):
        """Vertices whose star holds node g: |g_k - 2 v_k| <= 1 in every direction."""
        per_dim = [[g[k] // 2] if g[k] % 2 == 0 else [(g[k] - 1) // 2, (g[k] + 1) // 2]
                   for k in range(self.d)]
        return [np.array(v) for v in itertools.product(*per_dim)]

    def smooth_rows(self, r, dofs):
        """z_i, sum_j |A_v^-1|_ij |r_j| summed over the stars, and
        sum_v cond(A_v) ||A_v^-1||_F ||r_v|| (the scale of the inverse's own error)."""
        N, nb = self.m.N, self.nb
        val, absum, cscale = np.zeros(len(dofs)), np.zeros(len(dofs)), np.zeros(len(dofs))
        for s, i in enumerate(dofs):
            a, node = divmod(int(i), N)
            if not self.free_node[node]:
                continue
            g = self.node_multi(node)
            for v in self.vertices_of_node(g):
                inv, keep, gdofs, cond = self.patch_inverse(v)
                o = g - 2 * v + 1
                p = a * nb + int((o * (3 ** np.arange(self.d))).sum())
                row = int(np.flatnonzero(keep == p)[0])
                rv = r[gdofs]
                val[s] += inv[row] @ rv
                absum[s] += np.abs(inv[row]) @ np.abs(rv)
                cscale[s] += cond * np.linalg.norm(inv) * np.linalg.norm(rv)
        return val, absum, cscale


class LocalTransfer:
    """P_H, P~ and P~^T between a coarse and a fine LocalLevel (Sec. 4.2, Eq. Ptilde)."""

    def __init__(self, coarse: LocalLevel, fine: LocalLevel):
        self.c, self.f = coarse, fine
        self.d = fine.d
        self.w1 = [prolongation_1d(int(coarse.n[k])) for k in range(self.d)]   # (4nc+1, 2nc+1)
        self.m5 = np.array(list(itertools.product(range(5), repeat=self.d)))[:, ::-1]  # x fastest

    def fine_nodes_of_cell(self, K):
        """Fine nodes of coarse cell K (multi-indices 4K + 0..4), x-fastest."""
        return 4 * np.asarray(K) + self.m5

    def ph_weight(self, gf, gc):
        """P_H entry between fine node gf and coarse node gc (0 at Dirichlet nodes)."""
        if not self.f.free_node[self.f.node_id(gf)] or not self.c.free_node[self.c.node_id(gc)]:
            return 0.0
        return float(np.prod([self.w1[k][gf[k], gc[k]] for k in range(self.d)]))

    def ph_on_cell(self, K, ec, absval=False):
        """(P_H e_c) on the fine nodes of coarse cell K: array (d, 5^d)."""
        K = np.asarray(K)
        gcs = 2 * K + self.c.mi
        out = np.zeros((self.d, len(self.m5)))
        for j, gf in enumerate(self.fine_nodes_of_cell(K)):
            for gc in gcs:
                w = self.ph_weight(gf, gc)
                if w == 0.0:
                    continue
                nc = self.c.node_id(gc)
                for a in range(self.d):
                    e = ec[a * self.c.m.N + nc]
                    out[a, j] += abs(w * e) if absval else w * e
        return out

    def _fine_cells_of(self, K):
        return [2 * np.asarray(K) + np.array(s) for s in itertools.product((0, 1), repeat=self.d)]

    def _g_apply_on_cell(self, K, vals, absval=False):
        """t = G (vals on the fine nodes of K), G = gamma B^T W^-1 B summed over the 2^d
        fine cells of K, both as (d, 5^d) arrays on K's fine nodes (boundary columns zero)."""
        f, d = self.f, self.d
        fn = self.fine_nodes_of_cell(K)
        index = {tuple(int(t) for t in g): j for j, g in enumerate(fn)}
        out = np.zeros((d, len(fn)))
        for c in self._fine_cells_of(K):
            Ge = f.G_elem([f.cell_id(c)])[0]
            if absval:
                Ge = np.abs(Ge)
            g = 2 * c + f.mi
            js = [index[tuple(int(t) for t in gg)] for gg in g]
            free = np.array([f.free_node[f.node_id(gg)] for gg in g])
            x = np.concatenate([np.where(free, vals[a, js], 0.0) for a in range(d)])
            y = Ge @ x
            for a in range(d):
                out[a, js] += np.where(free, y[a * f.nb:(a + 1) * f.nb], 0.0)
        return out

    def prolong_rows(self, ec, dofs):
        """(P~ e_c)_i, the running-error scale, and the inverse-error scale."""
        f, d = self.f, self.d
        val, absum, cscale = np.zeros(len(dofs)), np.zeros(len(dofs)), np.zeros(len(dofs))
        for s, i in enumerate(dofs):
            a, node = divmod(int(i), f.m.N)
            g = f.node_multi(node)
            if not f.free_node[node]:
                continue
            K = np.minimum(g // 4, self.c.n - 1)
            ef = self.ph_on_cell(K, ec)
            ef_abs = self.ph_on_cell(K, ec, absval=True)
            j = int(np.flatnonzero(np.all(self.fine_nodes_of_cell(K) == g, axis=1))[0])
            val[s], absum[s] = ef[a, j], ef_abs[a, j]
            if np.all(g % 4 != 0):                        # node of int(K): subtract the local solve
                w = self._g_apply_on_cell(K, ef)
                w_abs = self._g_apply_on_cell(K, ef_abs, absval=True)
                inv, keep, gdofs, cond = f.patch_inverse(2 * K + 1)
                wv = self._on_keep(K, w, keep)
                wv_abs = self._on_keep(K, w_abs, keep)
                o = g - 2 * (2 * K + 1) + 1
                row = int(np.flatnonzero(keep == a * f.nb + int((o * (3 ** np.arange(d))).sum()))[0])
                val[s] -= inv[row] @ wv
                absum[s] += np.abs(inv[row]) @ wv_abs
                cscale[s] += cond * np.linalg.norm(inv) * np.linalg.norm(wv)
        return val, absum, cscale

    def _on_keep(self, K, vals, keep):
        """Entries of a (d, 5^d) array on K's fine nodes at the star dofs of vertex 2K+1."""
        f = self.f
        v = 2 * np.asarray(K) + 1
        fn = self.fine_nodes_of_cell(K)
        out = np.zeros(len(keep))
        for t, k in enumerate(keep):
            a, p = divmod(int(k), f.nb)
            g = 2 * v + f.mi[p] - 1
            out[t] = vals[a, int(np.flatnonzero(np.all(fn == g, axis=1))[0])]
        return out

    def _from_keep(self, K, y, keep):
        f = self.f
        v = 2 * np.asarray(K) + 1
        fn = self.fine_nodes_of_cell(K)
        out = np.zeros((self.d, len(fn)))
        for t, k in enumerate(keep):
            a, p = divmod(int(k), f.nb)
            g = 2 * v + f.mi[p] - 1
            out[a, int(np.flatnonzero(np.all(fn == g, axis=1))[0])] = y[t]
        return out

    def restrict_rows(self, rf, dofs):
        """(P~^T r_f)_j = (P_H^T (r_f - G sum_K E_K A_K^-1 E_K^T r_f))_j for coarse dofs j,
        the running-error scale and the inverse-error scale."""
        c, f, d = self.c, self.f, self.d
        val, absum, cscale = np.zeros(len(dofs)), np.zeros(len(dofs)), np.zeros(len(dofs))
        for s, j in enumerate(dofs):
            a, cnode = divmod(int(j), c.m.N)
            if not c.free_node[cnode]:
                continue
            gc = c.node_multi(cnode)
            corr, corr_abs = {}, {}
            cells = [np.array(cc) for cc in itertools.product(
                *[[q for q in (gc[k] // 2 - 1, gc[k] // 2) if 0 <= q < c.n[k] and 2 * q <= gc[k] <= 2 * q + 2]
                  for k in range(d)])]
            for K in cells:
                inv, keep, gdofs, cond = f.patch_inverse(2 * K + 1)
                rv = rf[gdofs]
                y = inv @ rv
                y_abs = np.abs(inv) @ np.abs(rv)
                t = self._g_apply_on_cell(K, self._from_keep(K, y, keep))
                t_abs = self._g_apply_on_cell(K, self._from_keep(K, y_abs, keep), absval=True)
                cscale[s] += cond * np.linalg.norm(inv) * np.linalg.norm(rv)
                for jn, g in enumerate(self.fine_nodes_of_cell(K)):
                    key = tuple(int(q) for q in g)
                    corr[key] = corr.get(key, 0.0) + t[a, jn]
                    corr_abs[key] = corr_abs.get(key, 0.0) + t_abs[a, jn]
            for key in corr:
                w = self.ph_weight(np.array(key), gc)
                if w == 0.0:
                    continue
                rfi = rf[a * f.m.N + f.node_id(key)]
                val[s] += w * (rfi - corr[key])
                absum[s] += abs(w) * (abs(rfi) + corr_abs[key])
        return val, absum, cscale


def load_vector(mesh: Mesh, f_qp):
    """F_(alpha,i) = sum_K sum_q w_q |J| f_alpha(x_q) phi_i(x_q)."""
    F = np.zeros(mesh.nu)
    loc = np.einsum("q,cqa,qi->cai", mesh.wdet, f_qp, mesh.ref.phi)
    np.add.at(F, mesh.cell_dofs, loc.reshape(mesh.ncells, -1))
    return F


def stokes_residual(lv: LocalLevel, f_qp, u, p, chunk=2048):
    """Relative residual ||b - K [u; p]|| / ||b|| of the augmented system (Eq.
    augstokessys) with zero Dirichlet data and zero divergence data, evaluated cell
    by cell: K = [[A_gamma, B^T], [B, 0]] with identity rows at boundary dofs."""
    m, d = lv.m, lv.d
    uf = np.where(lv.free_dof, u, 0.0)
    Be = m.B_elem
    yu = np.zeros(m.nu)
    yp = np.zeros(m.npres)
    P = np.asarray(p).reshape(m.ncells, d + 1)
    for s in range(0, m.ncells, chunk):
        cells = np.arange(s, min(m.ncells, s + chunk))
        Ke = lv.Agamma_elem(cells)
        uK = uf[m.cell_dofs[cells]]
        loc = np.einsum("cij,cj->ci", Ke, uK) + P[cells] @ Be
        np.add.at(yu, m.cell_dofs[cells], loc)
        yp[(d + 1) * s:(d + 1) * cells[-1] + d + 1] = (uK @ Be.T).reshape(-1)
    yu = np.where(lv.free_dof, yu, u)
    b1 = np.where(lv.free_dof, load_vector(m, f_qp), 0.0)
    res = np.concatenate([b1 - yu, -yp])
    return float(np.linalg.norm(res) / np.linalg.norm(b1))
