"""Factor injection for the GPU parity tests: the oracle's own patch and coarse inverses,
in the library's layouts, and an oracle hierarchy that applies exactly those matrices.

The oracle factors each patch and the coarsest operator with LAPACK Cholesky; its
explicit inverses are symmetric only up to rounding.  Both sides must apply the SAME
matrices, so the upper triangles are mirrored (what the packed layout keeps), the oracle's
robust prolongation P~ is rebuilt from the mirrored interior inverses with the oracle's
formula (Eq. (Ptilde): P~ = P_H - sum_K E_K A_K^-1 E_K^T G P_H), and its coarse solve is
the product with the mirrored explicit inverse.  What is left between the two cycles is
the order of the floating-point sums."""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from oracle.mg import all_vertices


def mirror_upper(X):
    return np.triu(X) + np.swapaxes(np.triu(X, 1), -1, -2)


def packed_by_diagonals(full, np_):
    stride = ((np_ * (np_ + 1) // 2) + 3) & ~3
    out = np.zeros((len(full), stride))
    for v, F in enumerate(full):
        pos = 0
        for t in range(np_):
            out[v, pos:pos + np_ - t] = np.diagonal(F, offset=t)
            pos += np_ - t
    return out


def unpack_by_diagonals(pv, np_):
    F = np.zeros((np_, np_))
    pos = 0
    for t in range(np_):
        k = np_ - t
        F[np.arange(k), np.arange(t, np_)] = pv[pos:pos + k]
        F[np.arange(t, np_), np.arange(k)] = pv[pos:pos + k]
        pos += k
    return F


def library_patch_inverses(H, lvl):
    """The oracle's star-patch inverses of level lvl in the library's layout: per vertex
    (x-fastest) the full d 3^d matrix, component-major, star offsets x-fastest, identity
    at absent and boundary nodes."""
    m = H.levels[lvl].mesh
    d, NB = m.d, 3 ** m.d
    verts = all_vertices(m)
    offs = np.array([[o % 3, (o // 3) % 3, o // 9][:d] for o in range(NB)]) - 1
    full = np.tile(np.eye(d * NB), (len(verts), 1, 1))
    for ids, _, _, inv in H.patches[lvl].groups.values():
        for i, X in zip(ids, inv):
            g = 2 * verts[i] + offs
            free = np.all(g > 0, axis=1) & np.all(g < np.array(m.nn) - 1, axis=1)
            keep = [a * NB + o for a in range(d) for o in range(NB) if free[o]]
            full[i][np.ix_(keep, keep)] = mirror_upper(X)
    return full


def inject(H):
    """Mirror every inverse of the oracle hierarchy H in place (patches, coarse-cell
    interiors, coarse operator), rebuild P~ from them, and return the coarse inverse."""
    for lvl in range(1, H.L):
        for ps in (H.patches[lvl], H.interiors[lvl]):
            if ps is None:
                continue
            for ids, idx, blocks, inv in ps.groups.values():
                inv[:] = mirror_upper(inv)
        ps = H.interiors[lvl]
        if ps is not None:
            fine = H.levels[lvl]
            rows, cols, vals = [], [], []
            for ids, idx, _, inv in ps.groups.values():
                for j in range(idx.shape[0]):
                    rows.append(np.repeat(idx[j], idx.shape[1]))
                    cols.append(np.tile(idx[j], idx.shape[1]))
                    vals.append(inv[j].ravel())
            Ablk = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                                 shape=fine.A.shape).tocsr()
            H.P[lvl] = (H.PH[lvl] - Ablk @ (fine.G @ H.PH[lvl])).tocsr()
    free = H.coarse_free
    inv0 = mirror_upper(sla.cho_solve(H.coarse_chol, np.eye(len(free))))

    def coarse_solve(b):
        x = np.zeros_like(b)
        x[free] = inv0 @ b[free]
        return x

    H.coarse_solve = coarse_solve
    return inv0


def load_into(ctx, H, inv0):
    """Load the (mirrored) oracle inverses of every level into a library context."""
    for lvl in range(1, H.L):
        m = H.levels[lvl].mesh
        np_ = m.d * 3 ** m.d
        ctx.load_patch_inverses(lvl, packed_by_diagonals(library_patch_inverses(H, lvl), np_))
    ctx.load_coarse_inverse(np.ascontiguousarray(inv0))
