"""A probabilistic rounding model of the oracle's cycle: how far two FP64 evaluations of
the SAME multigrid cycle on the SAME matrices may drift apart through the order and
grouping of their sums.

Model (the probabilistic rounding-error analysis of Higham and Mary, SIAM J. Sci. Comput.
41 (2019): a sum of n products, evaluated in any order, is within about sqrt(n) u
sum |terms| of the exact value; u = 2^-53): every sum the cycle forms is perturbed by
sqrt(n) u sum|terms| xi, xi uniform in [-1, 1] per computed entry, for
  * each level-operator apply y = A x, with sum|terms| majorised by |A|_e |x|, where |A|_e
    assembles the cells' ABSOLUTE point contributions (|eps(phi_i)| : 2|mu| |eps(phi_j)| at
    each Gauss point plus gamma |B_K|^T |M_K^-1| |B_K|): the terms a matrix-free, point by
    point evaluation adds up; n = the number of cells x points x dofs behind a row;
  * each patch product y_v = A_v^-1 r_v (n = patch size);
  * each Gram-Schmidt inner product and norm of the GMRES relaxation (n = vector length);
the GMRES relaxation is the oracle's (oracle.mg.smooth_gmres) restated here with those
perturbations.  The largest relative change of the cycle's output over a few draws
measures the cycle's sensitivity to rounding: at moderate contrast ~1e-11, at the extreme
contrasts the method exists for (DR 1e8, gamma 1e4, cond(A_v) ~ 1e12) ~1e-7, far above the
1e-12 bar, for any FP64 implementation."""
import numpy as np
import scipy.sparse as sp

import oracle.mg as mg
from oracle.fem import assemble

U64 = 2.0 ** -53


def abs_majorant(lv):
    """|A|_e of a scalar-viscosity level, Dirichlet rows and columns as in lv.A."""
    m = lv.mesh
    e = np.abs(m.strain_basis)
    ee = np.einsum("qikl,qjkl->qij", e, e)
    Ae = np.einsum("q,cq,qij->cij", 2.0 * m.wdet, np.abs(lv.coeff), ee)
    B = np.abs(m.B_elem)
    Ge = lv.gamma * B.T @ np.abs(np.linalg.inv(m.M_elem)) @ B
    Aabs = assemble(m, Ae + Ge[None], m.cell_dofs, m.cell_dofs, (m.nu, m.nu))
    f = sp.diags(lv.free.astype(float))
    return (f @ Aabs @ f + sp.diags((~lv.free).astype(float))).tocsr()


class _Perturbed:
    def __init__(self, A, Aabs, nterms, rng):
        self.A, self.Aabs, self.k, self.rng, self.shape = A, Aabs, np.sqrt(nterms) * U64, rng, A.shape

    def __matmul__(self, x):
        y = self.A @ x
        return y + self.k * (self.Aabs @ np.abs(x)) * self.rng.uniform(-1.0, 1.0, y.shape)


def _noisy_patch_apply(ps, rng):
    def apply(r):
        z = np.zeros_like(r)
        for _, idx, _, inv in ps.groups.values():
            y = np.einsum("pij,pj->pi", inv, r[idx])
            k = np.sqrt(idx.shape[1]) * U64
            y += k * np.einsum("pij,pj->pi", np.abs(inv), np.abs(r[idx])) * rng.uniform(-1.0, 1.0, y.shape)
            np.add.at(z, idx, y)
        return z
    return apply


def _noisy_gmres(rng):
    """oracle.mg.smooth_gmres with perturbed inner products and norms."""
    def smooth_gmres(A, Dinv, x, b, steps):
        r0 = b - A @ x
        k = np.sqrt(r0.size) * U64
        beta = np.linalg.norm(r0) * (1.0 + k * rng.uniform(-1.0, 1.0))
        if beta == 0.0:
            return x
        V, Z = [r0 / beta], []
        H = np.zeros((steps + 1, steps))
        for j in range(steps):
            z = Dinv(V[j])
            w = A @ z
            Vm = np.stack(V, 1)
            h = Vm.T @ w + k * (np.abs(Vm).T @ np.abs(w)) * rng.uniform(-1.0, 1.0, j + 1)
            w = w - Vm @ h
            H[: j + 1, j] = h
            H[j + 1, j] = np.linalg.norm(w) * (1.0 + k * rng.uniform(-1.0, 1.0))
            Z.append(z)
            V.append(w / H[j + 1, j] if H[j + 1, j] > 0 else np.zeros_like(w))
        e1 = np.zeros(steps + 1)
        e1[0] = beta
        y = np.linalg.lstsq(H, e1, rcond=None)[0]
        return x + np.stack(Z, 1) @ y
    return smooth_gmres


def cycle_rounding_spread(H, b, draws=3, seed=100):
    """max over `draws` of |cycle_perturbed(b) - cycle(b)| / |cycle(b)| for the oracle
    hierarchy H (scalar viscosity); H is left unchanged."""
    ref = H.vcycle(b)
    saved_A = [lv.A for lv in H.levels]
    maj = [None] + [abs_majorant(lv) for lv in H.levels[1:]]
    worst = 0.0
    orig_gmres = mg.smooth_gmres
    for t in range(draws):
        rng = np.random.default_rng(seed + t)
        for lvl in range(1, H.L):
            nterms = (2 ** H.d) * (3 ** H.d) * (H.d * 3 ** H.d)
            H.levels[lvl].A = _Perturbed(saved_A[lvl], maj[lvl], nterms, rng)
            H.patches[lvl].apply = _noisy_patch_apply(H.patches[lvl], rng)
        mg.smooth_gmres = _noisy_gmres(rng)
        try:
            out = H.vcycle(b)
        finally:
            mg.smooth_gmres = orig_gmres
            for lvl in range(1, H.L):
                del H.patches[lvl].apply       # back to the class method
            for lv, A in zip(H.levels, saved_A):
                lv.A = A
        worst = max(worst, float(np.linalg.norm(out - ref) / np.linalg.norm(ref)))
    return worst
