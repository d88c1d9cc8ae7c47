"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every check here compares the oracle with something other than itself:
printed counts, closed-form integrals, invariants, brute force on tiny
meshes, or the textbook a-priori rates.  CPU only.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle.fem import (GAUSS_PTS, GAUSS_WTS, Level, Mesh, RefElement, lagrange_q2,
                        mandel_pairs)
from oracle.mg import (Hierarchy, PatchSet, prolongation_1d, smooth_gmres,
                       standard_prolongation, star_patches)
from oracle.stokes import StokesSolver, direct_solve, schur_blocks
from synthetic import problems as P

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append([float(v) for v in line.split()])
    return np.array(rows)


# --------------------------------------------------------------------------
# quadrature, bases, bookkeeping
# --------------------------------------------------------------------------
def test_gauss_rule_exact_to_degree_five():
    for k in range(6):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs((GAUSS_WTS * GAUSS_PTS ** k).sum() - exact) < 1e-14
    assert abs((GAUSS_WTS * GAUSS_PTS ** 6).sum() - 2.0 / 7) > 1e-3


def test_sample_points_are_the_quadrature_points():
    for d, n in [(2, (3, 2)), (3, (2, 1, 3))]:
        m = Mesh(d, n)
        xq_ref = m.ref.xq
        x = (m.cells[:, None, :] + 0.5 * (1 + xq_ref[None])) * np.array(m.h)
        assert np.allclose(P.sample_points(d, n), x, atol=1e-15)


def test_dof_counts_printed_in_paper():
    for d, n, nv, npr, nvert in _golden("dof_counts.txt").astype(int):
        m = Mesh(d, n)
        assert m.nu == nv and m.npres == npr
        assert (n + 1) ** d == nvert


def test_q2_basis_nodal_and_partition_of_unity():
    L = lagrange_q2(np.array([-1.0, 0.0, 1.0]))
    assert np.allclose(L, np.eye(3))
    ref = RefElement(3)
    assert np.allclose(ref.phi.sum(1), 1.0)
    assert np.allclose(ref.dphi.sum(1), 0.0)


# --------------------------------------------------------------------------
# element matrices: closed forms and invariants
# --------------------------------------------------------------------------
def _field_dofs(mesh, fn):
    x = mesh.node_coords()
    u = fn(x)                                   # (N, d)
    return u.T.reshape(-1)


@pytest.mark.parametrize("d", [2, 3])
def test_rigid_motions_in_kernel_and_symmetry(d):
    m = Mesh(d, 2)
    lv = Level(d, 2, np.random.default_rng(0).uniform(0.5, 2, (m.ncells, 3 ** d)), 7.0)
    A = lv.Agam_raw
    assert abs(A - A.T).max() < 1e-12 * abs(A).max()
    modes = [lambda x, k=k: np.eye(d)[k][None].repeat(x.shape[0], 0) for k in range(d)]
    for i in range(d):
        for j in range(i + 1, d):
            def rot(x, i=i, j=j):
                u = np.zeros_like(x)
                u[:, i], u[:, j] = -x[:, j], x[:, i]
                return u
            modes.append(rot)
    for fn in modes:
        u = _field_dofs(m, fn)
        assert np.abs(A @ u).max() < 1e-12 * abs(A).max()


def test_B_on_divergence_free_and_unit_divergence_fields():
    m = Mesh(2, 2)
    lv = Level(2, 2, np.ones((4, 9)), 1.0)
    u = _field_dofs(m, lambda x: np.stack([x[:, 0] ** 2, -2 * x[:, 0] * x[:, 1]], 1))
    assert np.abs(lv.B_raw @ u).max() < 1e-14
    u = _field_dofs(m, lambda x: np.stack([x[:, 0], 0 * x[:, 0]], 1))
    Bu = (lv.B_raw @ u).reshape(-1, 3)          # -(psi, 1)_K = -(|K|, 0, 0)
    assert np.allclose(Bu, [[-0.25, 0, 0]] * 4, atol=1e-15)


def test_pressure_mass_closed_form():
    for d in (2, 3):
        m = Mesh(d, 4)
        vol = 4.0 ** -d
        assert np.allclose(m.M_elem, vol * np.diag([1.0] + [1.0 / 3] * d), atol=1e-16)


@pytest.mark.parametrize("d", [2, 3])
def test_viscous_energy_closed_forms(d):
    """u^T A u = int 2 mu |eps(u)|^2 and u^T G u = gamma int (Pi div u)^2, exact integrals."""
    m = Mesh(d, 2)
    xq = P.sample_points(d, 2)
    mu = 1.0 + xq[..., 0]                       # linear viscosity: 3-point Gauss is exact here
    lv = Level(d, 2, mu, 3.0)
    # u = (x^2, 0, ..): eps = diag(2x, 0..), 2 mu eps:eps = 8 x^2 (1 + x) -> 8 (1/3 + 1/4)
    u = _field_dofs(m, lambda x: np.stack([x[:, 0] ** 2] + [0 * x[:, 0]] * (d - 1), 1))
    assert abs(u @ lv.A_raw @ u - 8 * (1 / 3 + 1 / 4)) < 1e-12
    # linear field u = M x: div = tr M, |eps|^2 = |sym M|^2; mu = 1 + x has mean 3/2
    M = np.arange(1.0, d * d + 1).reshape(d, d) * np.array([1, -1] * d)[: d]
    u = _field_dofs(m, lambda x: x @ M.T)
    S = 0.5 * (M + M.T)
    assert abs(u @ lv.A_raw @ u - 2 * 1.5 * (S * S).sum()) < 1e-11
    assert abs(u @ lv.G_raw @ u - 3.0 * np.trace(M) ** 2) < 1e-11
    # (Pi div u) for u = (x^2, ..) is the P1 projection of 2x on each cell = 2x exactly
    u = _field_dofs(m, lambda x: np.stack([x[:, 0] ** 2] + [0 * x[:, 0]] * (d - 1), 1))
    assert abs(u @ lv.G_raw @ u - 3.0 * 4.0 / 3.0) < 1e-12


@pytest.mark.parametrize("d", [2, 3])
def test_tensor_path_reduces_to_scalar(d):
    m = Mesh(d, 2)
    mu = np.random.default_rng(1).uniform(0.1, 10, (m.ncells, 3 ** d))
    nm = len(mandel_pairs(d))
    iu = np.triu_indices(nm)
    C = np.zeros((m.ncells, 3 ** d, len(iu[0])))
    diag = np.flatnonzero(iu[0] == iu[1])
    C[:, :, diag] = 2 * mu[:, :, None]
    assert np.allclose(m.A_elem(C, "tensor"), m.A_elem(mu, "scalar"), atol=1e-12)


@pytest.mark.parametrize("d", [2, 3])
def test_tensor_energy_closed_form(d):
    """Anisotropic C (Eq. stokes-lin): for a linear field u = M x the strain is the constant
    S = sym M, so u^T A u = int_(0,1)^d (C S) : S = s^T K s with s the Mandel vector of S
    (diagonal entries, then sqrt2 times the off-diagonal ones in the documented order) and K
    the full Mandel matrix whose upper triangle, row-major, is stored per point.  Fails for
    a wrong packing order, a missing sqrt2 or an unsymmetrised upper triangle."""
    m = Mesh(d, 2)
    pairs = [(0, 0), (1, 1), (0, 1)] if d == 2 else [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
    nm = len(pairs)
    rng = np.random.default_rng(5)
    R = rng.standard_normal((nm, nm))
    K = R @ R.T + nm * np.eye(nm)                    # SPD, all entries distinct
    iu = np.triu_indices(nm)
    C = np.broadcast_to(K[iu], (m.ncells, 3 ** d, len(iu[0]))).copy()
    lv = Level(d, 2, C, 0.0, kind="tensor", mu_eff=np.ones((m.ncells, 3 ** d)))
    M = rng.standard_normal((d, d))
    S = 0.5 * (M + M.T)
    s = np.array([S[k, l] * (1.0 if k == l else math.sqrt(2.0)) for k, l in pairs])
    u = _field_dofs(m, lambda x: x @ M.T)
    assert abs(u @ lv.A_raw @ u - s @ K @ s) < 1e-11 * abs(s @ K @ s)


@pytest.mark.parametrize("d,n", [(2, 4), (3, 2)])
def test_Agamma_spd_and_AL_nullity(d, n):
    lv = Level(d, n, np.ones((n ** d, 3 ** d)), 10.0)
    A = lv.A.toarray()
    assert np.linalg.eigvalsh(A).min() > 0
    f = lv.free
    G = lv.G.toarray()[np.ix_(f, f)]
    ev = np.linalg.eigvalsh(G)
    nullity = int((ev < 1e-10 * ev.max()).sum())
    assert nullity == f.sum() - (lv.mesh.npres - 1)
    assert ev.min() > -1e-10 * ev.max()


# --------------------------------------------------------------------------
# Sec. 3: AL invariance, Schur identity, eigenvalue lemma and remarks
# --------------------------------------------------------------------------
def _tiny_sinker(gamma, d=2, n=4, dr=1e4):
    return P.sinker_problem(d, n, 1, 3, 0.3, 50.0, dr, 10.0, gamma, seed=3)


def test_AL_solution_invariance():
    sols = []
    for g in (0.0, 1.0, 1e4):
        pb = _tiny_sinker(g)
        lv = Level(2, pb.n, pb.mu[0], g)
        u, p = direct_solve(lv, pb.f, pb.u_bc)
        sols.append((u, p))
    for u, p in sols[1:]:
        assert np.linalg.norm(u - sols[0][0]) <= 1e-9 * np.linalg.norm(sols[0][0])
        assert np.linalg.norm(p - sols[0][1]) <= 1e-8 * np.linalg.norm(sols[0][1])


def _mean_zero_basis(lv):
    m = lv.mesh.npres
    n = np.zeros(m)
    n[:: lv.mesh.d + 1] = 1.0
    return sla.null_space(n[None, :])               # orthonormal basis of the complement


def _schur_pieces(lv):
    f = lv.free
    A = lv.A_raw.toarray()[np.ix_(f, f)]
    B = lv.B.toarray()[:, f]
    Z = _mean_zero_basis(lv)
    W = sp.block_diag([lv.mesh.M_elem] * lv.mesh.ncells).toarray()
    Shat = sp.block_diag(list(lv.Mp_mu_blocks)).toarray()
    return A, B, Z, W, Shat


def test_schur_identity_smw():
    """S_gamma^-1 = S^-1 + gamma W^-1 on the mean-zero subspace (Eq. (AL-Schur))."""
    gamma = 37.0
    lv = Level(2, 4, _tiny_sinker(gamma).mu[0], gamma)
    A, B, Z, W, _ = _schur_pieces(lv)
    Winv = np.linalg.inv(W)
    Ag = A + gamma * B.T @ Winv @ B
    S = Z.T @ B @ np.linalg.solve(A, B.T) @ Z
    Sg = Z.T @ B @ np.linalg.solve(Ag, B.T) @ Z
    # on the subspace the identity holds for the compressed W: (Z^T W^-1 Z)
    lhs = np.linalg.inv(Sg)
    rhs = np.linalg.inv(S) + gamma * Z.T @ Winv @ Z
    assert np.allclose(lhs, rhs, rtol=1e-8, atol=1e-8 * abs(rhs).max())


def _gen_eig(X, Y):
    return sla.eigh(X, Y, eigvals_only=True)


@pytest.mark.parametrize("gamma", [0.0, 1.0, 100.0, 1e4])
def test_eigenvalue_lemma_bounds(gamma):
    """sigma(S_hat_gamma^-1 S_gamma) in [f_mu, F_mu] (Lemma, Eqs. (f_mu), (F_mu))."""
    lv = Level(2, 4, _tiny_sinker(gamma, dr=1e3).mu[0], gamma)
    A, B, Z, W, Shat = _schur_pieces(lv)
    # compressed operators on the mean-zero subspace (S is singular on constants)
    S = Z.T @ B @ np.linalg.solve(A, B.T) @ Z
    Wz = np.linalg.inv(Z.T @ np.linalg.inv(W) @ Z)
    Sz = np.linalg.inv(Z.T @ np.linalg.inv(Shat) @ Z)
    c, C = _gen_eig(S, Sz)[[0, -1]]
    dd, D = _gen_eig(S, Wz)[[0, -1]]
    e, E = _gen_eig(Sz, Wz)[[0, -1]]
    f_mu = max(c / (1 + gamma * c * E) + gamma * dd / (1 + gamma * dd),
               (1 + gamma * e) / (max(1, 1 / c) + gamma * e))
    F_mu = min(C / (1 + gamma * C * e) + gamma * D / (1 + gamma * D),
               (1 + gamma * e) / (min(1, 1 / C) + gamma * e))
    Sg = np.linalg.inv(np.linalg.inv(S) + gamma * np.linalg.inv(Wz))
    Shat_g = np.linalg.inv(np.linalg.inv(Sz) + gamma * np.linalg.inv(Wz))
    lam = _gen_eig(Sg, Shat_g)
    assert lam.min() >= f_mu * (1 - 1e-8) and lam.max() <= F_mu * (1 + 1e-8)


def test_remark_shat_equals_w():
    """S_hat = W: lambda = (1 + gamma) / (nu^-1 + gamma), eigenvalue by eigenvalue."""
    gamma = 25.0
    lv = Level(2, 4, _tiny_sinker(gamma).mu[0], gamma)
    A, B, Z, W, _ = _schur_pieces(lv)
    S = Z.T @ B @ np.linalg.solve(A, B.T) @ Z
    Wz = np.linalg.inv(Z.T @ np.linalg.inv(W) @ Z)
    nu = _gen_eig(S, Wz)
    Sg = np.linalg.inv(np.linalg.inv(S) + gamma * np.linalg.inv(Wz))
    Wg = np.linalg.inv((1 + gamma) * np.linalg.inv(Wz))
    lam = _gen_eig(Sg, Wg)
    assert np.allclose(np.sort(lam), np.sort((1 + gamma) / (1 / nu + gamma)), rtol=1e-8)


def test_exact_A_preconditioned_spectrum_and_counts():
    """With the exact (1,1) inverse the preconditioned operator has eigenvalues 1 and
    sigma(S_hat_gamma^-1 S_gamma) (Remark after the lemma); FGMRES then needs few steps."""
    counts = []
    for gamma in (1.0, 1e2, 1e4):
        pb = _tiny_sinker(gamma, n=8, dr=1e4)
        H = Hierarchy(2, pb.n, [pb.mu[0]], gamma, smoother="richardson", steps=1)
        s = StokesSolver(H, "P1", exact_A=True)
        u, p, its, _ = s.solve(pb.f, pb.u_bc, rtol=1e-10)
        counts.append(its)
    assert counts[0] >= counts[1] >= counts[2]
    assert counts[2] <= 6


def _table_exacttopleft():
    out = {}
    path = os.path.join(os.path.dirname(__file__), "golden", "table_exacttopleft.txt")
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        out[f[0], float(f[1])] = [int(v) for v in f[2:]]
    return out


def test_exact_A_counts_as_in_table_exacttopleft():
    """Table exacttopleft at small scale (2D 16^2 sinker problem, exact (1,1) solve, 1e6
    residual reduction, DR 1e4/1e6/1e8): P1 and P2 coincide at gamma = 0 (both reduce to
    M_p(1/mu)^-1 with no augmentation), counts fall with gamma for both and rise with DR at
    gamma = 0, P1 needs no more than P2 at gamma = 10, and at gamma = 1e3 the counts are
    within one of the printed ones (2/3/4 for P1 and 2/4/5 for P2; measured here 2/3/4 and
    3/3/4).  The printed gamma = 0 row is 32/48/59 against 32/49/71 here, gamma = 10 7/9/10
    (P1) and 10/16/20 (P2) against 9/12/16 and 10/16/22: the sinker positions are random."""
    table = _table_exacttopleft()
    drs = (1e4, 1e6, 1e8)
    its = {}
    for j, dr in enumerate(drs):
        for g in (0.0, 10.0, 1e3):
            pb = P.sinker_problem(2, 16, 1, 8, 0.1, 200.0, dr, 10.0, g, 0)
            for var, W in (("P1", "Mp"), ("P2", "Mp_mu")):
                H = Hierarchy(2, pb.n, [pb.mu[0]], g, smoother="richardson", steps=1, W=W)
                its[var, g, dr] = StokesSolver(H, var, exact_A=True).solve(pb.f, pb.u_bc, rtol=1e-6)[2]
    for dr in drs:
        assert its["P1", 0.0, dr] == its["P2", 0.0, dr]
        for var in ("P1", "P2"):
            assert its[var, 0.0, dr] > its[var, 10.0, dr] >= its[var, 1e3, dr], (var, dr, its)
        assert its["P1", 10.0, dr] <= its["P2", 10.0, dr]
    assert its["P1", 0.0, 1e4] < its["P1", 0.0, 1e6] < its["P1", 0.0, 1e8]
    for var in ("P1", "P2"):
        for j, dr in enumerate(drs):
            assert abs(its[var, 1e3, dr] - table[var, 1000.0][j]) <= 1, (var, dr, its[var, 1e3, dr])


def test_stored_table_vanka_counts_against_the_printed_column():
    """The oracle's counts on the AL column of Table vanka (Sec. 5.2.3: 2D 128^2, 4 levels,
    P2 with gamma 100, F-cycle, 1e6 reduction), stored by tests/golden/make_table_vanka.py:
    with one sinker they are within one of the printed 4/6/8/9 at DR 1e4..1e10 (5/7/8/9);
    with 6 and 24 seeded sinkers (the paper's are random) they stay at or below the printed
    counts; every count is non-decreasing in DR and bounded (the robustness the column
    shows, where the Vanka column fails at DR 1e10)."""
    rows = []
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "table_vanka_oracle.txt")):
        if not line.startswith("#") and line.strip():
            s, dr, ours, paper = line.split()
            rows.append((int(s), float(dr), int(ours), int(paper)))
    assert len(rows) == 12
    for s, dr, ours, paper in rows:
        if s == 1:
            assert abs(ours - paper) <= 1, (s, dr, ours, paper)
        assert ours <= paper + 1 and ours <= 30, (s, dr, ours, paper)
    for s in (1, 6, 24):
        seq = [ours for ss, _, ours, _ in sorted(rows) if ss == s]
        assert all(b >= a for a, b in zip(seq, seq[1:])), (s, seq)


# --------------------------------------------------------------------------
# discretisation: manufactured solution rates and discrete divergence
# --------------------------------------------------------------------------
def _errors(lv, u, p):
    m = lv.mesh
    g, w = np.polynomial.legendre.leggauss(5)
    X = np.stack(np.meshgrid(g, g, indexing="ij"), -1).reshape(-1, 2)[:, ::-1]
    W = np.outer(w, w).reshape(-1) * m.detJ
    Lx = lagrange_q2(X[:, 0]); Ly = lagrange_q2(X[:, 1])
    from oracle.fem import lagrange_q2_deriv
    dLx = lagrange_q2_deriv(X[:, 0]); dLy = lagrange_q2_deriv(X[:, 1])
    phi = np.einsum("qa,qb->qba", Lx, Ly).reshape(len(X), 9)
    gx = np.einsum("qa,qb->qba", dLx, Ly).reshape(len(X), 9) * (2 / m.h[0])
    gy = np.einsum("qa,qb->qba", Lx, dLy).reshape(len(X), 9) * (2 / m.h[1])
    xphys = (m.cells[:, None, :] + 0.5 * (1 + X[None])) * np.array(m.h)
    U = u.reshape(2, -1)[:, m.cell_nodes]       # (2, ncells, 9)
    uh = np.einsum("qa,ica->ciq", phi, U)
    guh = np.stack([np.einsum("qa,ica->ciq", gx, U), np.einsum("qa,ica->ciq", gy, U)], -1)
    ue = P.manufactured_u(xphys).transpose(0, 2, 1)
    ge = P.manufactured_grad_u(xphys).transpose(0, 2, 1, 3)
    ph = np.einsum("cb,qb->cq", p.reshape(-1, 3), np.concatenate([np.ones((len(X), 1)), X], 1))
    eL2 = math.sqrt((W * ((uh - ue) ** 2).sum(1)).sum())
    eH1 = math.sqrt((W * ((guh - ge) ** 2).sum((1, 3))).sum())
    pL2 = math.sqrt((W * ph ** 2).sum())
    return eL2, eH1, pL2


def test_manufactured_convergence_rates():
    errs = []
    for n in (4, 8, 16):
        pb = P.manufactured_problem(n, 1, 1.0)
        lv = Level(2, pb.n, pb.mu[0], 1.0)
        u, p = direct_solve(lv, pb.f, pb.u_bc)
        errs.append(_errors(lv, u, p))
    errs = np.array(errs)
    rates = np.log2(errs[:-1] / errs[1:])
    assert np.all(rates[:, 0] > 2.8), rates      # L2 velocity O(h^3)
    assert np.all(rates[:, 1] > 1.8), rates      # H1 velocity O(h^2)
    assert np.all(rates[:, 2] > 1.7), rates      # L2 pressure O(h^2)


def test_discrete_divergence_at_roundoff():
    pb = _tiny_sinker(1e2, n=8)
    lv = Level(2, pb.n, pb.mu[0], 1e2)
    u, p = direct_solve(lv, pb.f, pb.u_bc)
    Bu = lv.B_raw @ u
    scale = abs(lv.B_raw).max() * np.abs(u).max()
    assert np.abs(Bu).max() < 1e-11 * scale


# --------------------------------------------------------------------------
# Sec. 4: transfers, smoother, V-cycle
# --------------------------------------------------------------------------
def test_prolongation_1d_closed_form():
    assert np.allclose(prolongation_1d(1), _golden("prolongation_1d.txt"), atol=0)


@pytest.mark.parametrize("d", [2, 3])
def test_standard_prolongation_reproduces_coarse_fields(d):
    """P_H is the identity on V_H (Lemma P, proof of (d))."""
    cm, fm = Mesh(d, 2), Mesh(d, 4)
    PH = standard_prolongation(cm, fm)
    rng = np.random.default_rng(2)
    uc = rng.standard_normal(cm.nu)
    uc[cm.boundary_dof] = 0
    xf = fm.node_coords()
    # evaluate the coarse Q2 field at fine nodes by direct Lagrange evaluation
    cell = np.minimum((xf * np.array(cm.n)).astype(int), np.array(cm.n) - 1)
    xi = 2 * (xf * np.array(cm.n) - cell) - 1
    vals = np.zeros((d, fm.N))
    Uc = uc.reshape(d, -1)
    for a in cm.ref.mi:
        w = np.prod([lagrange_q2(xi[:, k])[:, a[k]] for k in range(d)], axis=0)
        node = cm.node_index(2 * cell + a)
        vals += w * Uc[:, node]
    vals[:, fm.boundary_node] = 0
    assert np.allclose(PH @ uc, vals.reshape(-1), atol=1e-13)


def test_robust_prolongation_local_problem():
    """u~ = P_H u_H - P~ u_H lives in V^_h and solves a(u~, v) = gamma (Pi div P_H u_H, Pi div v)."""
    pb = _tiny_sinker(1e3, n=8)
    H = Hierarchy(2, 8, P.sinker_problem(2, 8, 2, 3, 0.3, 50.0, 1e4, seed=3).mu, 1e3,
                  smoother="richardson", steps=1)
    fine = H.levels[1]
    uc = np.random.default_rng(4).standard_normal(H.levels[0].mesh.nu)
    uc[H.levels[0].bdof] = 0
    ut = H.PH[1] @ uc - H.P[1] @ uc
    interior = np.concatenate(H.interiors[1].index_sets)
    outside = np.setdiff1d(np.arange(fine.mesh.nu), interior)
    assert np.abs(ut[outside]).max() <= 1e-14 * np.abs(H.PH[1] @ uc).max()
    lhs = (fine.A @ ut)[interior]
    rhs = (fine.G @ (H.PH[1] @ uc))[interior]
    assert np.allclose(lhs, rhs, rtol=1e-10, atol=1e-10 * np.abs(rhs).max())


def _energy_ratio(Pm, Af, Ac, free_c):
    X = (Pm.T @ Af @ Pm).toarray()[np.ix_(free_c, free_c)]
    Y = Ac.toarray()[np.ix_(free_c, free_c)]
    return sla.eigh(X, Y, eigvals_only=True)[-1]


def test_robust_prolongation_energy_continuity():
    """||P~ u_H||_(A_h,gamma) <~ ||u_H||_(A_H,gamma) uniformly in gamma (Eq. (conP));
    the standard P_H degrades like gamma."""
    rob, std = [], []
    for g in (1.0, 1e2, 1e4, 1e6):
        mus = [np.ones((4 ** 2, 9)), np.ones((8 ** 2, 9))]
        H = Hierarchy(2, 8, mus, g, smoother="richardson", steps=1)
        fc = H.levels[0].free
        rob.append(_energy_ratio(H.P[1], H.levels[1].A, H.levels[0].A, fc))
        std.append(_energy_ratio(H.PH[1], H.levels[1].A, H.levels[0].A, fc))
    assert max(rob) < 3.0 * min(rob)
    assert std[-1] > 1e3 * std[0]


@pytest.mark.parametrize("d,n", [(2, 4), (3, 2)])
def test_star_smoother_spectrum(d, n):
    """lambda_max(D^-1 A) <= 2^d (each dof lies in at most 2^d stars, a colouring bound)
    and lambda_min independent of gamma (kernel decomposition, Eq. (kdp))."""
    lmins = []
    for g in (0.0, 1.0, 1e3, 1e6):
        lv = Level(d, n, np.ones((n ** d, 3 ** d)), g)
        ps = star_patches(lv)
        f = lv.free
        A = lv.A.toarray()[np.ix_(f, f)]
        Dinv = np.stack([ps.apply(e) for e in np.eye(lv.mesh.nu)[f]], 1)[f]
        ev = np.sort(np.linalg.eigvals(Dinv @ A).real)
        assert ev[-1] <= 2 ** d * (1 + 1e-8)
        lmins.append(ev[0])
    # bounded below uniformly in gamma: no decay like 1/gamma between 1e3 and 1e6
    assert min(lmins) > 0.05 and lmins[2] < 1.2 * lmins[3]


def test_gmres_smoother_is_minimal_residual():
    lv = Level(2, 4, _tiny_sinker(1e2).mu[0], 1e2)
    ps = star_patches(lv)
    rng = np.random.default_rng(5)
    b = rng.standard_normal(lv.mesh.nu); b[lv.bdof] = 0
    x0 = rng.standard_normal(lv.mesh.nu); x0[lv.bdof] = 0
    A = lv.A
    x = smooth_gmres(A, ps.apply, x0, b, 3)
    # brute force: minimise ||b - A(x0 + Z c)|| over the explicit Krylov space
    r0 = b - A @ x0
    K = [ps.apply(r0)]
    for _ in range(2):
        K.append(ps.apply(A @ K[-1]))
    Z = np.stack(K, 1)
    c = np.linalg.lstsq(A @ Z, r0, rcond=None)[0]
    assert abs(np.linalg.norm(b - A @ x) - np.linalg.norm(r0 - A @ Z @ c)) < 1e-10 * np.linalg.norm(r0)


def _vcycle_matrix(H, lvl):
    """Dense linear operator of the Richardson V-cycle from its error propagation
    I - M_l A_l = S^s (I - P M_(l-1) P^T A_l) S^s, S = I - tau D^-1 A_l."""
    A = H.levels[lvl].A.toarray()
    f = H.levels[lvl].free
    n = A.shape[0]
    if lvl == 0:
        M = np.zeros_like(A)
        M[np.ix_(f, f)] = np.linalg.inv(A[np.ix_(f, f)])
        return M
    Dinv = np.stack([H.patches[lvl].apply(e) for e in np.eye(n)], 1)
    S = np.eye(n) - H.tau * Dinv @ A
    Pm = H.P[lvl].toarray()
    Mc = _vcycle_matrix(H, lvl - 1)
    Ss = np.linalg.matrix_power(S, H.steps)
    E = Ss @ (np.eye(n) - Pm @ Mc @ Pm.T @ A) @ Ss
    Ainv = np.zeros_like(A)
    Ainv[np.ix_(f, f)] = np.linalg.inv(A[np.ix_(f, f)])
    return (np.eye(n) - E) @ Ainv


def test_vcycle_equals_explicit_operator_product():
    mus = P.sinker_problem(2, 8, 3, 3, 0.3, 50.0, 1e4, seed=1).mu
    H = Hierarchy(2, 8, mus, 1e2, smoother="richardson", steps=2)
    M = _vcycle_matrix(H, 2)
    rng = np.random.default_rng(6)
    for _ in range(3):
        b = rng.standard_normal(H.levels[2].mesh.nu); b[H.levels[2].bdof] = 0
        assert np.allclose(H.vcycle(b), M @ b, rtol=1e-9, atol=1e-9 * np.abs(M @ b).max())


def _fcycle_matrix(H, lvl):
    """Dense operator of the Richardson F-cycle from the textbook error propagation:
    I - F_l A_l = S^s (I - P C P^T A_l) S^s, where the coarse correction C satisfies
    I - C A_c = (I - V_(l-1) A_c)(I - F_(l-1) A_c)  (F-cycle, then a V-cycle from its
    result), and C = A_c^-1 when level l-1 is the coarsest."""
    A = H.levels[lvl].A.toarray()
    f = H.levels[lvl].free
    n = A.shape[0]
    Ainv = np.zeros_like(A)
    Ainv[np.ix_(f, f)] = np.linalg.inv(A[np.ix_(f, f)])
    if lvl == 0:
        return Ainv
    Ac = H.levels[lvl - 1].A.toarray()
    fc = H.levels[lvl - 1].free
    Acinv = np.zeros_like(Ac)
    Acinv[np.ix_(fc, fc)] = np.linalg.inv(Ac[np.ix_(fc, fc)])
    if lvl - 1 == 0:
        C = Acinv
    else:
        Ic = np.eye(Ac.shape[0])
        Ec = (Ic - _vcycle_matrix(H, lvl - 1) @ Ac) @ (Ic - _fcycle_matrix(H, lvl - 1) @ Ac)
        C = (Ic - Ec) @ Acinv
    Dinv = np.stack([H.patches[lvl].apply(e) for e in np.eye(n)], 1)
    Ss = np.linalg.matrix_power(np.eye(n) - H.tau * Dinv @ A, H.steps)
    Pm = H.P[lvl].toarray()
    E = Ss @ (np.eye(n) - Pm @ C @ Pm.T @ A) @ Ss
    return (np.eye(n) - E) @ Ainv


def test_fcycle_equals_textbook_error_propagation():
    """The recursive F-cycle against its error-propagation formula (3 levels, so the
    coarse correction on level 1 is an F-cycle followed by a V-cycle from its result);
    it also contracts at least as well as the V-cycle."""
    mus = P.sinker_problem(2, 8, 3, 3, 0.3, 50.0, 1e4, seed=1).mu
    H = Hierarchy(2, 8, mus, 1e2, smoother="richardson", steps=2, cycle="F")
    MF = _fcycle_matrix(H, 2)
    MV = _vcycle_matrix(H, 2)
    rng = np.random.default_rng(7)
    for _ in range(3):
        b = rng.standard_normal(H.levels[2].mesh.nu); b[H.levels[2].bdof] = 0
        ref = MF @ b
        assert np.allclose(H.cycle(b), ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())
        assert not np.allclose(H.vcycle(b), ref, rtol=1e-6, atol=1e-6 * np.abs(ref).max())
    f = H.levels[2].free
    A = H.levels[2].A.toarray()
    I = np.eye(A.shape[0])
    rho = lambda M: np.abs(np.linalg.eigvals((I - M @ A)[np.ix_(f, f)])).max()  # noqa: E731
    assert rho(MF) <= rho(MV) + 1e-12


def _two_level_rho(gamma, smoother, transfer):
    mus = [np.ones((16, 9)), np.ones((64, 9))]
    H = Hierarchy(2, 8, mus, gamma, smoother=smoother, steps=2, transfer=transfer,
                  tau=0.25 if smoother == "richardson" else 0.6)
    if smoother == "jacobi":
        H.patches = [None, PatchSet.__new__(PatchSet)]
        dg = H.levels[1].A.diagonal()
        H.patches[1].apply = lambda r: r / dg
    M = _vcycle_matrix(H, 1)
    f = H.levels[1].free
    A = H.levels[1].A.toarray()
    E = (np.eye(A.shape[0]) - M @ A)[np.ix_(f, f)]
    return np.abs(np.linalg.eigvals(E)).max()


def test_vcycle_contraction_gamma_robust_and_standard_mg_fails():
    rob = [_two_level_rho(g, "richardson", "robust") for g in (1.0, 1e2, 1e4)]
    std = [_two_level_rho(g, "jacobi", "standard") for g in (1.0, 1e2, 1e4)]
    assert max(rob) < 0.6 and max(rob) - min(rob) < 0.15, rob
    assert std[-1] > 0.99 and std[-1] > std[0], std


# --------------------------------------------------------------------------
# outer solver
# --------------------------------------------------------------------------
@pytest.mark.parametrize("fact,its", [("full", 1), ("upper", 2), ("lower", 2), ("diag", 3)])
def test_factorisation_types_with_exact_blocks(fact, its):
    """With the exact A_gamma^-1 and the exact Schur complement, the full factorisation
    is the inverse (1 FGMRES iteration), the block-triangular ones leave a
    preconditioned operator with the single eigenvalue 1 and minimal polynomial of
    degree 2 (2 iterations), and the block-diagonal one three distinct eigenvalues
    (3 iterations) -- Murphy, Golub & Wathen (2000), Ipsen (2001).  A sign or a
    dropped factor in any variant changes these counts."""
    from oracle.stokes import StokesSolver
    mus = [np.ones((4, 9)), np.ones((16, 9))]
    H = Hierarchy(2, 4, mus, 10.0, smoother="richardson", steps=1)
    sol = StokesSolver(H, "P1", exact_A=True, fact=fact)
    lv = sol.fine
    A = lv.A.toarray()
    S = lv.B.toarray() @ np.linalg.solve(A, lv.Bt.toarray())
    sol.Sinv = np.linalg.pinv(S, rcond=1e-10)
    rng = np.random.default_rng(11)
    rhs = rng.standard_normal(sol.nu + sol.np_)
    rhs[np.flatnonzero(lv.bdof)] = 0.0
    rhs[sol.nu:] = sol.project(rhs[sol.nu:])
    x, k, hist = sol.fgmres(rhs, rtol=1e-10, maxit=10)
    assert k == its, (fact, k, hist)
    assert np.linalg.norm(sol.matvec(x) - rhs) <= 1e-8 * np.linalg.norm(rhs)
    # the minimal polynomial of T = K P on compatible vectors fixes the signs too:
    # full: T = I; triangular: (T - I)^2 = 0 (a flipped S gives (T - I)(T + I) = 0);
    # diagonal with -S^-1: (T - I)(T^2 - T + I) = 0 (eigenvalues 1, (1 +- i sqrt 3)/2)
    T = lambda v: sol.matvec(sol.precondition(v))  # noqa: E731
    v = rhs / np.linalg.norm(rhs)
    if fact == "full":
        r = T(v) - v
    elif fact in ("upper", "lower"):
        w = T(v) - v
        r = T(w) - w
    else:
        w = T(v) - v
        r = T(T(w)) - T(w) + w
    assert np.linalg.norm(r) <= 1e-8, (fact, np.linalg.norm(r))

@pytest.mark.parametrize("schur,W", [("P1", "Mp"), ("P2", "Mp_mu")])
def test_fgmres_matches_direct_solve(schur, W):
    pb = P.sinker_2d(n=16, levels=3, gamma=1e2, dr=1e4, seed=2)
    H = Hierarchy(2, pb.n, pb.mu, pb.gamma, W=W)
    s = StokesSolver(H, schur)
    u, p, its, hist = s.solve(pb.f, pb.u_bc, rtol=1e-11)
    ud, pd = direct_solve(H.levels[-1], pb.f, pb.u_bc)
    pd[::3] -= pd[::3].mean()
    assert np.linalg.norm(u - ud) < 1e-7 * np.linalg.norm(ud)
    assert np.linalg.norm(p - pd) < 1e-6 * np.linalg.norm(pd)
    assert its < 40 and hist[-1] <= 1e-11 * hist[0]


def test_iteration_counts_flat_in_gamma():
    counts = []
    for g in (1.0, 1e2, 1e4):
        pb = P.sinker_2d(n=16, levels=3, gamma=g, dr=1e6, seed=0)
        s = StokesSolver(Hierarchy(2, pb.n, pb.mu, g))
        counts.append(s.solve(pb.f, pb.u_bc, rtol=1e-8)[2])
    assert counts[-1] <= counts[0] and max(counts) <= 40, counts


@pytest.mark.parametrize("d", [2, 3])
def test_weighted_pressure_mass_exact_integrals(d):
    """M_p(1/mu) of Eq. (inv-visc-mass), the P2 Schur block and the W of the P2 pairing,
    for a viscosity varying inside each cell: with 1/mu linear in x the 3-point Gauss rule is
    exact, so every cell block equals the exact integral of (1/mu) psi_a psi_b over the cell,
    psi = {1, xi_0, .., xi_(d-1)} in reference coordinates (computed symbolically here)."""
    sympy = pytest.importorskip("sympy")
    n = 2
    xq = P.sample_points(d, n)
    coef = np.array([1.0, 2.0, 0.5][:d])
    mu = 1.0 / (1.0 + xq @ coef)
    lv = Level(d, n, mu, 1.0, W="Mp_mu")
    X = sympy.symbols("x0:%d" % d)
    h = sympy.Rational(1, n)
    cells = list(np.ndindex(*(n,) * d))
    for cid, c in enumerate(c[::-1] for c in cells):   # cell index x-fastest
        lo = [sympy.Rational(int(ci), n) for ci in c]
        psi = [sympy.Integer(1)] + [2 * (X[k] - lo[k]) / h - 1 for k in range(d)]
        w = 1 + sum(sympy.Rational(coef[k]).limit_denominator(4) * X[k] for k in range(d))
        ref = np.zeros((d + 1, d + 1))
        for a in range(d + 1):
            for b in range(d + 1):
                e = w * psi[a] * psi[b]
                for k in range(d):
                    e = sympy.integrate(e, (X[k], lo[k], lo[k] + h))
                ref[a, b] = float(e)
        assert np.allclose(lv.Mp_mu_blocks[cid], ref, rtol=1e-13, atol=1e-15), cid


def test_schur_blocks_closed_form_constant_mu():
    lv = Level(2, 2, 2.0 * np.ones((4, 9)), 5.0)
    blk = schur_blocks(lv, "P1")[0]
    vol = 0.25
    expect = np.diag([1.0, 3.0, 3.0]) / vol * (2.0 + 5.0)
    assert np.allclose(blk, expect)
    lv2 = Level(2, 2, 2.0 * np.ones((4, 9)), 5.0, W="Mp_mu")
    assert np.allclose(schur_blocks(lv2, "P2")[0], 6.0 * 2.0 * np.diag([1.0, 3.0, 3.0]) / vol)
    # with constant mu, W = M_p(1/mu) = M_p / mu: the AL term scales by mu
    assert abs(lv2.G_raw - 2.0 * lv.G_raw).max() < 1e-12 * abs(lv.G_raw).max()


def _round_patch_inverses(H, fn):
    for ps in H.patches[1:]:
        for key, (ids, idx, blocks, inv) in list(ps.groups.items()):
            ps.groups[key] = (ids, idx, blocks, fn(inv))


def _bf16(x):
    b = x.astype(np.float32).view(np.uint32)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)   # round to nearest even
    return b.view(np.float32).astype(np.float64)


def test_reduced_precision_patch_storage():
    """Storing the star-patch inverses in FP32 changes no FGMRES iteration count; storing them
    in BF16 (8-bit mantissa, the scope's optional variant) holds at gamma 10 but loses the
    convergence at gamma 1e3 (2D 32^2 sinker problem, DR 1e4, three levels, GMRES(5)): the
    inverse of a star block of A_gamma resolves its small divergence-free eigenvalues beside
    entries of order gamma, so a relative storage error eps perturbs the smoother by about
    eps gamma on the kernel the star patches exist to capture (Sec. 4.1)."""
    its = {}
    for gamma in (10.0, 1e3):
        pb = P.sinker_problem(2, 32, 3, 8, 0.1, 200.0, 1e4, 10.0, gamma, 0)
        for store in ("fp64", "fp32", "bf16"):
            H = Hierarchy(2, pb.n, pb.mu, gamma, steps=5)
            if store == "fp32":
                _round_patch_inverses(H, lambda x: x.astype(np.float32).astype(np.float64))
            elif store == "bf16":
                _round_patch_inverses(H, _bf16)
            its[gamma, store] = StokesSolver(H).solve(pb.f, pb.u_bc, rtol=1e-8, maxit=60)[2]
    assert its[10.0, "fp32"] == its[10.0, "fp64"] and its[1e3, "fp32"] == its[1e3, "fp64"], its
    assert its[10.0, "bf16"] <= its[10.0, "fp64"] + 2, its
    assert its[1e3, "fp64"] < 20 and its[1e3, "bf16"] == 60, its           # 60 = not converged
