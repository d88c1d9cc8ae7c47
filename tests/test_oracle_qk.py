"""Pins of the order-k oracle (oracle/qk.py), [Q_k]^d x P_(k-1)^disc, against what the
mathematics fixes: k = 2 reproduces the k = 2 oracle matrix for matrix; Gauss exactness;
nodal bases; rigid motions; discrete divergence of divergence-free fields; the inf-sup
rank of B; the a-priori rates O(h^(k+1)) / O(h^k) / O(h^k) of a manufactured solution;
the star dimensions; P_H reproducing coarse fields; and the gamma-robust two-level
contraction of the star smoother with the robust transfer against point Jacobi with the
standard one (the k = 3 form of Table k's claim).  CPU only."""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle.fem import Level
from oracle.qk import (LevelK, MeshK, all_vertices_k, lagrange_1d, lagrange_1d_deriv, lagrange_nodes,
                       pressure_exponents, prolongation_1d_k, standard_prolongation_k, star_nodes_k,
                       two_level_error)
from synthetic import problems as P


@pytest.mark.parametrize("d,n,W", [(2, 2, "Mp"), (2, (3, 2), "Mp"), (3, 2, "Mp"), (2, 2, "Mp_mu"), (3, 2, "Mp_mu")])
def test_k2_equals_the_q2_oracle(d, n, W):
    """At k = 2 the order-k definitions are the k = 2 oracle's, entry for entry (both
    augmentation weights)."""
    rng = np.random.default_rng(1)
    nc = int(np.prod((n,) * d if np.isscalar(n) else n))
    mu = np.exp(rng.standard_normal((nc, 3 ** d)))
    a = LevelK(d, n, 2, mu, 7.0, W)
    b = Level(d, n, mu, 7.0, W=W)
    for x, y in ((a.A, b.A), (a.B, b.B), (a.G, b.G)):
        assert abs(x - y).max() <= 1e-12 * abs(y).max()


@pytest.mark.parametrize("d,n,smoother,cycle", [(2, 8, "gmres", "F"), (2, 8, "richardson", "V"),
                                                (2, 8, "richardson", "F"), (3, 4, "richardson", "F")])
def test_k2_cycles_equal_the_q2_oracle(d, n, smoother, cycle):
    """At k = 2 the order-k hierarchy's cycles (V and F, GMRES and Richardson smoothing) are
    the k = 2 oracle's (itself pinned by its error-propagation formula), and the F-cycle and
    the V-cycle really differ."""
    from oracle.mg import Hierarchy
    from oracle.qk import HierarchyK
    rng = np.random.default_rng(2)
    L = 3 if d == 2 else 2
    sizes = [n // 2 ** (L - 1 - l) for l in range(L)]
    mus = [np.exp(rng.standard_normal((m ** d, 3 ** d))) for m in sizes]
    a = HierarchyK(d, n, 2, mus, 5.0, steps=2, smoother=smoother, cycle=cycle)
    b = Hierarchy(d, n, mus, 5.0, steps=2, smoother=smoother, cycle=cycle)
    r = rng.standard_normal(a.levels[-1].mesh.nu)
    r[~a.levels[-1].free] = 0.0
    x, y = a.cycle(r), b.cycle(r)
    assert np.linalg.norm(x - y) <= 1e-12 * np.linalg.norm(y)
    if cycle == "F" and L > 2:
        assert np.linalg.norm(a.vcycle(r) - x) > 1e-6 * np.linalg.norm(x)


@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_gauss_exact_and_lagrange_nodal(k):
    g, w = np.polynomial.legendre.leggauss(k + 1)
    for p in range(2 * k + 2):               # exact through degree 2k + 1
        exact = (1 - (-1) ** (p + 1)) / (p + 1)
        assert abs((w * g ** p).sum() - exact) < 1e-13
    t = lagrange_nodes(k)
    assert np.allclose(lagrange_1d(k, t), np.eye(k + 1), atol=1e-14)
    xs = np.linspace(-1, 1, 17)
    assert np.allclose(lagrange_1d(k, xs).sum(1), 1.0, atol=1e-13)
    assert np.allclose(lagrange_1d_deriv(k, xs).sum(1), 0.0, atol=1e-11)
    # the derivative table against a centred difference of the value table
    h = 1e-6
    fd = (lagrange_1d(k, xs + h) - lagrange_1d(k, xs - h)) / (2 * h)
    assert np.allclose(lagrange_1d_deriv(k, xs), fd, atol=1e-6)


@pytest.mark.parametrize("d,k", [(2, 3), (3, 3), (2, 4)])
def test_pressure_space_dimension(d, k):
    assert len(pressure_exponents(d, k)) == math.comb(k - 1 + d, d)


@pytest.mark.parametrize("d,k", [(2, 3), (3, 3), (2, 4)])
def test_rigid_motions_and_symmetry(d, k):
    m = MeshK(d, 1, k)
    K = m.A_elem(np.ones((1, m.ref.nq)))[0]
    assert np.allclose(K, K.T, atol=1e-12 * abs(K).max())
    x = m.node_coords()[m.cell_nodes[0]]
    motions = [np.concatenate([np.ones(m.ref.nb) if c == a else np.zeros(m.ref.nb) for c in range(d)])
               for a in range(d)]
    for i in range(d):
        for j in range(i + 1, d):        # rotation in the (i, j) plane: u_i = -x_j, u_j = x_i
            v = [np.zeros(m.ref.nb) for _ in range(d)]
            v[i], v[j] = -x[:, j], x[:, i]
            motions.append(np.concatenate(v))
    for r in motions:
        assert np.abs(K @ r).max() < 1e-11 * abs(K).max()


def test_B_on_divergence_free_and_unit_divergence_fields():
    """u = (2 x^2 y, -2 x y^2) lies in Q_3 and is divergence free: B u = 0 exactly.
    u = (x, 0) has div u = 1: B u = -(psi_p, 1)_K cell by cell."""
    lv = LevelK(2, 3, 3, np.ones((9, 16)), 1.0)
    m = lv.mesh
    x = m.node_coords()
    u = np.concatenate([2 * x[:, 0] ** 2 * x[:, 1], -2 * x[:, 0] * x[:, 1] ** 2])
    Bu = lv.B_raw @ u
    assert np.abs(Bu).max() < 1e-13
    u1 = np.concatenate([x[:, 0], np.zeros(m.N)])
    Bu1 = (lv.B_raw @ u1).reshape(m.ncells, m.ref.npr)
    ref = -np.array([m.detJ * np.prod([(1 - (-1) ** (a + 1)) / (a + 1) for a in al]) for al in m.ref.alpha])
    assert np.allclose(Bu1, ref[None, :], atol=1e-14)


def test_inf_sup_rank_of_B():
    """Q_3 x P_2^disc: B on the free velocities has rank npres - 1 (constants only)."""
    lv = LevelK(2, 2, 3, np.ones((4, 16)), 1.0)
    Bf = lv.B.toarray()[:, lv.free]
    assert np.linalg.matrix_rank(Bf, tol=1e-10 * abs(Bf).max()) == lv.mesh.npres - 1


def _solve_manufactured(n, k):
    lv = LevelK(2, n, k, np.ones((n * n, (k + 1) ** 2)), 0.0)
    m = lv.mesh
    xq = lv.gauss_points()
    F = lv.load_vector(P.manufactured_f(xq))
    uD = np.zeros(m.nu)
    ue = P.manufactured_u(m.node_coords())
    bd = m.boundary_dof
    uD[bd] = ue.T.reshape(-1)[bd]
    rhs_u = F - (lv.A_raw + lv.G_raw) @ uD
    rhs_u[bd] = 0.0
    rhs_p = -(lv.B_raw @ uD)
    nvec = np.zeros(m.npres)
    nvec[:: m.ref.npr] = 1.0                       # the constant pressure mode
    K = sp.bmat([[lv.A, lv.B.T, None], [lv.B, None, sp.csr_matrix(nvec[:, None])],
                 [None, sp.csr_matrix(nvec[None, :]), None]], format="csc")
    x = spla.spsolve(K, np.concatenate([rhs_u, rhs_p, [0.0]]))
    return lv, x[: m.nu] + uD, x[m.nu: -1]


def _errors(lv, u, p):
    m = lv.mesh
    k = m.k
    g, w = np.polynomial.legendre.leggauss(k + 3)
    X = np.stack(np.meshgrid(g, g, indexing="ij"), -1).reshape(-1, 2)[:, ::-1]
    W = np.outer(w, w).reshape(-1) * m.detJ
    Lx, Ly = lagrange_1d(k, X[:, 0]), lagrange_1d(k, X[:, 1])
    dLx, dLy = lagrange_1d_deriv(k, X[:, 0]), lagrange_1d_deriv(k, X[:, 1])
    nb = (k + 1) ** 2
    phi = np.einsum("qa,qb->qba", Lx, Ly).reshape(len(X), nb)
    gx = np.einsum("qa,qb->qba", dLx, Ly).reshape(len(X), nb) * (2 / m.h[0])
    gy = np.einsum("qa,qb->qba", Lx, dLy).reshape(len(X), nb) * (2 / m.h[1])
    xphys = (m.cells[:, None, :] + 0.5 * (1 + X[None])) * np.array(m.h)
    U = u.reshape(2, -1)[:, m.cell_nodes]
    uh = np.einsum("qa,ica->ciq", phi, U)
    guh = np.stack([np.einsum("qa,ica->ciq", gx, U), np.einsum("qa,ica->ciq", gy, U)], -1)
    ue = P.manufactured_u(xphys).transpose(0, 2, 1)
    ge = P.manufactured_grad_u(xphys).transpose(0, 2, 1, 3)
    psi = np.stack([np.prod(X ** np.array(a)[None, :], axis=1) for a in m.ref.alpha], -1)
    ph = np.einsum("cb,qb->cq", p.reshape(m.ncells, -1), psi)
    ph = ph - (W * ph).sum() / (W.sum() * m.ncells)
    eL2 = math.sqrt((W * ((uh - ue) ** 2).sum(1)).sum())
    eH1 = math.sqrt((W * ((guh - ge) ** 2).sum((1, 3))).sum())
    pL2 = math.sqrt((W * ph ** 2).sum())
    return eL2, eH1, pL2


def test_manufactured_rates_q3():
    """k = 3: velocity O(h^4) in L2 and O(h^3) in H1, pressure O(h^3) (p = 0 exactly)."""
    errs = np.array([_errors(*_solve_manufactured(n, 3)) for n in (2, 4, 8)])
    rates = np.log2(errs[:-1] / errs[1:])
    assert np.all(rates[:, 0] > 3.6), rates
    assert np.all(rates[:, 1] > 2.7), rates
    assert np.all(rates[:, 2] > 2.5), rates


@pytest.mark.parametrize("d,k", [(2, 3), (3, 3), (2, 4)])
def test_star_dimensions(d, k):
    m = MeshK(d, 4, k)
    sizes = {tuple(v): len(star_nodes_k(m, v)) for v in map(tuple, all_vertices_k(m))}
    assert sizes[(2,) * d] == (2 * k - 1) ** d
    assert sizes[(0,) * d] == (k - 1) ** d
    covered = set()
    for v in all_vertices_k(m):
        covered.update(star_nodes_k(m, v).tolist())
    assert covered == set(np.flatnonzero(~m.boundary_node).tolist())


def test_standard_prolongation_reproduces_coarse_fields():
    """P_H is the identity on V_H: a coarse Q_3 field evaluated at the fine nodes."""
    cm, fm = MeshK(2, 2, 3), MeshK(2, 4, 3)
    PH = standard_prolongation_k(cm, fm)
    rng = np.random.default_rng(3)
    uc = rng.standard_normal(cm.nu)
    uc[cm.boundary_dof] = 0.0
    xf = fm.node_coords()
    cell = np.minimum((xf * np.array(cm.n)).astype(int), np.array(cm.n) - 1)
    xi = 2.0 * (xf * np.array(cm.n) - cell) - 1.0
    ref = np.zeros(fm.nu)
    for i in range(fm.N):
        lx, ly = lagrange_1d(3, [xi[i, 0]])[0], lagrange_1d(3, [xi[i, 1]])[0]
        for a in range(4):
            for b in range(4):
                node = (3 * cell[i, 0] + a) + cm.nn[0] * (3 * cell[i, 1] + b)
                for c in range(2):
                    ref[c * fm.N + i] += lx[a] * ly[b] * uc[c * cm.N + node]
    ref[fm.boundary_dof] = 0.0
    assert np.allclose(PH @ uc, ref, atol=1e-13)
    assert np.allclose(prolongation_1d_k(1, 3).sum(1), 1.0)


def _rho(gamma, smoother, transfer):
    fine = LevelK(2, 4, 3, np.ones((16, 16)), gamma)
    coarse = LevelK(2, 2, 3, np.ones((4, 16)), gamma)
    E = two_level_error(fine, coarse, smoother, transfer, steps=2, tau=0.25 if smoother == "star" else 0.6)
    return np.abs(np.linalg.eigvals(E)).max()


def test_two_level_q3_gamma_robust_and_standard_fails():
    rob = [_rho(g, "star", "robust") for g in (1.0, 1e2, 1e4)]
    std = [_rho(g, "jacobi", "standard") for g in (1.0, 1e2, 1e4)]
    assert max(rob) < 0.6 and max(rob) - min(rob) < 0.15, rob
    assert std[-1] > 0.99 and std[-1] > std[0], std


def _sinker_qk(n, k, gamma, dr=1e4, seed=0, count=4, W="Mp"):
    from oracle.qk import HierarchyK
    c = P.sinker_centres(seed, count, 2)

    def pts(nl):
        m = MeshK(2, nl, k)
        return (m.cells[:, None, :] + 0.5 * (1.0 + m.ref.xq[None])) * np.array(m.h)

    mus = [P.sinker_viscosity(pts(nl), c, 0.1, 200.0, dr) for nl in (n // 2, n)]
    H = HierarchyK(2, n, k, mus, gamma, steps=5, W=W)
    f = P.sinker_force(pts(n), c, 0.1, 200.0, 10.0)
    return H, f, np.zeros((2, (k * n + 1) ** 2))


def test_q3_fgmres_matches_direct_solve():
    """FGMRES with the two-level gamma-robust cycle at k = 3 reaches the sparse direct
    solution of the same augmented system."""
    from oracle.stokes import StokesSolver, direct_solve
    H, f, ubc = _sinker_qk(8, 3, 1e2)
    u, p, its, _ = StokesSolver(H).solve(f, ubc, rtol=1e-10)
    ud, pd = direct_solve(H.levels[-1], f, ubc)
    npr = H.levels[-1].mesh.ref.npr
    pd = pd.copy()
    pd[::npr] -= pd[::npr].mean()
    assert np.linalg.norm(u - ud) <= 1e-7 * np.linalg.norm(ud)
    assert np.linalg.norm(p - pd) <= 1e-6 * np.linalg.norm(pd)


def test_q3_iteration_trends_of_table_k():
    """Table k's two trends at small scale (two levels, 2D, DR 1e4): at fixed gamma the
    k = 3 solver needs no more iterations than k = 2, and larger gamma needs fewer."""
    from oracle.stokes import StokesSolver
    its = {}
    for k in (2, 3):
        for g in (0.0, 10.0, 1e3):
            H, f, ubc = _sinker_qk(8, k, g)
            its[k, g] = StokesSolver(H).solve(f, ubc, rtol=1e-8)[2]
    for g in (0.0, 10.0, 1e3):
        assert its[3, g] <= its[2, g], its
    for k in (2, 3):
        assert its[k, 1e3] <= its[k, 10.0] < its[k, 0.0], its


def test_q3_p2_pairing_as_in_table_k():
    """Table k's configuration: the P2 pairing (W = M_p(1/mu), S^-1 ~ (1 + gamma) M_p(1/mu)^-1),
    two levels, k = 2..5.  At small scale (2D, 8^2 cells, DR 1e6) the iteration counts fall
    with gamma at every k and do not rise with k at gamma 1e3, the paper's 27/13/8/6 trend
    (66/42/31/26 at gamma 10 and 16/13/10/9 at gamma 1e3 here)."""
    from oracle.stokes import StokesSolver
    its = {}
    ks = (2, 3, 4, 5)
    for k in ks:
        for g in (10.0, 1e3):
            H, f, ubc = _sinker_qk(8, k, g, dr=1e6, W="Mp_mu")
            its[k, g] = StokesSolver(H, schur="P2").solve(f, ubc, rtol=1e-8)[2]
    for g in (10.0, 1e3):
        assert its[3, g] <= its[2, g], its
    for lo, hi in zip(ks, ks[1:]):
        assert its[hi, 1e3] <= its[lo, 1e3], its
    for k in ks:
        assert its[k, 1e3] <= its[k, 10.0], its


def test_table_linear_2d_pattern():
    """Table linear's 2D block ([Q3]^2 x P2disc, P1 and P2, DR 1e6 and 1e10, 1e6 residual
    reduction) at small scale (8^2 cells, two levels): at gamma = 0 both Schur blocks reduce
    to M_p(1/mu)^-1, so P1 and P2 need the same count, with the Jacobi smoother and standard
    transfer as with the robust ones, and at DR 1e10 the gamma = 0 solve does not converge
    within 300 iterations (the table's dashes); with gamma > 0 the robust solver converges at
    both contrasts, P1 needs no more iterations than P2 at gamma = 10, and gamma = 1e3 needs
    no more than gamma = 10 (printed 11/22 and 19/27 at gamma 10, 13/15 and 12/16 at 1e3;
    here 17/28, 33/152 and 10/15, 11/24)."""
    from oracle.qk import HierarchyK
    from oracle.stokes import StokesSolver
    c = P.sinker_centres(0, 4, 2)

    def run(g, dr, var, smoother="gmres", transfer="robust"):
        def pts(nl):
            m = MeshK(2, nl, 3)
            return (m.cells[:, None, :] + 0.5 * (1.0 + m.ref.xq[None])) * np.array(m.h)
        mus = [P.sinker_viscosity(pts(nl), c, 0.1, 200.0, dr) for nl in (4, 8)]
        H = HierarchyK(2, 8, 3, mus, g, steps=5, W="Mp" if var == "P1" else "Mp_mu",
                       smoother=smoother, transfer=transfer)
        f = P.sinker_force(pts(8), c, 0.1, 200.0, 10.0)
        return StokesSolver(H, schur=var).solve(f, np.zeros((2, 25 ** 2)), rtol=1e-6)[2]

    assert run(0.0, 1e6, "P1", "jacobi", "standard") == run(0.0, 1e6, "P2", "jacobi", "standard")
    assert run(0.0, 1e6, "P1") == run(0.0, 1e6, "P2") < 300
    assert run(0.0, 1e10, "P1") == 300
    for dr in (1e6, 1e10):
        its = {(g, v): run(g, dr, v) for g in (10.0, 1e3) for v in ("P1", "P2")}
        assert max(its.values()) < 300, (dr, its)
        assert its[10.0, "P1"] <= its[10.0, "P2"], (dr, its)
        for v in ("P1", "P2"):
            assert its[1e3, v] <= its[10.0, v], (dr, its)


def test_table_k_trend_in_3d():
    """Table k is a 3D experiment: at gamma 1e3 with the P2 pairing (DR 1e6, two levels) the
    printed counts fall from 27 at k = 2 to 13 at k = 3.  On a 4^3 mesh (6 seeded sinkers,
    omega 0.15, a 1e6 residual reduction) the oracle's counts fall the same way, 20 to 10."""
    from oracle.qk import HierarchyK
    from oracle.stokes import StokesSolver
    c = P.sinker_centres(0, 6, 3)

    def run(k):
        def pts(nl):
            m = MeshK(3, nl, k)
            return (m.cells[:, None, :] + 0.5 * (1.0 + m.ref.xq[None])) * np.array(m.h)
        mus = [P.sinker_viscosity(pts(nl), c, 0.15, 200.0, 1e6) for nl in (2, 4)]
        H = HierarchyK(3, 4, k, mus, 1e3, steps=5, W="Mp_mu")
        f = P.sinker_force(pts(4), c, 0.15, 200.0, 10.0)
        return StokesSolver(H, schur="P2").solve(f, np.zeros((3, (4 * k + 1) ** 3)), rtol=1e-6)[2]

    its2, its3 = run(2), run(3)
    assert its3 < its2 <= 30, (its2, its3)


@pytest.mark.parametrize("k", [3, 4])
def test_prolongation_1d_exact_rationals(k):
    """The 1D coarse-to-fine weights of Q_k against exact rational Lagrange values."""
    from fractions import Fraction as Fr
    t = [Fr(-1) + Fr(2 * a, k) for a in range(k + 1)]
    nf = 2 * k + 1
    ref = np.zeros((nf, k + 1))
    for f in range(nf):
        x = Fr(f, 2 * k)                       # fine node in the coarse cell (0, 1)
        xi = 2 * x - 1
        for a in range(k + 1):
            v = Fr(1)
            for b in range(k + 1):
                if b != a:
                    v *= (xi - t[b]) / (t[a] - t[b])
            ref[f, a] = float(v)
    assert np.allclose(prolongation_1d_k(1, k), ref, atol=1e-15)
