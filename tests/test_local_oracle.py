"""The cell-local oracle evaluations (tests/local_oracle.py) against the assembled oracle.

The full-size GPU tests sample outputs one by one with the cell-local forms; here each
form is checked, on small meshes, entry for entry against the assembled matrices,
patch sets and transfer operators of `oracle/` (2D and 3D, scalar and tensor
coefficients, W = M_p and W = M_p(1/mu), vertices and nodes on every kind of boundary)."""
import numpy as np
import pytest

from local_oracle import LocalLevel, LocalTransfer, stokes_residual
from oracle.mg import Hierarchy, all_vertices, star_dofs
from oracle.stokes import StokesSolver
from synthetic import problems as P

EPS64 = 2.0 ** -53    # the two sides invert each patch with different rounding: cond(A_v) eps apart


def _sinker(d, n, levels, gamma, dr, seed):
    if d == 2:
        return P.sinker_problem(2, n, levels, 8, 0.1, 200.0, dr, 10.0, gamma, seed)
    return P.sinker_problem(3, n, levels, 16, 0.15, 200.0, dr, 10.0, gamma, seed)


CASES = [
    ("scalar", 2, 4, "Mp"),
    ("scalar", 3, 2, "Mp"),
    ("scalar", 2, 4, "Mp_mu"),
    ("tensor", 2, 4, "Mp"),
    ("tensor", 3, 2, "Mp_mu"),
]


def _problem(kind, d, n, W):
    """Two-level problem (finest mesh n^d cells), its oracle hierarchy and the
    cell-local form of both levels."""
    if kind == "scalar":
        pb = _sinker(d, n, 2, 1e3, 1e4, seed=3)
        H = Hierarchy(d, pb.n, pb.mu, pb.gamma, smoother="richardson", steps=1, W=W)
    else:
        pb = P.viscoplastic_problem(d, n, 2, 1e2, seed=4)
        H = Hierarchy(d, pb.n, pb.mu, pb.gamma, kind="tensor", mu_eff=pb.meta["mu_eff"],
                      smoother="richardson", steps=1, W=W)
    levels = [LocalLevel(d, lv.mesh.n, lv.coeff, pb.gamma, kind=lv.kind,
                         mu_eff=None if kind == "scalar" else lv.mu, W=W) for lv in H.levels]
    return pb, H, levels


@pytest.mark.parametrize("kind,d,n,W", CASES)
def test_apply_rows_equal_assembled_operator(kind, d, n, W):
    _, H, L = _problem(kind, d, n, W)
    for l in range(2):
        lv = H.levels[l]
        x = np.random.default_rng(l + 1).standard_normal(lv.mesh.nu)
        ref = lv.A @ x
        dofs = np.arange(lv.mesh.nu)
        val, scale = L[l].apply_rows(x, dofs)
        assert np.all(np.abs(val - ref) <= 1e-13 * scale + 1e-300), l
        assert np.all(scale >= np.abs(ref) * (1 - 1e-12))


@pytest.mark.parametrize("kind,d,n,W", CASES)
def test_patches_equal_assembled_restrictions(kind, d, n, W):
    _, H, L = _problem(kind, d, n, W)
    lv = H.levels[1]
    A = lv.A.tocsr()
    for v in all_vertices(lv.mesh):
        Pm, keep, gdofs = L[1].patch(v)
        idx = star_dofs(lv.mesh, v)
        assert np.array_equal(gdofs, idx)
        ref = A[idx][:, idx].toarray()
        got = Pm[np.ix_(keep, keep)]
        assert np.allclose(got, ref, rtol=0, atol=1e-13 * np.abs(ref).max())   # same terms, any order
        other = np.setdiff1d(np.arange(Pm.shape[0]), keep)
        assert not Pm[other].any() and not Pm[:, other].any()


@pytest.mark.parametrize("kind,d,n,W", CASES)
def test_smoother_rows_equal_patch_sum(kind, d, n, W):
    _, H, L = _problem(kind, d, n, W)
    lv = H.levels[1]
    r = np.random.default_rng(5).standard_normal(lv.mesh.nu)
    r[lv.bdof] = 0.0
    ref = H.patches[1].apply(r)
    dofs = np.arange(lv.mesh.nu)
    val, absum, cscale = L[1].smooth_rows(r, dofs)
    assert np.all(np.abs(val - ref) <= 1e-12 * absum + 100 * EPS64 * cscale + 1e-300)


@pytest.mark.parametrize("kind,d,n,W", CASES)
def test_transfer_rows_equal_assembled_transfers(kind, d, n, W):
    _, H, L = _problem(kind, d, n, W)
    T = LocalTransfer(L[0], L[1])
    rng = np.random.default_rng(7)
    ec = rng.standard_normal(H.levels[0].mesh.nu)
    ec[H.levels[0].bdof] = 0.0
    rf = rng.standard_normal(H.levels[1].mesh.nu)
    rf[H.levels[1].bdof] = 0.0
    Pt = H.P[1]
    ref_p = Pt @ ec
    val, absum, cscale = T.prolong_rows(ec, np.arange(H.levels[1].mesh.nu))
    assert np.all(np.abs(val - ref_p) <= 1e-12 * absum + 100 * EPS64 * cscale + 1e-300)
    ref_r = Pt.T @ rf
    val, absum, cscale = T.restrict_rows(rf, np.arange(H.levels[0].mesh.nu))
    assert np.all(np.abs(val - ref_r) <= 1e-12 * absum + 100 * EPS64 * cscale + 1e-300)


@pytest.mark.parametrize("d,n", [(2, 8), (3, 4)])
def test_stokes_residual_equals_assembled_residual(d, n):
    pb = _sinker(d, n, 2, 1e2, 1e4, seed=9)
    H = Hierarchy(d, pb.n, pb.mu, pb.gamma)
    s = StokesSolver(H)
    lv = H.levels[-1]
    L = LocalLevel(d, lv.mesh.n, lv.coeff, pb.gamma)
    b, _ = s.rhs(pb.f, pb.u_bc)
    rng = np.random.default_rng(11)
    u = rng.standard_normal(lv.mesh.nu)
    u[lv.bdof] = 0.0
    p = rng.standard_normal(lv.mesh.npres)
    ref = np.linalg.norm(b - s.matvec(np.concatenate([u, p]))) / np.linalg.norm(b)
    assert stokes_residual(L, pb.f, u, p, chunk=7) == pytest.approx(ref, rel=1e-12)
    uo, po, its, _ = s.solve(pb.f, pb.u_bc, rtol=1e-10)
    assert stokes_residual(L, pb.f, uo, po) <= 2e-10
