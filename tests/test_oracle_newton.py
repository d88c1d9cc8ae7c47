"""Pins of the Newton oracle for the viscoplastic rheology (oracle/newton.py, Sec. 5.3).

The linearised coefficient is checked against the derivative of the nonlinear residual
taken by central differences (a dropped term, a wrong factor or sign in the tensor fails
it, and the Picard tensor 2 mu I is shown to fail it), the rheology against its closed
forms (the stress stays below the yield stress; the tensor's spectrum), the strain-rate
evaluation at other levels' points against exact fields, and the iteration against what
Newton's method must do: one step in the viscous limit (a linear problem) and a
superlinear tail on a problem that yields."""
import numpy as np
import pytest

from oracle.fem import Level, Mesh, unpack_mandel
from oracle.newton import (ViscoplasticProblem, newton_tensor, second_invariant, strain_at_qp,
                           strain_on_level, viscosity)


def _problem(n=8, levels=2, tau_y=1.0, gamma=1e2):
    m = Mesh(2, n)
    x = m.node_coords()
    uD = np.stack([np.sin(np.pi * x[:, 0]) * np.cos(np.pi * x[:, 1]),
                   -np.cos(np.pi * x[:, 0]) * np.sin(np.pi * x[:, 1])])
    f = np.zeros((m.ncells, 9, 2))
    return ViscoplasticProblem(2, n, levels, f, uD, 1.0, tau_y, gamma)


def _random_state(pb, seed):
    rng = np.random.default_rng(seed)
    u = rng.standard_normal(pb.fine.nu)
    u[pb.bdof] = pb.uD[pb.bdof]
    return u, rng.standard_normal(pb.fine.npres)


@pytest.mark.parametrize("tau_y", [0.3, 3.0])
def test_linearisation_is_the_derivative_of_the_residual(tau_y):
    pb = _problem(tau_y=tau_y)
    u, p = _random_state(pb, 1)
    rng = np.random.default_rng(2)
    du = rng.standard_normal(pb.fine.nu)
    du[pb.bdof] = 0.0
    h = 1e-5
    fd = (pb.residual(u + h * du, p)[0] - pb.residual(u - h * du, p)[0]) / (2 * h)
    Cs, mus = pb.linearisation(u)
    J = Level(2, pb.n, Cs[-1], 0.0, kind="tensor", mu_eff=mus[-1]).A_raw
    Jd = J @ du
    Jd[pb.bdof] = 0.0
    assert np.linalg.norm(Jd - fd) <= 1e-7 * np.linalg.norm(fd)
    # negative control: the Picard tensor 2 mu I misses the derivative of mu
    C_picard = np.zeros_like(Cs[-1])
    C_picard[..., [0, 3, 5]] = 2.0 * mus[-1][..., None]
    Jp = Level(2, pb.n, C_picard, 0.0, kind="tensor", mu_eff=mus[-1]).A_raw @ du
    Jp[pb.bdof] = 0.0
    assert np.linalg.norm(Jp - fd) >= 1e-2 * np.linalg.norm(fd)


def test_rheology_closed_forms():
    mu_ref, tau_y = 2.0, 3.0
    e = np.logspace(-6, 6, 49)
    mu = viscosity(e, mu_ref, tau_y)
    tII = 2 * mu * e
    assert np.all(tII < tau_y) and tII[-1] > 0.999 * tau_y          # stress below yield, -> tau_y
    assert abs(mu[0] - mu_ref) < 1e-5 * mu_ref                          # viscous regime
    ey = tau_y / (2 * mu_ref)                                          # where the regimes meet
    assert viscosity(ey, mu_ref, tau_y) == pytest.approx(mu_ref / 2)
    assert 2 * viscosity(ey, mu_ref, tau_y) * ey == pytest.approx(tau_y / 2)


@pytest.mark.parametrize("d", [2, 3])
def test_newton_tensor_spectrum(d):
    """C = 2 mu (I - b e e^T) with tau = 2 mu eps: eigenvalue 2 mu on the complement of the
    strain's Mandel vector e and 2 mu tau_y / (2 mu_ref eps_II + tau_y) along e (SPD)."""
    rng = np.random.default_rng(d)
    mu_ref, tau_y = 1.5, 0.7
    for _ in range(5):
        M = rng.standard_normal((d, d))
        E = 0.5 * (M + M.T)
        C, mu = newton_tensor(E, mu_ref, tau_y)
        Cf = unpack_mandel(C, d)
        eII = second_invariant(E)
        w, V = np.linalg.eigh(Cf)
        small = 2 * mu * tau_y / (2 * mu_ref * eII + tau_y)
        m = Cf.shape[0]
        assert np.allclose(np.sort(w), np.sort([small] + [2 * mu] * (m - 1)), rtol=1e-12)
        from oracle.newton import mandel_vector
        ev = mandel_vector(E)
        assert abs(abs(V[:, 0] @ ev) - np.linalg.norm(ev)) < 1e-10 * np.linalg.norm(ev)


def test_strain_at_other_levels_points_is_exact_for_q2_fields():
    """A quadratic velocity is represented exactly by Q2: its strain rate evaluated at the
    Gauss points of a coarser level (points inside fine cells) is the analytic one."""
    fine = Mesh(2, 8)
    x = fine.node_coords()
    u = np.concatenate([x[:, 0] ** 2 + x[:, 0] * x[:, 1], 3 * x[:, 1] ** 2 - x[:, 0]])
    coarse = Mesh(2, 4)
    E = strain_on_level(fine, u, coarse)
    xc = (coarse.cells[:, None, :] + 0.5 * (1.0 + coarse.ref.xq[None])) * np.array(coarse.h)
    gx = np.stack([np.stack([2 * xc[..., 0] + xc[..., 1], xc[..., 0]], -1),
                   np.stack([-np.ones_like(xc[..., 0]), 6 * xc[..., 1]], -1)], -2)   # d u_a / d x_j
    ref = 0.5 * (gx + np.swapaxes(gx, -1, -2))
    assert np.allclose(E, ref, atol=1e-12)
    assert np.allclose(strain_on_level(fine, u, fine), strain_at_qp(fine, u), atol=1e-12)


def test_viscous_limit_converges_in_one_step():
    """tau_y -> infinity: mu = mu_ref, the problem is linear Stokes, one Newton step solves it."""
    pb = _problem(tau_y=1e14)
    u, p, hist, lin = pb.solve(rtol=1e-9, maxit=3)
    assert len(hist) == 2 and hist[-1] <= 1e-9 * hist[0], hist


def test_newton_converges_superlinearly_when_yielding():
    pb = _problem(tau_y=1.0)
    u, p, hist, lin = pb.solve(rtol=1e-10, maxit=25)
    assert hist[-1] <= 1e-10 * hist[0], hist
    m = pb.fine
    eII = second_invariant(strain_at_qp(m, u))
    mu = viscosity(eII, 1.0, 1.0)
    assert mu.min() < 0.5                                    # part of the domain has yielded
    r = np.array(hist) / hist[0]
    tail = [k for k in range(1, len(r) - 1) if r[k] < 1e-2]
    assert tail, r
    k = tail[0]
    assert r[k + 1] <= 10 * r[k] ** 1.5, r                    # faster than linear near the solution
    assert np.linalg.norm(pb.residual(u, p)[1]) <= 1e-9 * hist[0]
