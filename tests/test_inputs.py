"""The seeded input generators (synthetic/problems.py) against the input recipe.

The generators hold no method arithmetic; these tests check that what they produce is
what the recipe states: the multi-sinker law of Sec. 5.2 sampled at every level's own
Gauss points (rediscretisation), the tensor workload's divergence-free strain rate, RMS
scale, layered reference viscosity, yield cap and SPD Mandel tensor, and the batch's
size, level, contrast and gamma draws; all of it reproducible from the seed."""
import math

import numpy as np
import pytest

from oracle.fem import unpack_mandel
from synthetic import problems as P


def test_sinker_law_and_rediscretisation():
    dr, beta = 1e6, 10.0
    pb = P.sinker_problem(2, 16, 3, 3, 0.1, 200.0, dr, beta, 1.0, seed=5)
    c = P.sinker_centres(5, 3, 2)
    mu_max, mu_min = math.sqrt(dr), 1.0 / math.sqrt(dr)
    # a sinker centre carries mu_max (the sinkers are the viscous inclusions), far away mu_min
    assert P.sinker_viscosity(c[:1][None], c, 0.1, 200.0, dr)[0, 0] == pytest.approx(mu_max)
    for lvl, n in enumerate(P.level_sizes((16, 16), 3)):
        mu = pb.mu[lvl]
        assert mu.shape == (n[0] * n[1], 9)
        assert np.array_equal(mu, P.sinker_viscosity(P.sample_points(2, n), c, 0.1, 200.0, dr))
        assert mu.min() >= mu_min * (1 - 1e-12) and mu.max() <= mu_max * (1 + 1e-12)
    # force (0, -beta (1 - chi)) at the finest Gauss points: 0 in x, -beta (mu - mu_min)/(mu_max - mu_min) in y
    assert not pb.f[..., 0].any()
    assert np.allclose(pb.f[..., 1], -beta * (pb.mu[-1] - mu_min) / (mu_max - mu_min), rtol=1e-12, atol=1e-12)
    assert not pb.u_bc.any()
    again = P.sinker_problem(2, 16, 3, 3, 0.1, 200.0, dr, beta, 1.0, seed=5)
    assert all(np.array_equal(a, b) for a, b in zip(pb.mu, again.mu)) and np.array_equal(pb.f, again.f)
    other = P.sinker_problem(2, 16, 3, 3, 0.1, 200.0, dr, beta, 1.0, seed=6)
    assert not np.array_equal(pb.mu[-1], other.mu[-1])


@pytest.mark.parametrize("d,n", [(2, 8), (3, 4)])
def test_viscoplastic_recipe(d, n):
    pb = P.viscoplastic_problem(d, n, 2, 1e3, seed=2)
    m = 3 if d == 2 else 6
    x = P.sample_points(d, (n,) * d)
    modes = P.fourier_modes(2, d)
    eps = pb.meta["scale"] * P.solenoidal_strain_rate(x, modes)
    # the strain rate of a divergence-free field is trace free
    tr = np.trace(eps, axis1=-2, axis2=-1)
    assert np.abs(tr).max() <= 1e-12 * np.abs(eps).max()
    eii = np.sqrt(0.5 * (eps * eps).sum((-1, -2)))
    assert math.sqrt((eii ** 2).mean()) == pytest.approx(1e-4, rel=1e-12)       # RMS eps_II at the finest points
    mu = pb.meta["mu_eff"][-1]
    z = x[..., -1]
    mu0 = np.where(z < 1 / 3, 1e6, np.where(z < 2 / 3, 1e1, 1e-4))
    assert np.allclose(mu, np.maximum(1e-4, np.minimum(mu0, 1.0 / (2 * eii))), rtol=1e-12)
    assert pb.meta["contrast"] == pytest.approx(mu.max() / mu.min())
    C = unpack_mandel(pb.mu[-1], d)
    assert np.allclose(C, np.swapaxes(C, -1, -2))
    alpha = 0.99 * (1 - mu / mu0)
    w = np.linalg.eigvalsh(C)
    # C = 2 mu_eff (I - alpha e e^T / |e|^2): eigenvalues 2 mu_eff (1 - alpha) once and 2 mu_eff
    assert np.allclose(w[..., 0], 2 * mu * (1 - alpha), rtol=1e-9)
    assert np.allclose(w[..., 1:], 2 * mu[..., None] * np.ones(m - 1), rtol=1e-9)
    assert (w > 0).all()
    assert (alpha > 0).any() and (alpha == 0).any()          # yields in part of the domain only
    assert not pb.u_bc.any() and np.allclose(pb.f[..., -1], -10.0 * np.sin(2 * math.pi * x[..., 0]))


def test_batch_instances_recipe():
    inst = P.batch_instances(4, 4, seed=3)
    assert [pb.d for pb in inst] == [2] * 4 + [3] * 4
    for pb in inst:
        n = pb.n[0]
        assert n in (P.BATCH_SIZES_2D if pb.d == 2 else P.BATCH_SIZES_3D)
        floor = 4 if pb.d == 2 else 3
        L = pb.levels
        assert n % 2 ** (L - 1) == 0 and n // 2 ** (L - 1) >= floor
        assert not (n % 2 ** L == 0 and n // 2 ** L >= floor)        # the largest such L
        mu = pb.mu[-1]
        dr = mu.max() / mu.min()
        assert 1e4 * (1 - 1e-9) <= pb.meta["dr"] <= 1e8 * (1 + 1e-9) and dr <= pb.meta["dr"] * (1 + 1e-9)
        assert pb.gamma in (1e2, 1e4)
    again = P.batch_instances(4, 4, seed=3)
    assert all(np.array_equal(a.mu[-1], b.mu[-1]) and a.gamma == b.gamma for a, b in zip(inst, again))
