"""Seeded synthetic inputs for the augmented-Lagrangian Stokes workloads.

This module produces DATA only: coefficient fields sampled at quadrature
points, right-hand sides, Dirichlet values and sinker centres.  It holds none
of the discretisation or solver arithmetic, so the FP64 oracle and the GPU
library can both consume what it writes without sharing any method code.

Sampling layout (the one the C ABI expects):
  * unit box (0,1)^d, n[k] uniform cells per direction, cell index with the
    x index fastest;
  * 3 points per direction inside each cell at the Gauss-Legendre abscissae
    mapped from [-1,1], point index with the x index fastest;
  * nodal arrays live on the Q2 node lattice ((2n+1) nodes per direction,
    x fastest), one array per velocity component.

Workloads follow the multi-sinker benchmark of Sec. 5.2 (viscosity and
buoyancy law, DR(mu) = mu_max/mu_min with mu_max = DR^(1/2),
mu_min = DR^(-1/2)) and the manufactured solution used for the convergence
check.  The readings of the garbled sinker formula are stated in the
repository's design notes: mu = mu_min + (mu_max - mu_min)(1 - chi) with a
squared distance in the Gaussian, sinkers are the high-viscosity,
negatively buoyant inclusions.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Gauss-Legendre abscissae on [-1, 1] for the 3-point rule; these fix WHERE
# the coefficient fields are sampled (the layout contract of the inputs).
_SAMPLE_ABSCISSAE = (-math.sqrt(0.6), 0.0, math.sqrt(0.6))


def _as_tuple(n, d):
    if np.isscalar(n):
        return (int(n),) * d
    n = tuple(int(v) for v in n)
    assert len(n) == d
    return n


def level_sizes(n, levels):
    """Cells per direction on levels 0 (coarsest) .. levels-1 (finest)."""
    out = []
    for lvl in range(levels):
        f = 2 ** (levels - 1 - lvl)
        for v in n:
            if v % f:
                raise ValueError(f"n={n} not divisible by 2^{levels - 1}")
        out.append(tuple(v // f for v in n))
    return out


def sample_points(d, n):
    """Physical coordinates of the sampling points, shape (ncells, 3^d, d)."""
    n = _as_tuple(n, d)
    g = np.asarray(_SAMPLE_ABSCISSAE)
    axes = []
    for k in range(d):
        h = 1.0 / n[k]
        c = np.arange(n[k])
        axes.append(((c[:, None] + 0.5 * (1.0 + g[None, :])) * h))  # (n_k, 3)
    # cell multi-index (x fastest) and point multi-index (x fastest)
    cells = np.stack(np.meshgrid(*[np.arange(v) for v in n], indexing="ij"), -1)
    cells = cells.transpose(*reversed(range(d)), d).reshape(-1, d)  # x fastest
    pts = np.stack(np.meshgrid(*[np.arange(3)] * d, indexing="ij"), -1)
    pts = pts.transpose(*reversed(range(d)), d).reshape(-1, d)
    x = np.empty((cells.shape[0], pts.shape[0], d))
    for k in range(d):
        x[:, :, k] = axes[k][cells[:, k][:, None], pts[:, k][None, :]]
    return x


def sample_points_k(d, n, k):
    """Physical coordinates of the (k+1)^d Gauss-Legendre points of every cell (the
    quadrature of the order-k discretisation), shape (ncells, (k+1)^d, d), cells and
    points x fastest."""
    n = _as_tuple(n, d)
    g = np.polynomial.legendre.leggauss(k + 1)[0]
    axes = [((np.arange(n[a])[:, None] + 0.5 * (1.0 + g[None, :])) / n[a]) for a in range(d)]
    cells = np.stack(np.meshgrid(*[np.arange(v) for v in n], indexing="ij"), -1)
    cells = cells.transpose(*reversed(range(d)), d).reshape(-1, d)
    pts = np.stack(np.meshgrid(*[np.arange(k + 1)] * d, indexing="ij"), -1)
    pts = pts.transpose(*reversed(range(d)), d).reshape(-1, d)
    x = np.empty((cells.shape[0], pts.shape[0], d))
    for a in range(d):
        x[:, :, a] = axes[a][cells[:, a][:, None], pts[:, a][None, :]]
    return x


def sinker_problem_k(n, levels, k, count, omega, delta, dr, beta=10.0, gamma=1e2, seed=0, d=2):
    """The multi-sinker problem in d dimensions sampled at the order-k Gauss points of every
    level (rediscretisation): mu per level [cell][(k+1)^d], f at the finest points, u_D = 0."""
    c = sinker_centres(seed, count, d)
    sizes = [tuple(v // 2 ** (levels - 1 - l) for v in _as_tuple(n, d)) for l in range(levels)]
    mus = [sinker_viscosity(sample_points_k(d, nl, k), c, omega, delta, dr) for nl in sizes]
    f = sinker_force(sample_points_k(d, n, k), c, omega, delta, beta)
    nn = tuple(k * v + 1 for v in _as_tuple(n, d))
    u_bc = np.zeros((d, int(np.prod(nn))))
    return Problem(f"sinker{d}d_q{k}", d, _as_tuple(n, d), levels, gamma, mus, f, u_bc,
                   {"centres": c, "order": k, "dr": dr})


def node_points(d, n):
    """Coordinates of the Q2 node lattice, shape ((2n+1)^d, d), x fastest."""
    n = _as_tuple(n, d)
    ax = [np.arange(2 * v + 1) * (0.5 / v) for v in n]
    grid = np.meshgrid(*ax, indexing="ij")
    return np.stack([g.transpose(*reversed(range(d))).reshape(-1) for g in grid], -1)


# ----------------------------------------------------------------------------
# multi-sinker benchmark (Sec. 5.2)
# ----------------------------------------------------------------------------
def sinker_centres(seed, count, d):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 1.0, size=(count, d))


def sinker_chi(x, centres, omega, delta):
    """chi(x) = prod_i [1 - exp(-delta * max(0, |x - c_i| - omega/2)^2)]."""
    chi = np.ones(x.shape[:-1])
    for c in centres:
        dist = np.sqrt(((x - c) ** 2).sum(-1))
        s = np.maximum(0.0, dist - 0.5 * omega)
        chi *= 1.0 - np.exp(-delta * s * s)
    return chi


def sinker_viscosity(x, centres, omega, delta, dr):
    mu_max, mu_min = math.sqrt(dr), 1.0 / math.sqrt(dr)
    chi = sinker_chi(x, centres, omega, delta)
    return mu_min + (mu_max - mu_min) * (1.0 - chi)


def sinker_force(x, centres, omega, delta, beta):
    """f = (0, .., -beta (1 - chi)): buoyancy pulling the sinkers down."""
    chi = sinker_chi(x, centres, omega, delta)
    f = np.zeros(x.shape)
    f[..., -1] = -beta * (1.0 - chi)
    return f


# ----------------------------------------------------------------------------
# manufactured solution (2D): u = (sin pi x sin pi y, cos pi x cos pi y), p = 0
# ----------------------------------------------------------------------------
def manufactured_u(x):
    px, py = math.pi * x[..., 0], math.pi * x[..., 1]
    return np.stack([np.sin(px) * np.sin(py), np.cos(px) * np.cos(py)], -1)


def manufactured_grad_u(x):
    """Exact gradient, shape (..., 2, 2), [..., comp, direction]."""
    px, py = math.pi * x[..., 0], math.pi * x[..., 1]
    g = np.empty(x.shape[:-1] + (2, 2))
    g[..., 0, 0] = math.pi * np.cos(px) * np.sin(py)
    g[..., 0, 1] = math.pi * np.sin(px) * np.cos(py)
    g[..., 1, 0] = -math.pi * np.sin(px) * np.cos(py)
    g[..., 1, 1] = -math.pi * np.cos(px) * np.sin(py)
    return g


def manufactured_f(x):
    """-div(2 eps(u)) + grad p with mu = 1, p = 0, div u = 0: f = 2 pi^2 u."""
    return 2.0 * math.pi ** 2 * manufactured_u(x)


# ----------------------------------------------------------------------------
# problem bundles
# ----------------------------------------------------------------------------
@dataclass
class Problem:
    """Everything a solve needs, for every multigrid level."""
    name: str
    d: int
    n: tuple
    levels: int
    gamma: float
    mu: list                  # per level (ncells_l, 3^d) viscosity at sample points
    f: np.ndarray             # finest level (ncells, 3^d, d) body force at sample points
    u_bc: np.ndarray          # finest level (d, N) nodal Dirichlet values (boundary read only)
    meta: dict = field(default_factory=dict)

    @property
    def level_n(self):
        return level_sizes(self.n, self.levels)


def manufactured_problem(n=16, levels=2, gamma=1e4):
    d = 2
    nn = _as_tuple(n, d)
    mus = [np.ones((int(np.prod(m)), 9)) for m in level_sizes(nn, levels)]
    xq = sample_points(d, nn)
    xn = node_points(d, nn)
    u_bc = manufactured_u(xn).T.copy()
    return Problem("manufactured_2d", d, nn, levels, float(gamma), mus,
                   manufactured_f(xq), u_bc, {"mu": 1.0})


def sinker_problem(d, n, levels, count, omega, delta, dr, beta=10.0, gamma=1e4, seed=0):
    nn = _as_tuple(n, d)
    c = sinker_centres(seed, count, d)
    mus = [sinker_viscosity(sample_points(d, m), c, omega, delta, dr)
           for m in level_sizes(nn, levels)]
    xq = sample_points(d, nn)
    f = sinker_force(xq, c, omega, delta, beta)
    u_bc = np.zeros((d, int(np.prod([2 * v + 1 for v in nn]))))
    return Problem(f"sinker_{d}d", d, nn, levels, float(gamma), mus, f, u_bc,
                   {"centres": c, "omega": omega, "delta": delta, "dr": dr,
                    "beta": beta, "seed": seed})


# ---------------------------------------------------------------------------
# serving-style batch of independent multi-sinker instances
# ---------------------------------------------------------------------------
BATCH_SIZES_2D = (16, 32, 48, 64, 96, 128, 192, 256)
BATCH_SIZES_3D = (8, 12, 16, 24, 32)


def batch_levels(n, d):
    """Largest level count L with n / 2^(L-1) an integer >= 3 (3D) or >= 4 (2D)."""
    floor = 3 if d == 3 else 4
    L = 1
    while n % (2 ** L) == 0 and n // (2 ** L) >= floor:
        L += 1
    return L


def batch_instances(count_2d=32, count_3d=32, seed=0):
    """Independent multi-sinker instances of uneven size: per instance i (seed + i)
    the mesh size from BATCH_SIZES_2D / _3D, the contrast 10^U[4,8], gamma from
    {1e2, 1e4} and the sinker centres, all drawn from the instance's own seed;
    8 sinkers (2D, omega 0.1) or 16 (3D, omega 0.15), delta 200, beta 10."""
    out = []
    for i in range(count_2d + count_3d):
        d = 2 if i < count_2d else 3
        rng = np.random.default_rng(seed + i)
        n = int(rng.choice(BATCH_SIZES_2D if d == 2 else BATCH_SIZES_3D))
        dr = float(10.0 ** rng.uniform(4.0, 8.0))
        gamma = float(rng.choice([1e2, 1e4]))
        count, omega = (8, 0.1) if d == 2 else (16, 0.15)
        pb = sinker_problem(d, n, batch_levels(n, d), count, omega, 200.0, dr, 10.0, gamma,
                            seed=1000 + seed + i)
        out.append(pb)
    return out


def sinker_2d(n=128, levels=5, gamma=1e4, dr=1e6, seed=0, count=8):
    """2D multi-sinker, 8 sinkers, omega = 0.1, delta = 200, DR = 1e6."""
    return sinker_problem(2, n, levels, count, 0.1, 200.0, dr, 10.0, gamma, seed)


def sinker_3d(n=32, levels=4, gamma=1e4, dr=1e8, seed=0, count=16):
    """3D multi-sinker, 16 sinkers, omega = 0.15, delta = 200, DR = 1e8."""
    return sinker_problem(3, n, levels, count, 0.15, 200.0, dr, 10.0, gamma, seed)


def random_vector(seed, size, lo=-1.0, hi=1.0):
    return np.random.default_rng(seed).uniform(lo, hi, size=size)


# ----------------------------------------------------------------------------
# anisotropic viscoplastic linearisation (tensor viscosity, Eq. (stokes-lin))
# ----------------------------------------------------------------------------
def _mandel(eps, d):
    """Mandel vector of symmetric tensors eps (..., d, d)."""
    r2 = math.sqrt(2.0)
    if d == 2:
        return np.stack([eps[..., 0, 0], eps[..., 1, 1], r2 * eps[..., 0, 1]], -1)
    return np.stack([eps[..., 0, 0], eps[..., 1, 1], eps[..., 2, 2],
                     r2 * eps[..., 1, 2], r2 * eps[..., 0, 2], r2 * eps[..., 0, 1]], -1)


def fourier_modes(seed, d, count=12, kmax=4):
    """Seeded wave vectors (|k|_inf <= kmax, nonzero), amplitudes and phases."""
    rng = np.random.default_rng(seed)
    ks = []
    while len(ks) < count:
        k = rng.integers(-kmax, kmax + 1, size=d)
        if np.any(k != 0):
            ks.append(k)
    ncomp = 1 if d == 2 else 3
    return np.array(ks, float), rng.standard_normal((count, ncomp)), rng.uniform(0, 2 * math.pi, count)


def solenoidal_strain_rate(x, modes):
    """sym grad v of a divergence-free field: v = (d psi/dy, -d psi/dx) in 2D,
    v = curl Psi in 3D, with psi / Psi = sum_m A_m cos(2 pi k_m . x + phi_m)."""
    ks, amps, phases = modes
    d = x.shape[-1]
    grad = np.zeros(x.shape[:-1] + (d, d))
    for k, a, ph in zip(ks, amps, phases):
        c = np.cos(2 * math.pi * (x @ k) + ph)[..., None, None]
        if d == 2:
            # psi Hessian = -(2 pi)^2 a cos k k^T; grad v rows: (psi_yx, psi_yy), (-psi_xx, -psi_xy)
            h = -(2 * math.pi) ** 2 * a[0] * np.outer(k, k)
            g = np.array([[h[1, 0], h[1, 1]], [-h[0, 0], -h[0, 1]]])
        else:
            # d_j v_i = -(2 pi)^2 cos(theta) (k x A)_i k_j
            g = -(2 * math.pi) ** 2 * np.outer(np.cross(k, a), k)
        grad = grad + c * g
    return 0.5 * (grad + np.swapaxes(grad, -1, -2))


def viscoplastic_coefficients(x, modes, scale, tau_y=1.0, alpha_max=0.99, mu_floor=1e-4,
                              layers=((1.0 / 3.0, 1e6), (2.0 / 3.0, 1e1), (math.inf, 1e-4))):
    """C = 2 mu_eff [I - alpha (e e^T)/(e.e)] (Mandel, upper triangle row-major) and mu_eff.

    mu_eff = max(mu_floor, min(mu0(x), tau_y / (2 eps_II))), eps_II = (eps:eps / 2)^(1/2),
    alpha = alpha_max (1 - mu_eff / mu0): anisotropic where the material yields.
    mu0 is layered along the last coordinate.
    """
    d = x.shape[-1]
    eps = scale * solenoidal_strain_rate(x, modes)
    e = _mandel(eps, d)
    ee = (e * e).sum(-1)
    eii = np.sqrt(0.5 * ee)
    z = x[..., -1]
    mu0 = np.full(z.shape, layers[-1][1])
    for top, val in reversed(layers):
        mu0 = np.where(z < top, val, mu0)
    with np.errstate(divide="ignore"):
        mu_eff = np.maximum(mu_floor, np.minimum(mu0, tau_y / (2.0 * eii)))
    alpha = alpha_max * (1.0 - mu_eff / mu0)
    m = e.shape[-1]
    unit = e / np.sqrt(np.maximum(ee, 1e-300))[..., None]
    C = 2.0 * mu_eff[..., None, None] * (np.eye(m) - alpha[..., None, None] * unit[..., :, None] * unit[..., None, :])
    iu = np.triu_indices(m)
    return np.ascontiguousarray(C[..., iu[0], iu[1]]), np.ascontiguousarray(mu_eff)


def viscoplastic_problem(d=3, n=48, levels=4, gamma=1e3, seed=0, rms_strain_rate=1e-4, beta=10.0):
    """Tensor-viscosity workload: per-point 4th-order C on every level, mu_eff for the
    Schur block, and a body force f = (0, .., -beta sin(2 pi x)) that is not a gradient."""
    nn = _as_tuple(n, d)
    modes = fourier_modes(seed, d)
    xf = sample_points(d, nn)
    eps = solenoidal_strain_rate(xf, modes)
    eii = np.sqrt(0.5 * (_mandel(eps, d) ** 2).sum(-1))
    scale = rms_strain_rate / math.sqrt((eii ** 2).mean())
    Cs, mus = [], []
    for m in level_sizes(nn, levels):
        C, mu = viscoplastic_coefficients(sample_points(d, m), modes, scale)
        Cs.append(C)
        mus.append(mu)
    f = np.zeros(xf.shape)
    f[..., -1] = -beta * np.sin(2.0 * math.pi * xf[..., 0])      # not a gradient: drives flow
    u_bc = np.zeros((d, int(np.prod([2 * v + 1 for v in nn]))))
    pb = Problem(f"viscoplastic_{d}d", d, nn, levels, float(gamma), Cs, f, u_bc,
                 {"seed": seed, "scale": scale, "contrast": float(np.max(mus[-1]) / np.min(mus[-1]))})
    pb.meta["mu_eff"] = mus
    return pb
