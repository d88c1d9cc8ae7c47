"""Shared helpers for the GPU parity tests (torch device buffers, oracle builds)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.mg import Hierarchy  # noqa: E402
from synthetic import problems as P  # noqa: E402


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def host(t):
    return t.detach().double().cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def sinker(d, n, levels, gamma, dr, seed=0):
    if d == 2:
        return P.sinker_problem(2, n, levels, 8, 0.1, 200.0, dr, 10.0, gamma, seed)
    return P.sinker_problem(3, n, levels, 16, 0.15, 200.0, dr, 10.0, gamma, seed)


def context(pb, **opt):
    from paper_2107_00820_gb300 import Context
    return Context(pb.d, pb.n, pb.levels, pb.mu, pb.gamma, **opt)


def oracle(pb, **kw):
    return Hierarchy(pb.d, pb.n, pb.mu, pb.gamma, **kw)


def random_free(level, seed):
    v = np.random.default_rng(seed).standard_normal(level.mesh.nu)
    v[level.bdof] = 0.0
    return v
