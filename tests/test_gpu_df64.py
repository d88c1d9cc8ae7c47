"""Mixed mode assembles and inverts the vertex-star patches and the coarse operator in
double-float arithmetic (FP32 pairs, unit roundoff about 2^-48).  These tests pin that
path directly against LAPACK on the oracle's assembled matrices: the inverse may differ
from the exact one by a small multiple of cond * 2^-48 (FP64: cond * 2^-53), scalar and
tensor coefficients, and the coarse solve likewise."""
import numpy as np
import pytest

from gpu_helpers import context, dev, host, oracle, random_free, sinker, torch  # noqa: F401
from test_gpu_parity import _patch_cond, _tensor_ctx, _tensor_oracle, _tensor_problem, all_vertices

from paper_2107_00820_gb300 import alstokes as A  # noqa: E402

pytestmark = pytest.mark.gpu

U_DF = 2.0 ** -48


def _check_patches(ctx, H, d, picks, factor):
    m = H.levels[1].mesh
    verts = all_vertices(m)
    NB = 3 ** d
    worst = 0.0
    for vid in picks:
        v = verts[vid]
        cond, idx, Av = _patch_cond(H, 1, v)
        full = ctx.patch_inverse(1, int(vid))
        keep = [a * NB + o for a in range(d) for o in range(NB)
                if np.all((g := 2 * v + (np.array([o % 3, (o // 3) % 3, o // 9][:d]) - 1)) > 0)
                and np.all(g < np.array(m.nn) - 1)]
        got = full[np.ix_(keep, keep)]
        ref = np.linalg.inv(Av)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= max(1e-13, factor * cond * U_DF), (vid, cond, err)
        worst = max(worst, err / (cond * U_DF))
    return worst


@pytest.mark.parametrize("d,n,gamma,dr,schur", [(2, 8, 1e2, 1e6, A.ALS_SCHUR_P1), (2, 8, 1e4, 1e6, A.ALS_SCHUR_P2),
                                                (3, 4, 1e2, 1e4, A.ALS_SCHUR_P1), (3, 4, 1e3, 1e8, A.ALS_SCHUR_P2)])
def test_mixed_patch_inverses_double_float(d, n, gamma, dr, schur):
    """(Mixed mode refuses the P1 pairing beyond 2^-24 gamma / mu_min = 0.1, so the extreme
    cases use P2, whose augmentation weight W = M_p(1/mu) enters the patch matrices.)"""
    pb = sinker(d, n, 2, gamma, dr, seed=61)
    ctx = context(pb, mode=A.ALS_MODE_MIXED, schur=schur)
    H = oracle(pb, smoother="richardson", steps=1, W="Mp_mu" if schur == A.ALS_SCHUR_P2 else "Mp")
    nverts = len(all_vertices(H.levels[1].mesh))
    picks = list(np.random.default_rng(62).choice(nverts, size=min(12, nverts), replace=False)) + [0, nverts - 1]
    _check_patches(ctx, H, d, picks, 40.0)


@pytest.mark.parametrize("d,n", [(2, 12), (3, 4)])
def test_mixed_tensor_patch_inverses_double_float(d, n):
    pb = _tensor_problem(d, n, 2, 1e2)
    ctx = _tensor_ctx(pb, mode=A.ALS_MODE_MIXED)
    H = _tensor_oracle(pb, smoother="richardson", steps=1)
    nverts = len(all_vertices(H.levels[1].mesh))
    picks = list(np.random.default_rng(63).choice(nverts, size=10, replace=False)) + [0]
    _check_patches(ctx, H, d, picks, 40.0)


@pytest.mark.parametrize("d,n,levels", [(2, 16, 3), (3, 8, 2)])
def test_mixed_coarse_solve_double_float(d, n, levels):
    """The coarse inverse of a mixed context (double-float sweep) applied in FP64 meets the
    oracle's dense coarse solve within a small multiple of cond * 2^-48."""
    pb = sinker(d, n, levels, 1e2, dr=1e6, seed=64)
    ctx = context(pb, mode=A.ALS_MODE_MIXED)
    H = oracle(pb)
    lv0 = H.levels[0]
    b = random_free(lv0, 65)
    x = torch.zeros_like(dev(b))
    ctx.coarse_solve(dev(b), x, A.ALS_PREC_FP64)
    ref = H.coarse_solve(b)
    f = np.flatnonzero(lv0.free)
    cond = np.linalg.cond(lv0.A.toarray()[np.ix_(f, f)])
    err = np.linalg.norm(host(x) - ref) / np.linalg.norm(ref)
    assert err <= max(1e-13, 100 * cond * U_DF), (err, cond)
